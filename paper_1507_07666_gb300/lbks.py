"""ctypes binding of liblbks (include/lbks.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions carry the C names; device arrays are passed as torch CUDA tensors
(their data pointers), streams as torch.cuda.Stream or raw handles.  If the
shared library is missing the import fails: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbks.so")

MAX_ORB = 64
OK, EINVAL, ENOMEM, ENOTCONV, ETIMEDOUT, EBUSY, ECUDA, ENOTFOUND = range(8)
FP64, FP32, BF16 = 0, 1, 2
STORE_POPULATIONS, STORE_PSI = 0, 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1507_07666_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)


class LbksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbks error {code}: {msg}")
        self.code = code


class lbks_params(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("theta", ctypes.c_double), ("n_inner", ctypes.c_int),
                ("mix", ctypes.c_double), ("e_tol", ctypes.c_double), ("max_cycles", ctypes.c_int),
                ("precision", ctypes.c_int), ("softening", ctypes.c_double),
                ("poisson_rtol", ctypes.c_double), ("poisson_max_iter", ctypes.c_int),
                ("polish_tol", ctypes.c_double), ("storage", ctypes.c_int), ("eig_tol", ctypes.c_double),
                ("rho_tol", ctypes.c_double), ("seed", ctypes.c_uint64), ("poisson_adapt", ctypes.c_double)]


class lbks_result(ctypes.Structure):
    _fields_ = [("E_total", ctypes.c_double), ("dE", ctypes.c_double),
                ("eigenvalues", ctypes.c_double * MAX_ORB), ("n_electrons", ctypes.c_double),
                ("cycles", ctypes.c_int), ("steps", ctypes.c_int), ("converged", ctypes.c_int),
                ("poisson_iters", ctypes.c_int), ("wall_s", ctypes.c_double), ("d_eig", ctypes.c_double),
                ("d_rho", ctypes.c_double), ("err_E", ctypes.c_double), ("err_eig", ctypes.c_double),
                ("err_rho", ctypes.c_double), ("poisson_s", ctypes.c_double)]


class lbks_energy_terms(ctypes.Structure):
    _fields_ = [("T_s", ctypes.c_double), ("E_ext", ctypes.c_double), ("E_H", ctypes.c_double),
                ("E_xc", ctypes.c_double), ("E_nn", ctypes.c_double), ("E_total", ctypes.c_double),
                ("eigenvalues", ctypes.c_double * MAX_ORB), ("orbital_energies", ctypes.c_double * MAX_ORB),
                ("n_electrons", ctypes.c_double)]


class lbks_request(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("n_orb", ctypes.c_int), ("n_atoms", ctypes.c_int), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("Z", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int), ("n_inner", ctypes.c_int),
                ("e_tol", ctypes.c_double), ("max_cycles", ctypes.c_int)]


class lbks_timing(ctypes.Structure):
    _fields_ = [("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double)]


class lbks_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("running", ctypes.c_int), ("pooled", ctypes.c_int),
                ("completed", ctypes.c_uint64), ("bytes_in_use", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t)]


class lbks_cd_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("kappa", ctypes.c_double), ("n_pot", ctypes.c_int)]


_vp, _d, _i, _sz = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "lbks_params_default": (None, [ctypes.POINTER(lbks_params)]),
    "lbks_last_error": (_i, [ctypes.c_char_p, _sz]),
    "lbks_version": (ctypes.c_char_p, []),
    "lbks_kernel_launches": (ctypes.c_uint64, []),
    "lbks_set_wait_limit": (ctypes.c_uint32, [ctypes.c_uint32]),
    "lbks_wait_timeouts": (ctypes.c_uint64, []),
    "lbks_create_system": (_i, [ctypes.POINTER(lbks_params), _i, _i, _i, _d, _i, ctypes.POINTER(_vp)]),
    "lbks_destroy_system": (_i, [_vp]),
    "lbks_system_bytes": (_sz, [ctypes.POINTER(lbks_params), _i, _i, _i, _i]),
    "lbks_set_geometry": (_i, [_vp, _i, _dp, _dp]),
    "lbks_create_batch": (_i, [ctypes.POINTER(lbks_params), _i, _i, _i, _d, _i, _i, ctypes.POINTER(_vp)]),
    "lbks_batch_bytes": (_sz, [ctypes.POINTER(lbks_params), _i, _i, _i, _i, _i]),
    "lbks_batch_set_geometry": (_i, [_vp, _i, _i, _dp, _dp]),
    "lbks_batch_init": (_i, [_vp]),
    "lbks_batch_scf": (_i, [_vp, _vp, ctypes.POINTER(lbks_result)]),
    "lbks_batch_energy": (_i, [_vp, _i, ctypes.POINTER(lbks_energy_terms)]),
    "lbks_batch_get_density": (_i, [_vp, _i, _dp, _sz]),
    "lbks_scf": (_i, [_vp, _vp, ctypes.POINTER(lbks_result)]),
    "lbks_scf_cycles": (_i, [_vp, _i, _vp, ctypes.POINTER(lbks_result)]),
    "lbks_energy": (_i, [_vp, ctypes.POINTER(lbks_energy_terms)]),
    "lbks_forces": (_i, [_vp, _dp, _sz]),
    "lbks_batch_forces": (_i, [_vp, _i, _dp, _sz]),
    "lbks_move_atoms": (_i, [_vp, _dp]),
    "lbks_md": (_i, [_vp, _i, _d, _dp, _dp, _vp, _dp, _dp]),
    "lbks_relax_geometry": (_i, [_vp, _i, _d, _d, ctypes.POINTER(_i), _vp, ctypes.POINTER(lbks_result), _dp,
                                 ctypes.POINTER(_i)]),
    "lbks_get_density": (_i, [_vp, _dp, _sz]),
    "lbks_get_orbitals": (_i, [_vp, _dp, _sz]),
    "lbks_get_potential": (_i, [_vp, _i, _dp, _sz]),
    "lbks_server_create": (_i, [ctypes.POINTER(lbks_params), _sz, _i, ctypes.POINTER(_vp)]),
    "lbks_server_destroy": (_i, [_vp]),
    "lbks_submit": (_i, [_vp, ctypes.POINTER(lbks_request), ctypes.POINTER(ctypes.c_uint64)]),
    "lbks_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(lbks_result), ctypes.POINTER(lbks_timing),
                       ctypes.POINTER(_i)]),
    "lbks_server_wait": (_i, [_vp, ctypes.c_uint64, _d]),
    "lbks_server_get_stats": (_i, [_vp, ctypes.POINTER(lbks_server_stats)]),
    "lbks_relax_step": (_i, [_i, _i, _i, _i, _i, _d, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                             _vp]),
    "lbks_relax_step_psi": (_i, [_i, _i, _i, _i, _i, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lbks_relax_step_noalloc": (_i, [_i, _i, _i, _i, _i, _d, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp]),
    "lbks_w_field": (_i, [_i, _sz, _i, _d, _vp, _vp, _vp, _vp]),
    "lbks_energy_matrix": (_i, [_i, _i, _i, _i, _i, _d, _d, _vp, _vp, _vp, _vp]),
    "lbks_overlap": (_i, [_i, _sz, _i, _d, _vp, _vp, _i, _vp]),
    "lbks_set_relax_variant": (_i, [_i]),
    "lbks_get_relax_variant": (_i, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "lbks_cholesky_inverse": (_i, [_i, _vp, _vp, _vp, _vp]),
    "lbks_orth_apply": (_i, [_i, _sz, _i, _vp, _vp, _vp, _vp]),
    "lbks_hartree": (_i, [_i, _i, _i, _d, _vp, _vp, _d, _i, ctypes.POINTER(_i), _dp, _vp]),
    "lbks_lda": (_i, [_sz, _vp, _vp, _vp, _vp]),
    "lbks_cd_start": (_i, [_vp, ctypes.POINTER(lbks_cd_params), _dp, _vp, _dp]),
    "lbks_cd_run": (_i, [_vp, _i, _dp, _dp, _vp, _dp, _dp]),
    "lbks_cd_get_orbitals": (_i, [_vp, _i, _dp, _sz]),
    "lbks_cd_get_state": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_int64), _dp, _sz]),
    "lbks_cd_step": (_i, [_i, _i, _i, _i, _i, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lbks_cd_overlap": (_i, [_i, _sz, _i, _d, _vp, _vp, _vp, _vp]),
    "lbks_set_cd_kernel": (_i, [_i]),
    "lbks_set_psi_tile": (_i, [_i]),
    "lbks_get_psi_tile": (_i, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    _lib.lbks_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(code):
    if code != OK:
        raise LbksError(code, last_error())
    return code


def _ptr(t, dtype=None, optional=False):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        if optional:
            return None
        raise ValueError("tensor required")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _tdtype(precision):
    """torch dtype of stored populations."""
    import torch
    return {FP64: torch.float64, FP32: torch.float32, BF16: torch.bfloat16}[precision]


def _psitype(precision):
    """torch dtype of orbitals and the W field (the compute type)."""
    import torch
    return torch.float64 if precision == FP64 else torch.float32


# ------------------------------------------------------------------ functions
def lbks_params_default(**overrides) -> lbks_params:
    p = lbks_params()
    _lib.lbks_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def lbks_version() -> str:
    return _lib.lbks_version().decode()


def lbks_kernel_launches() -> int:
    return int(_lib.lbks_kernel_launches())


def lbks_set_wait_limit(polls: int) -> int:
    return int(_lib.lbks_set_wait_limit(int(polls)))


def lbks_wait_timeouts() -> int:
    return int(_lib.lbks_wait_timeouts())


def lbks_system_bytes(params, nx, ny, nz, n_orb) -> int:
    return int(_lib.lbks_system_bytes(ctypes.byref(params), nx, ny, nz, n_orb))


def lbks_create_system(params, nx, ny, nz, h, n_orb):
    handle = ctypes.c_void_p()
    _check(_lib.lbks_create_system(ctypes.byref(params), nx, ny, nz, h, n_orb, ctypes.byref(handle)))
    return handle


def lbks_destroy_system(handle):
    _check(_lib.lbks_destroy_system(handle))


def lbks_set_geometry(handle, xyz, Z):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    Z = np.ascontiguousarray(Z, dtype=np.float64).ravel()
    _check(_lib.lbks_set_geometry(handle, len(Z), xyz.ctypes.data_as(_dp), Z.ctypes.data_as(_dp)))


def _result_dict(r: lbks_result, n_orb: int) -> dict:
    return {"E_total": r.E_total, "dE": r.dE, "eigenvalues": np.array(r.eigenvalues[:n_orb]),
            "n_electrons": r.n_electrons, "cycles": r.cycles, "steps": r.steps,
            "converged": bool(r.converged), "poisson_iters": r.poisson_iters, "wall_s": r.wall_s,
            "d_eig": r.d_eig, "d_rho": r.d_rho, "err_E": r.err_E, "err_eig": r.err_eig, "err_rho": r.err_rho,
            "poisson_s": r.poisson_s}


def lbks_scf(handle, stream=None, n_orb=MAX_ORB, allow_notconv=False) -> dict:
    r = lbks_result()
    code = _lib.lbks_scf(handle, _stream(stream), ctypes.byref(r))
    if code != OK and not (allow_notconv and code == ENOTCONV):
        _check(code)
    return _result_dict(r, n_orb)


def lbks_scf_cycles(handle, n, stream=None, n_orb=MAX_ORB) -> dict:
    r = lbks_result()
    _check(_lib.lbks_scf_cycles(handle, n, _stream(stream), ctypes.byref(r)))
    return _result_dict(r, n_orb)


def lbks_energy(handle, n_orb=MAX_ORB) -> dict:
    t = lbks_energy_terms()
    _check(_lib.lbks_energy(handle, ctypes.byref(t)))
    return {"T_s": t.T_s, "E_ext": t.E_ext, "E_H": t.E_H, "E_xc": t.E_xc, "E_nn": t.E_nn,
            "E_total": t.E_total, "eigenvalues": np.array(t.eigenvalues[:n_orb]),
            "orbital_energies": np.array(t.orbital_energies[:n_orb]), "n_electrons": t.n_electrons}


def lbks_forces(handle, n_atoms):
    out = np.empty((n_atoms, 3), dtype=np.float64)
    _check(_lib.lbks_forces(handle, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_batch_forces(handle, system, n_atoms):
    out = np.empty((n_atoms, 3), dtype=np.float64)
    _check(_lib.lbks_batch_forces(handle, system, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_move_atoms(handle, xyz):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    _check(_lib.lbks_move_atoms(handle, xyz.ctypes.data_as(_dp)))


def lbks_md(handle, n_steps, dt, masses, velocities, stream=None):
    """Returns (velocities after, energies [n_steps + 1, 2], positions [n_steps + 1, n_atoms, 3])."""
    masses = np.ascontiguousarray(masses, dtype=np.float64).ravel()
    v = np.ascontiguousarray(velocities, dtype=np.float64).reshape(-1, 3).copy()
    e = np.empty((n_steps + 1, 2), dtype=np.float64)
    traj = np.empty((n_steps + 1, len(masses), 3), dtype=np.float64)
    _check(_lib.lbks_md(handle, n_steps, dt, masses.ctypes.data_as(_dp), v.ctypes.data_as(_dp), _stream(stream),
                        e.ctypes.data_as(_dp), traj.ctypes.data_as(_dp)))
    return v, e, traj


def lbks_cd_start(handle, tau=0.0, kappa=0.0, n_pot=0, E_target=None, stream=None):
    """Starts the concurrent dynamics from the handle's orbitals; returns
    (E_total, n_electrons) of the start."""
    p = lbks_cd_params(tau, kappa, n_pot)
    E = None if E_target is None else np.ascontiguousarray(E_target, dtype=np.float64)
    out = np.empty(2, dtype=np.float64)
    _check(_lib.lbks_cd_start(handle, ctypes.byref(p), None if E is None else E.ctypes.data_as(_dp),
                              _stream(stream), out.ctypes.data_as(_dp)))
    return float(out[0]), float(out[1])


def lbks_cd_run(handle, n_blocks, n_atoms, masses=None, velocities=None, stream=None):
    """Returns (velocities after or None, energies [n_blocks, 3] = (E_total,
    E_kin nuclei, n_electrons), positions [n_blocks, n_atoms, 3])."""
    m = None if masses is None else np.ascontiguousarray(masses, dtype=np.float64).ravel()
    v = None
    if velocities is not None:
        v = np.ascontiguousarray(velocities, dtype=np.float64).reshape(-1, 3).copy()
    elif m is not None:
        v = np.zeros((n_atoms, 3))
    e = np.empty((max(n_blocks, 1), 3), dtype=np.float64)
    traj = np.empty((max(n_blocks, 1), n_atoms, 3), dtype=np.float64)
    _check(_lib.lbks_cd_run(handle, n_blocks, None if m is None else m.ctypes.data_as(_dp),
                            None if v is None else v.ctypes.data_as(_dp), _stream(stream), e.ctypes.data_as(_dp),
                            traj.ctypes.data_as(_dp)))
    return v, e[:n_blocks], traj[:n_blocks]


def lbks_cd_get_orbitals(handle, level, n_orb, shape):
    """Complex orbitals [n_orb, nz, ny, nx] of level 0 (older) or 1 (current)."""
    out = np.empty((n_orb, 2) + tuple(shape), dtype=np.float64)
    _check(_lib.lbks_cd_get_orbitals(handle, level, out.ctypes.data_as(_dp), out.size))
    return out[:, 0] + 1j * out[:, 1]


def lbks_cd_get_state(handle, n_atoms):
    t, steps = ctypes.c_double(), ctypes.c_int64()
    F = np.empty((n_atoms, 3), dtype=np.float64)
    _check(_lib.lbks_cd_get_state(handle, ctypes.byref(t), ctypes.byref(steps), F.ctypes.data_as(_dp), F.size))
    return {"time": t.value, "steps": steps.value, "forces": F}


def lbks_cd_step(precision, nx, ny, nz, n_orb, h, theta, tau, phi_prev, phi, V, lam, u_coef, phi_next, S_next=None,
                 lam_next=None, stream=None):
    """phi tensors: [n_orb, 2, nz, ny, nx] of the compute type (real, imaginary planes)."""
    import torch
    P = _psitype(precision)
    _check(_lib.lbks_cd_step(precision, nx, ny, nz, n_orb, h, theta, tau, _ptr(phi_prev, P, optional=True),
                             _ptr(phi, P), _ptr(V, torch.float64), _ptr(lam, torch.float64, optional=True),
                             _ptr(u_coef, torch.float64, optional=True), _ptr(phi_next, P),
                             _ptr(S_next, torch.float64, optional=True), _ptr(lam_next, torch.float64, optional=True),
                             _stream(stream)))


def lbks_set_cd_kernel(mode):
    """-1 automatic, 0 one site per thread, 1 staged; returns the previous mode."""
    code = _lib.lbks_set_cd_kernel(mode)
    if code < -1:
        raise LbksError(EINVAL, last_error())
    return code


def lbks_cd_overlap(precision, n_sites, n_orb, h, phi, S, lam=None, stream=None):
    import torch
    _check(_lib.lbks_cd_overlap(precision, n_sites, n_orb, h, _ptr(phi, _psitype(precision)), _ptr(S, torch.float64),
                                _ptr(lam, torch.float64, optional=True), _stream(stream)))


def lbks_relax_geometry(handle, n_atoms, max_steps, fmax, step, stream=None, n_orb=MAX_ORB, allow_notconv=False,
                        fixed=None):
    r = lbks_result()
    xyz = np.empty((n_atoms, 3), dtype=np.float64)
    steps = ctypes.c_int()
    fx = None
    if fixed is not None:
        fx = (ctypes.c_int * n_atoms)(*[1 if f else 0 for f in fixed])
    code = _lib.lbks_relax_geometry(handle, max_steps, fmax, step, fx, _stream(stream), ctypes.byref(r),
                                    xyz.ctypes.data_as(_dp), ctypes.byref(steps))
    if code != OK and not (allow_notconv and code == ENOTCONV):
        _check(code)
    out = _result_dict(r, n_orb)
    out.update({"xyz": xyz, "moves": steps.value, "relaxed": code == OK})
    return out


def lbks_get_density(handle, shape):
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.lbks_get_density(handle, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_get_orbitals(handle, shape):
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.lbks_get_orbitals(handle, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_get_potential(handle, which, shape):
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.lbks_get_potential(handle, which, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_relax_step(precision, nx, ny, nz, n_orb, h, omega, theta, dt, f_in, u_in, V, sigma_in, f_out,
                    psi_out, S_out, lambda_out, sigma_out, stream=None):
    import torch
    T, P = _tdtype(precision), _psitype(precision)
    _check(_lib.lbks_relax_step(precision, nx, ny, nz, n_orb, h, omega, theta, dt, _ptr(f_in, T),
                                _ptr(u_in, P, optional=True), _ptr(V, torch.float64),
                                _ptr(sigma_in, torch.float64), _ptr(f_out, T), _ptr(psi_out, P),
                                _ptr(S_out, torch.float64), _ptr(lambda_out, torch.float64),
                                _ptr(sigma_out, torch.float64), _stream(stream)))


def lbks_relax_step_psi(precision, nx, ny, nz, n_orb, h, theta, dt, psi_in, lambda_in, Vc, sigma_in, psi_out,
                        S_out, lambda_out, sigma_out, stream=None):
    import torch
    P = _psitype(precision)
    _check(_lib.lbks_relax_step_psi(precision, nx, ny, nz, n_orb, h, theta, dt, _ptr(psi_in, P),
                                    _ptr(lambda_in, torch.float64, optional=True), _ptr(Vc, torch.float64),
                                    _ptr(sigma_in, torch.float64), _ptr(psi_out, P), _ptr(S_out, torch.float64),
                                    _ptr(lambda_out, torch.float64), _ptr(sigma_out, torch.float64),
                                    _stream(stream)))


def lbks_relax_step_noalloc(precision, nx, ny, nz, n_orb, h, omega, theta, dt, f_in, u_in, V, sigma_in, f_out,
                            psi_out, S_out, lambda_out, sigma_out, stream=None):
    """As lbks_relax_step, with the reduction scratch in the library's fixed
    device array (nothing is allocated; overlapping calls race)."""
    import torch
    T, P = _tdtype(precision), _psitype(precision)
    _check(_lib.lbks_relax_step_noalloc(precision, nx, ny, nz, n_orb, h, omega, theta, dt, _ptr(f_in, T),
                                        _ptr(u_in, P, optional=True), _ptr(V, torch.float64),
                                        _ptr(sigma_in, torch.float64), _ptr(f_out, T), _ptr(psi_out, P),
                                        _ptr(S_out, torch.float64), _ptr(lambda_out, torch.float64),
                                        _ptr(sigma_out, torch.float64), _stream(stream)))


def lbks_w_field(precision, n_sites, n_orb, omega, psi, lam, u_out, stream=None):
    import torch
    P = _psitype(precision)
    _check(_lib.lbks_w_field(precision, n_sites, n_orb, omega, _ptr(psi, P), _ptr(lam, torch.float64),
                             _ptr(u_out, P, optional=True), _stream(stream)))


def lbks_energy_matrix(precision, nx, ny, nz, n_orb, h, theta, psi, V, out, stream=None):
    import torch
    _check(_lib.lbks_energy_matrix(precision, nx, ny, nz, n_orb, h, theta, _ptr(psi, _psitype(precision)),
                                   _ptr(V, torch.float64), _ptr(out, torch.float64), _stream(stream)))


def lbks_overlap(precision, n_sites, n_orb, h, psi, S, tensor_cores=False, stream=None):
    import torch
    _check(_lib.lbks_overlap(precision, n_sites, n_orb, h, _ptr(psi, _psitype(precision)), _ptr(S, torch.float64),
                             int(bool(tensor_cores)), _stream(stream)))


RELAX_VARIANTS = ("sites", "pairs", "prefetch", "bulk")


def lbks_set_relax_variant(mode: int) -> int:
    """0: tuned per shape (default); 1 + v: variant v of RELAX_VARIANTS forced. Returns the previous mode."""
    prev = _lib.lbks_set_relax_variant(int(mode))
    if prev < 0:
        raise LbksError(EINVAL, f"bad relax variant mode {mode}")
    return prev


def lbks_get_relax_variant(handle) -> dict:
    v, ms = ctypes.c_int(), (ctypes.c_double * len(RELAX_VARIANTS))()
    _check(_lib.lbks_get_relax_variant(handle, ctypes.byref(v), ms))
    out = {"variant": RELAX_VARIANTS[v.value], "index": v.value}
    out.update({f"ms_{name}": ms[k] for k, name in enumerate(RELAX_VARIANTS)})
    return out


# staged orbital-storage stencil tile shapes (x, y, z sites), the sites per thread of each and
# whether it sums by velocity class from per-plane sums
PSI_TILES = ((32, 8, 4), (32, 8, 8), (64, 4, 4), (32, 8, 2), (64, 8, 4), (64, 8, 2), (32, 8, 8), (32, 8, 4))
PSI_TILE_SITES_PER_THREAD = (1, 1, 1, 1, 2, 2, 1, 1)
PSI_TILE_PLANE_SUMS = (False, False, False, False, False, False, True, True)


def lbks_set_psi_tile(shape):
    """-1: tuned per grid shape; 0..7: forced (PSI_TILES).  Returns the previous setting."""
    code = _lib.lbks_set_psi_tile(shape)
    if code < -1:
        raise LbksError(EINVAL, last_error())
    return code


def lbks_get_psi_tile(handle) -> dict:
    sh, ms = ctypes.c_int(), (ctypes.c_double * len(PSI_TILES))()
    _check(_lib.lbks_get_psi_tile(handle, ctypes.byref(sh), ms))
    return {"shape": sh.value, "tile": PSI_TILES[sh.value], "ms": [ms[k] for k in range(len(PSI_TILES))]}


def lbks_cholesky_inverse(n, S, Linv, status, stream=None):
    import torch
    _check(_lib.lbks_cholesky_inverse(n, _ptr(S, torch.float64), _ptr(Linv, torch.float64),
                                      _ptr(status, torch.int32), _stream(stream)))


def lbks_orth_apply(precision, n_sites, n_orb, Linv, f, psi, stream=None):
    import torch
    T, P = _tdtype(precision), _psitype(precision)
    _check(_lib.lbks_orth_apply(precision, n_sites, n_orb, _ptr(Linv, torch.float64), _ptr(f, T, optional=True),
                                _ptr(psi, P, optional=True), _stream(stream)))


def lbks_hartree(nx, ny, nz, h, rho, v, rtol=1e-11, max_iter=20000, stream=None):
    import torch
    it = ctypes.c_int()
    rr = ctypes.c_double()
    _check(_lib.lbks_hartree(nx, ny, nz, h, _ptr(rho, torch.float64), _ptr(v, torch.float64), rtol, max_iter,
                             ctypes.byref(it), ctypes.byref(rr), _stream(stream)))
    return it.value, rr.value


def lbks_lda(n_sites, rho, eps, v, stream=None):
    import torch
    _check(_lib.lbks_lda(n_sites, _ptr(rho, torch.float64), _ptr(eps, torch.float64), _ptr(v, torch.float64),
                         _stream(stream)))


def lbks_create_batch(params, nx, ny, nz, h, n_orb, n_systems):
    handle = ctypes.c_void_p()
    _check(_lib.lbks_create_batch(ctypes.byref(params), nx, ny, nz, h, n_orb, n_systems, ctypes.byref(handle)))
    return handle


def lbks_batch_bytes(params, nx, ny, nz, n_orb, n_systems) -> int:
    return int(_lib.lbks_batch_bytes(ctypes.byref(params), nx, ny, nz, n_orb, n_systems))


def lbks_batch_set_geometry(handle, system, xyz, Z):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    Z = np.ascontiguousarray(Z, dtype=np.float64).ravel()
    _check(_lib.lbks_batch_set_geometry(handle, system, len(Z), xyz.ctypes.data_as(_dp), Z.ctypes.data_as(_dp)))


def lbks_batch_init(handle):
    _check(_lib.lbks_batch_init(handle))


def lbks_batch_scf(handle, n_systems, stream=None, n_orb=MAX_ORB, allow_notconv=False):
    res = (lbks_result * n_systems)()
    code = _lib.lbks_batch_scf(handle, _stream(stream), res)
    if code != OK and not (allow_notconv and code == ENOTCONV):
        _check(code)
    return [_result_dict(res[i], n_orb) for i in range(n_systems)]


def lbks_batch_scf_cycles(handle, n_systems, n, stream=None, n_orb=MAX_ORB):
    res = (lbks_result * n_systems)()
    _check(_lib.lbks_scf_cycles(handle, n, _stream(stream), res))
    return [_result_dict(res[i], n_orb) for i in range(n_systems)]


def lbks_batch_energy(handle, system, n_orb=MAX_ORB) -> dict:
    t = lbks_energy_terms()
    _check(_lib.lbks_batch_energy(handle, system, ctypes.byref(t)))
    return {"T_s": t.T_s, "E_ext": t.E_ext, "E_H": t.E_H, "E_xc": t.E_xc, "E_nn": t.E_nn,
            "E_total": t.E_total, "eigenvalues": np.array(t.eigenvalues[:n_orb]),
            "orbital_energies": np.array(t.orbital_energies[:n_orb]), "n_electrons": t.n_electrons}


def lbks_batch_get_density(handle, system, shape):
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.lbks_batch_get_density(handle, system, out.ctypes.data_as(_dp), out.size))
    return out


def lbks_server_create(params=None, budget_bytes=0, max_slots=4):
    handle = ctypes.c_void_p()
    _check(_lib.lbks_server_create(ctypes.byref(params) if params is not None else None, budget_bytes, max_slots,
                                   ctypes.byref(handle)))
    return handle


def lbks_server_destroy(handle):
    _check(_lib.lbks_server_destroy(handle))


def lbks_submit(handle, n, h, xyz, Z, n_orb=None, precision=-1, n_inner=0, e_tol=0.0, max_cycles=0) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    Z = np.ascontiguousarray(Z, dtype=np.float64).ravel()
    if n_orb is None:
        n_orb = int(round(Z.sum())) // 2
    req = lbks_request(int(n[0]), int(n[1]), int(n[2]), float(h), int(n_orb), len(Z), xyz.ctypes.data_as(_dp),
                       Z.ctypes.data_as(_dp), int(precision), int(n_inner), float(e_tol), int(max_cycles))
    rid = ctypes.c_uint64()
    _check(_lib.lbks_submit(handle, ctypes.byref(req), ctypes.byref(rid)))
    return int(rid.value)


def lbks_poll(handle, rid, n_orb=MAX_ORB):
    """None while running; (result dict, timing dict) once done (raises on a failed solve)."""
    r, tm, done = lbks_result(), lbks_timing(), ctypes.c_int()
    code = _lib.lbks_poll(handle, ctypes.c_uint64(rid), ctypes.byref(r), ctypes.byref(tm), ctypes.byref(done))
    if code != OK and not done.value:
        _check(code)
    if not done.value:
        return None
    res = _result_dict(r, n_orb)
    res["status"] = code
    if code not in (OK, ENOTCONV):
        _check(code)
    return res, {"queue_s": tm.queue_s, "run_s": tm.run_s, "latency_s": tm.latency_s}


def lbks_server_wait(handle, rid, timeout_s=600.0):
    _check(_lib.lbks_server_wait(handle, ctypes.c_uint64(rid), float(timeout_s)))


def lbks_server_get_stats(handle) -> dict:
    st = lbks_server_stats()
    _check(_lib.lbks_server_get_stats(handle, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in lbks_server_stats._fields_}


# ------------------------------------------------------------- convenience
class Batch:
    """Owning wrapper of a batched handle: n_systems systems of one shape."""

    def __init__(self, n, h, n_orb, n_systems, **params):
        self.n = tuple(int(x) for x in n)
        self.h = float(h)
        self.n_orb = int(n_orb)
        self.n_systems = int(n_systems)
        self.params = lbks_params_default(**params)
        self.handle = lbks_create_batch(self.params, *self.n, self.h, self.n_orb, self.n_systems)

    @property
    def grid_shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    def set_geometries(self, molecules):
        for i, (xyz, Z) in enumerate(molecules):
            lbks_batch_set_geometry(self.handle, i, xyz, Z)
        lbks_batch_init(self.handle)

    def scf(self, stream=None, allow_notconv=False):
        return lbks_batch_scf(self.handle, self.n_systems, stream, self.n_orb, allow_notconv)

    def scf_cycles(self, n, stream=None):
        return lbks_batch_scf_cycles(self.handle, self.n_systems, n, stream, self.n_orb)

    def energy(self, i):
        return lbks_batch_energy(self.handle, i, self.n_orb)

    def density(self, i):
        return lbks_batch_get_density(self.handle, i, self.grid_shape)

    def forces(self, i, n_atoms):
        return lbks_batch_forces(self.handle, i, n_atoms)

    def close(self):
        if self.handle is not None:
            lbks_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """Owning wrapper of one lbks_system handle."""

    def __init__(self, n, h, n_orb, **params):
        self.n = tuple(int(x) for x in n)
        self.h = float(h)
        self.n_orb = int(n_orb)
        self.params = lbks_params_default(**params)
        self.handle = lbks_create_system(self.params, *self.n, self.h, self.n_orb)

    @property
    def grid_shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    def set_geometry(self, xyz, Z):
        lbks_set_geometry(self.handle, xyz, Z)
        self.n_atoms = len(np.ravel(Z))

    def forces(self):
        return lbks_forces(self.handle, self.n_atoms)

    def move_atoms(self, xyz):
        lbks_move_atoms(self.handle, xyz)

    def md(self, n_steps, dt, masses, velocities, stream=None):
        return lbks_md(self.handle, n_steps, dt, masses, velocities, stream)

    def cd_start(self, tau=0.0, kappa=0.0, n_pot=0, E_target=None, stream=None):
        return lbks_cd_start(self.handle, tau, kappa, n_pot, E_target, stream)

    def cd_run(self, n_blocks, masses=None, velocities=None, stream=None):
        return lbks_cd_run(self.handle, n_blocks, self.n_atoms, masses, velocities, stream)

    def cd_orbitals(self, level=1):
        return lbks_cd_get_orbitals(self.handle, level, self.n_orb, self.grid_shape)

    def cd_state(self):
        return lbks_cd_get_state(self.handle, self.n_atoms)

    def relax_geometry(self, max_steps=50, fmax=1e-3, step=0.5, stream=None, allow_notconv=False, fixed=None):
        return lbks_relax_geometry(self.handle, self.n_atoms, max_steps, fmax, step, stream, self.n_orb,
                                   allow_notconv, fixed)

    def scf(self, stream=None, allow_notconv=False):
        return lbks_scf(self.handle, stream, self.n_orb, allow_notconv)

    def scf_cycles(self, n, stream=None):
        return lbks_scf_cycles(self.handle, n, stream, self.n_orb)

    def energy(self):
        return lbks_energy(self.handle, self.n_orb)

    def density(self):
        return lbks_get_density(self.handle, self.grid_shape)

    def orbitals(self):
        return lbks_get_orbitals(self.handle, (self.n_orb,) + self.grid_shape)

    def potential(self, which=1):
        return lbks_get_potential(self.handle, which, self.grid_shape)

    def close(self):
        if self.handle is not None:
            lbks_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
