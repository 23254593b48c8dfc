"""Concurrent dynamics (Eq. KSLBCD of Sec. 3) through the C ABI against the
oracle (oracle/cd.py): one step on random complex levels, the start from a
ground state, Ehrenfest blocks with moving nuclei, and stationarity."""
import numpy as np
import pytest

from oracle import cd, lattice

from gpu_util import require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

THETA = 0.5


def _levels(rng, no, n):
    nx, ny, nz = n
    shape = (no, nz, ny, nx)
    smooth = np.sin(np.linspace(0, 3, nx))[None, None, None, :]
    a = rng.uniform(-1, 1, size=shape) + smooth + 1j * (rng.uniform(-1, 1, size=shape) - smooth)
    b = a + 0.05 * (rng.uniform(-1, 1, size=shape) + 1j * rng.uniform(-1, 1, size=shape))
    return a, b


def _split(phi):
    """[n_orb, nz, ny, nx] complex -> [n_orb, 2, nz, ny, nx] real, imaginary planes."""
    return np.stack([phi.real, phi.imag], axis=1)


def _rounded(phi, prec):
    if prec == 0:
        return phi
    f = lambda x: x.astype(np.float32).astype(np.float64)
    return f(phi.real) + 1j * f(phi.imag)


STEP_CASES = [((13, 11, 9), 1, False), ((13, 11, 9), 3, True), ((40, 33, 17), 2, False), ((40, 33, 17), 5, True),
              ((24, 20, 22), 8, False), ((2, 2, 2), 4, True), ((31, 29, 27), 8, True)]


@pytest.fixture(params=[0, 1], ids=["one_site", "staged"])
def cd_kernel(request):
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_cd_kernel(request.param)
    yield request.param
    lbks.lbks_set_cd_kernel(prev)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("n,no,with_u", STEP_CASES)
def test_step_matches_the_oracle(prec, n, no, with_u, cd_kernel):
    """phi_next, its overlap and Lambda against oracle.cd_step on the same
    levels (FP32: the same rounded inputs), W source from the device Lambda;
    both kernels (the staged one where its box fits, else one site)."""
    torch, lbks = require_gpu()
    rng = np.random.default_rng(hash((n, no, with_u)) % 2**32)
    nx, ny, nz = n
    h = 0.3
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.5 * dt
    prev, cur = (_rounded(x, prec) for x in _levels(rng, no, n))
    V = rng.uniform(-3.0, 1.0, size=(nz, ny, nx))
    kappa = 0.7 if with_u else 0.0
    E = rng.uniform(-1.0, -0.2, size=no)
    P = torch.float64 if prec == 0 else torch.float32
    d_prev, d_cur = to_dev(torch, _split(prev), P), to_dev(torch, _split(cur), P)
    d_V = to_dev(torch, V, torch.float64)
    S0 = torch.zeros((no, no, 2), dtype=torch.float64, device="cuda")
    lam0 = torch.zeros_like(S0)
    lbks.lbks_cd_overlap(prec, nx * ny * nz, no, h, d_cur, S0, lam0)
    u = to_dev(torch, 2 * tau * kappa * E, torch.float64) if with_u else None
    d_next = torch.empty_like(d_cur)
    S1, lam1 = torch.zeros_like(S0), torch.zeros_like(S0)
    lbks.lbks_cd_step(prec, nx, ny, nz, no, h, THETA, tau, d_prev, d_cur, d_V, lam0, u, d_next, S1, lam1)
    torch.cuda.synchronize()
    ref = cd.cd_step(prev, cur, V, THETA, dt, h, tau, kappa, E)
    got = to_np(d_next)
    got = got[:, 0] + 1j * got[:, 1]
    tol = 1e-12 if prec == 0 else 3e-6
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale
    # overlaps and Lambda: of cur (device, before the step) and of next (fused);
    # FP32 levels: products in FP32 per thread, sums over threads in FP64
    stol = 1e-12 if prec == 0 else 2e-6
    for dS, dlam, phi in ((S0, lam0, cur), (S1, lam1, got)):
        Sref = cd.overlap(phi, h)
        Sg = to_np(dS)
        np.testing.assert_allclose(Sg[..., 0] + 1j * Sg[..., 1], Sref, rtol=0, atol=stol * np.abs(Sref).max())
        Lg = to_np(dlam)
        Lref = cd.lambda_matrix(Sref)
        np.testing.assert_allclose(Lg[..., 0] + 1j * Lg[..., 1], Lref, rtol=0,
                                   atol=10 * stol * max(1.0, np.abs(Lref).max()))


def test_step_without_previous_level_or_w_source():
    """phi_prev NULL is zero; lambda NULL drops the W source."""
    torch, lbks = require_gpu()
    rng = np.random.default_rng(4)
    n, no, h = (12, 10, 9), 3, 0.4
    nx, ny, nz = n
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.25 * dt
    _, cur = _levels(rng, no, n)
    V = rng.uniform(-2.0, 0.5, size=(nz, ny, nx))
    d_cur = to_dev(torch, _split(cur), torch.float64)
    d_next = torch.empty_like(d_cur)
    lbks.lbks_cd_step(0, nx, ny, nz, no, h, THETA, tau, None, d_cur, to_dev(torch, V, torch.float64), None, None,
                      d_next)
    torch.cuda.synchronize()
    ref = 2j * (tau / dt) * cd.increment(cur, V, THETA, dt, h, w_source=False)
    got = to_np(d_next)
    np.testing.assert_allclose(got[:, 0] + 1j * got[:, 1], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def _h2(d):
    return np.array([[-d / 2, 0.0, 0.0], [d / 2, 0.0, 0.0]]), np.array([1.0, 1.0])


H2_N, H2_H = (22, 18, 18), 0.35


def _ground_state(lbks, prec, xyz, Z, n=H2_N, h=H2_H, n_orb=1):
    s = lbks.System(n, h, n_orb, precision=prec, n_inner=40, e_tol=1e-9, eig_tol=1e-7, rho_tol=1e-7,
                    max_cycles=400, poisson_rtol=1e-12)
    s.set_geometry(xyz, Z)
    r = s.scf()
    assert r["converged"]
    return s


def test_start_matches_the_oracle():
    """Level 0 (the handle's orbitals), the rebuilt potential's energy and the
    Taylor second level against oracle.cd.Run on the same orbitals (FP64)."""
    torch, lbks = require_gpu()
    xyz, Z = _h2(1.5)
    s = _ground_state(lbks, 0, xyz, Z)
    psi = s.orbitals()
    e0, n_el = s.cd_start()
    run = cd.Run(psi, H2_N, H2_H, xyz, Z, theta=THETA, v_h=s.potential(2))
    ref = run.energies()
    assert abs(e0 - ref["E_total"]) < 1e-9
    assert abs(n_el - 2.0) < 1e-6
    np.testing.assert_allclose(s.cd_orbitals(0), psi, rtol=0, atol=1e-14)
    np.testing.assert_allclose(s.cd_orbitals(1), run.cur, rtol=0, atol=1e-10 * np.abs(run.cur).max())
    st = s.cd_state()
    assert st["steps"] == 1 and abs(st["time"] - run.tau) < 1e-15
    np.testing.assert_allclose(st["forces"], run.F, rtol=1e-8, atol=1e-10)
    s.close()


@pytest.mark.parametrize("n_orb", [1, 2])
def test_moving_nuclei_follow_the_oracle(n_orb):
    """Ehrenfest blocks from a stretched geometry, FP64 on both sides: energies,
    nuclear kinetic energy, positions and the final level.  Two orbitals: H2
    with a second pair of electrons' worth of charge (Z = 2, 2: He2 at short
    range), so the W source acts."""
    torch, lbks = require_gpu()
    xyz, Z = _h2(1.7)
    if n_orb == 2:
        xyz, Z = _h2(2.2)[0], np.array([2.0, 2.0])
    s = _ground_state(lbks, 0, xyz, Z, n_orb=n_orb)
    psi = s.orbitals()
    M = np.array([1836.15267, 1836.15267]) * (1.0 if n_orb == 1 else 4.0)
    s.cd_start(n_pot=5)
    run = cd.Run(psi, H2_N, H2_H, xyz, Z, theta=THETA, v_h=s.potential(2), masses=M)
    v, e, traj = s.cd_run(8, masses=M)
    for b in range(8):
        run.block(5)
        t = run.energies()
        assert abs(e[b, 0] - t["E_total"]) < 1e-8, (b, e[b, 0], t["E_total"])
        assert abs(e[b, 1] - t["E_kin_nuclei"]) < 1e-10 + 1e-6 * t["E_kin_nuclei"]
        np.testing.assert_allclose(traj[b], run.xyz, rtol=0, atol=1e-10)
    np.testing.assert_allclose(v, run.vel, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(s.cd_orbitals(1), run.cur, rtol=0, atol=1e-8 * np.abs(run.cur).max())
    assert e[-1, 1] > 0.0
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_ground_state_stays_put(prec):
    """A converged ground state with fixed nuclei: density, energy and
    electron count unchanged over 200 steps, the orbital rotating at
    arcsin(eps tau)/tau."""
    torch, lbks = require_gpu()
    xyz, Z = _h2(1.4)
    s = _ground_state(lbks, prec, xyz, Z)
    psi = s.orbitals()
    rho0 = s.density()
    e0, _ = s.cd_start(n_pot=10)
    _, e, _ = s.cd_run(20)
    rho1 = s.density()
    tol = 1e-9 if prec == 0 else 2e-6
    assert np.abs(e[:, 0] - e0).max() < tol
    # the ground state holds to its SCF tolerances (rho_tol 1e-7)
    assert np.linalg.norm(rho1 - rho0) / np.linalg.norm(rho0) < (1e-7 if prec == 0 else 1e-5)
    V = s.potential(0)
    g = psi[0].astype(complex)
    run_dt = lattice.time_step(THETA, 1.0, H2_H)
    tau = 0.5 * run_dt
    hg = (g - cd.pulled(g, lattice.xi(THETA))) / run_dt + cd.pulled(V * g, lattice.chi())
    eps = cd.inner(g, hg, H2_H).real / cd.inner(g, g, H2_H).real
    omega = np.arcsin(eps * tau) / tau
    st = s.cd_state()
    ov = cd.inner(g, s.cd_orbitals(1)[0], H2_H)
    assert abs(abs(ov) - 1.0) < (1e-8 if prec == 0 else 1e-5)
    assert abs(np.angle(ov * np.exp(1j * omega * st["steps"] * tau))) < (1e-6 if prec == 0 else 1e-4)
    s.close()


def test_errors():
    torch, lbks = require_gpu()
    with pytest.raises(lbks.LbksError):
        lbks.lbks_set_cd_kernel(2)
    assert lbks.lbks_set_cd_kernel(-1) == -1  # the default, unchanged
    xyz, Z = _h2(1.4)
    s = lbks.System(H2_N, H2_H, 1, precision=0, omega=0.9, n_inner=10)
    s.set_geometry(xyz, Z)
    with pytest.raises(lbks.LbksError):
        s.cd_start()  # built on the omega = 1 step
    s.close()
    s = lbks.System(H2_N, H2_H, 1, precision=0, n_inner=10)
    with pytest.raises(lbks.LbksError):
        s.cd_start()  # no geometry
    s.set_geometry(xyz, Z)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_cd_run(s.handle, 1, 2)  # not started
    with pytest.raises(lbks.LbksError):
        s.cd_start(tau=1.0)  # tau above theta h^2
    with pytest.raises(lbks.LbksError):
        s.cd_start(kappa=0.5)  # U source without target energies
    s.cd_start()
    with pytest.raises(lbks.LbksError):
        s.cd_run(1, masses=[1.0, -1.0])
    s.close()
    d = torch.zeros((9, 2, 2, 2, 2), dtype=torch.float64, device="cuda")
    V = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lbks.LbksError):
        lbks.lbks_cd_step(0, 2, 2, 2, 9, 0.3, THETA, 0.01, None, d, V, None, None, torch.empty_like(d))
    f = d[:1].float().contiguous()
    with pytest.raises(lbks.LbksError):  # bfloat16 has no dynamics
        lbks.lbks_cd_step(2, 2, 2, 2, 1, 0.3, THETA, 0.01, None, f, V, None, None, torch.empty_like(f))
