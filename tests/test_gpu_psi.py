"""Orbital storage at omega = 1 (LBKS_STORE_PSI): the step keeps psi alone and
applies the pull-and-sum of Eq. KSLB as a 19-point stencil.  Its results must
equal the oracle's population step fed the populations that the psi state
stands for, f*_p = xi_p psi - dt chi_p Vc psi + xi_p u with the W field
u_j = -sum_{k<j} Lambda_jk psi_k, element by element, and an orbital-storage
SCF must follow the oracle's trajectory."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice, lb, scf

from gpu_util import rel_err, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


def _populations(A, u, Vc, theta, dt):
    """The post-collision populations the psi-state (A, Vc, u) stands for."""
    xi = lattice.xi(theta)[None, :, None, None, None]
    chi = lattice.chi()[None, :, None, None, None]
    f = xi * A[:, None] - dt * chi * (Vc[None, None] * A[:, None])
    if A.shape[0] > 1:
        f[1:] += xi * u[:, None]
    return f


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("n,n_orb,seed", [
    ((7, 9, 11), 1, 0), ((33, 20, 17), 5, 1), ((16, 5, 40), 8, 2), ((2, 3, 2), 3, 3),
    ((21, 18, 23), 12, 4), ((9, 10, 11), 10, 5), ((12, 10, 9), 64, 6), ((70, 3, 9), 6, 7),
    # rows of whole 16-byte units (the TMA kernel's tensor maps): several tiles in x and y
    # with ragged ends, two planes, grids smaller than a box, each orbital bucket
    ((36, 11, 13), 5, 8), ((44, 9, 7), 12, 9), ((4, 3, 5), 3, 10), ((64, 17, 6), 40, 11),
    ((40, 8, 3), 8, 12), ((8, 2, 2), 1, 13), ((32, 9, 2), 2, 14), ((12, 20, 4), 33, 15),
    # many z runs of the z-marching kernel
    ((34, 17, 70), 5, 16),
])
@pytest.mark.parametrize("with_w", [True, False], ids=["W", "noW"])
@pytest.mark.parametrize("mode", [1, 2, 3, 4], ids=["tiled", "direct", "tma", "zmarch"])
def test_psi_step_matches_population_oracle(prec, n, n_orb, seed, with_w, mode):
    """mode 3 forces the TMA kernel where its tensor maps apply (nx a multiple
    of 16 / the value's bytes), the tiled one elsewhere; mode 4 the z-marching
    kernel up to eight orbitals (grids of one, two or many z runs, ragged x and
    y tiles), the tiled one above."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(mode)  # forced: tiled, one site per thread, or TMA
    try:
        _psi_step_case(torch, lbks, prec, n, n_orb, seed, with_w)
    finally:
        lbks.lbks_set_relax_variant(prev)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("n,n_orb,seed", [((36, 11, 13), 5, 8), ((40, 8, 3), 8, 12), ((64, 17, 19), 3, 20),
                                          ((68, 9, 10), 1, 21), ((8, 2, 2), 1, 13), ((33, 20, 17), 5, 1),
                                          ((132, 10, 5), 6, 22), ((4, 9, 9), 2, 23)])
@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6, 7],
                         ids=["32x8x4", "32x8x8", "64x4x4", "32x8x2", "64x8x4w2", "64x8x2w2", "32x8x8pl", "32x8x4pl"])
def test_psi_step_tile_shapes_match_population_oracle(prec, n, n_orb, seed, shape):
    """The staged stencil at every tile shape the tuner tries (ragged tiles in
    x, y and z; an odd nx runs the default shape's scalar staging); shapes 4
    and 5 sum two x-neighbouring sites per thread (FP32, FP64 up to three
    orbitals), shapes 6 and 7 by velocity class from plane sums (FP32 up to
    six orbitals, FP64 up to three)."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(1)
    prev_shape = lbks.lbks_set_psi_tile(shape)
    try:
        _psi_step_case(torch, lbks, prec, n, n_orb, seed, True)
    finally:
        lbks.lbks_set_relax_variant(prev)
        lbks.lbks_set_psi_tile(prev_shape)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("shape", [1, 4, 5, 6], ids=["32x8x8", "64x8x4w2", "64x8x2w2", "32x8x8pl"])
def test_psi_step_unaligned_output_runs_the_scalar_staging(prec, shape):
    """An output that is not 16-byte aligned (one value into its buffer)
    sends every forced shape to the default shape's scalar staging, whose
    one-value stores need no alignment: the results still match."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(1)
    prev_shape = lbks.lbks_set_psi_tile(shape)
    try:
        _psi_step_case(torch, lbks, prec, (36, 11, 13), 3, 24, True, out_offset=1)
    finally:
        lbks.lbks_set_relax_variant(prev)
        lbks.lbks_set_psi_tile(prev_shape)


def test_psi_tile_shape_is_tuned():
    """The tuner times every tile shape of the staged stencil and keeps the
    fastest; a bad shape is refused."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(0)
    try:
        s = lbks.System((44, 26, 18), 0.4, 5, precision=1, storage=lbks.STORE_PSI)  # a shape no other test tunes
        mol = W.methane()
        s.set_geometry(mol.xyz, mol.Z)
        got = lbks.lbks_get_psi_tile(s.handle)
        s.close()
    finally:
        lbks.lbks_set_relax_variant(prev)
    assert all(t > 0 for t in got["ms"])  # FP32, five orbitals: every shape runs as itself
    assert got["ms"][got["shape"]] == min(got["ms"])
    with pytest.raises(lbks.LbksError):
        lbks.lbks_set_psi_tile(len(lbks.PSI_TILES))


def _psi_step_case(torch, lbks, prec, n, n_orb, seed, with_w, out_offset=0):
    theta, h = 0.5, 0.3
    dt = lattice.time_step(theta, 1.0, h)
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(-0.5, 1.0, size=(n_orb, nz, ny, nx))
    Vc = rng.uniform(-3.0, 1.0, size=(nz, ny, nx))
    lam_in = np.tril(rng.uniform(-0.3, 0.3, size=(n_orb, n_orb)), -1) * (1.0 if with_w else 0.0)
    sigma = rng.uniform(0.5, 2.0, size=n_orb)
    if prec == 1:  # the oracle sees the values the GPU stores
        A = A.astype(np.float32).astype(np.float64)
    # the W field the step forms: u_j = -sum_{k<j} Lambda_jk psi_k (omega = 1)
    u = -np.tensordot(lam_in, A, axes=(1, 0))[1:]
    P = torch.float64 if prec == 0 else torch.float32
    psi_in = to_dev(torch, A, P)
    # out_offset > 0: the output starts that many values into its buffer (not 16-byte aligned)
    psi_out = torch.empty(psi_in.numel() + out_offset, dtype=P, device="cuda")[out_offset:].view(psi_in.shape)
    S = torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda")
    lam, sig_out = torch.empty_like(S), torch.empty(n_orb, dtype=torch.float64, device="cuda")
    lam_dev = to_dev(torch, lam_in, torch.float64) if with_w else None
    lbks.lbks_relax_step_psi(prec, nx, ny, nz, n_orb, h, theta, dt, psi_in, lam_dev,
                             to_dev(torch, Vc, torch.float64), to_dev(torch, sigma, torch.float64), psi_out, S, lam,
                             sig_out)
    torch.cuda.synchronize()
    ref = lb.step(_populations(A, u, Vc, theta, dt), sigma, np.zeros_like(Vc), 1.0, theta, dt, h)
    tol = TOL[prec]
    assert rel_err(to_np(psi_out), ref["psi"]) < tol
    # more than 8 FP32 orbitals: the per-step overlap runs on the tensor cores (~1e-6 relative)
    stol = 1e-5 if (prec == 1 and n_orb > 8) else tol
    assert rel_err(to_np(S), ref["S"]) < stol
    np.testing.assert_allclose(to_np(sig_out), ref["sigma"], rtol=stol)
    np.testing.assert_allclose(to_np(lam), ref["lam"], atol=stol * max(1.0, np.abs(ref["lam"]).max()))


def test_psi_step_rejects_bad_arguments():
    torch, lbks = require_gpu()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    xf = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(lbks.LbksError):  # bfloat16 has no orbital storage
        lbks.lbks_relax_step_psi(2, 2, 2, 2, 1, 0.2, 0.5, 0.02, xf, None, x[:8], x[:1], xf.clone(), x[:1], x[:1],
                                 x[:1])
    with pytest.raises(lbks.LbksError):  # in and out alias
        lbks.lbks_relax_step_psi(0, 2, 2, 2, 1, 0.2, 0.5, 0.02, x, None, x[:8], x[:1], x, x[:1], x[:1], x[:1])
    with pytest.raises(lbks.LbksError):  # omega != 1
        lbks.System((8, 8, 8), 0.4, 1, storage=lbks.STORE_PSI, omega=0.9)
    with pytest.raises(lbks.LbksError):
        lbks.System((8, 8, 8), 0.4, 1, storage=lbks.STORE_PSI, precision=lbks.BF16)


SCF_MODE = {"ch4": 0, "ch4_direct": 2, "ch4_tma": 3, "ch4_zmarch": 4, "water_dimer": 0, "water_dimer_tiled": 1}


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", list(SCF_MODE))
def test_psi_storage_scf_follows_the_oracle(prec, case):
    """Three fixed cycles from the Gaussian start: the first step pulls with no
    potential term (the start is f = xi psi), every cycle's first step with
    the previous cycle's collision potential.  ch4: the tuned kernel;
    ch4_direct: one site per thread forced; ch4_tma: the TMA kernel forced on
    a grid whose rows it takes; ch4_zmarch: the z-marching kernel forced;
    water_dimer (ten orbitals): the default, the
    TMA kernel with the W source formed in the step; water_dimer_tiled: the
    tiled kernel with the W field."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(SCF_MODE[case])
    try:
        _psi_scf_case(torch, lbks, prec, case)
    finally:
        lbks.lbks_set_relax_variant(prev)


def _psi_scf_case(torch, lbks, prec, case):
    if case.startswith("ch4"):
        mol, n, h, n_orb, n_inner = W.methane(), (32 if case == "ch4_tma" else 30, 28, 26), 0.45, 5, 12
    else:
        mol = W.water_cluster(2, seed=3, box=11.0, min_oo=5.0, margin=2.5)
        n, h, n_orb, n_inner = (36, 32, 34), 0.35, 10, 15
    st, ref = scf.scf(n, h, mol.xyz, mol.Z, n_orb, n_inner=n_inner, poisson_rtol=1e-12, fixed_cycles=3)
    s = lbks.System(n, h, n_orb, precision=prec, n_inner=n_inner, poisson_rtol=1e-12, storage=lbks.STORE_PSI)
    s.set_geometry(mol.xyz, mol.Z)
    g = s.scf_cycles(3)
    etol = 1e-8 if prec == 0 else 1e-5
    assert abs(g["E_total"] - ref["E_total"]) <= etol, (g["E_total"], ref["E_total"])
    np.testing.assert_allclose(np.sort(g["eigenvalues"][:n_orb]), np.sort(ref["eigenvalues"]), atol=etol)
    rho = s.density()
    assert np.linalg.norm(rho - st.rho) / np.linalg.norm(st.rho) <= (1e-8 if prec == 0 else 1e-5)
    s.close()


def test_psi_and_population_storage_converge_alike():
    """Full FP64 solves in the two storages stop at the same cycle with the
    same energy (the two differ only in rounding)."""
    torch, lbks = require_gpu()
    mol, n, h = W.water(1.8, 104.0), (30, 26, 28), 0.4
    out = []
    for storage in (lbks.STORE_POPULATIONS, lbks.STORE_PSI):
        s = lbks.System(n, h, 5, precision=0, n_inner=100, max_cycles=400, storage=storage)
        s.set_geometry(mol.xyz, mol.Z)
        out.append(s.scf())
        s.close()
    a, b = out
    assert a["converged"] and b["converged"] and a["cycles"] == b["cycles"]
    assert abs(a["E_total"] - b["E_total"]) <= 1e-10
    np.testing.assert_allclose(a["eigenvalues"][:5], b["eigenvalues"][:5], atol=1e-10)


def test_psi_storage_batch_matches_single():
    torch, lbks = require_gpu()
    n, h = (28, 26, 30), 0.4
    mols = W.water_scan(3, 2)
    b = lbks.Batch(n, h, 5, len(mols), precision=0, n_inner=100, max_cycles=400, storage=lbks.STORE_PSI)
    b.set_geometries([(m.xyz, m.Z) for m in mols])
    res = b.scf()
    for i, m in enumerate(mols):
        s = lbks.System(n, h, 5, precision=0, n_inner=100, max_cycles=400, storage=lbks.STORE_PSI)
        s.set_geometry(m.xyz, m.Z)
        ref = s.scf()
        assert res[i]["converged"] and res[i]["cycles"] == ref["cycles"]
        assert abs(res[i]["E_total"] - ref["E_total"]) <= 1e-9
        s.close()
    b.close()


@pytest.mark.parametrize("prec,nx,n_orb", [
    (1, 36, 10), (1, 34, 10), (0, 34, 10), (0, 35, 10), (1, 36, 5), (1, 34, 5),
])
def test_psi_kernel_choice(prec, nx, n_orb):
    """The tuner times the orbital-storage kernels that apply to the shape and
    keeps the fastest: up to eight orbitals tiled, one site per thread, TMA
    (where its tensor maps apply: nx a multiple of 16 / the value's bytes) and
    z-marching; more than eight the tiled step with its W-field pass against
    the TMA step, which forms the W source itself."""
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(0)
    try:
        s = lbks.System((nx, 12, 10), 0.4, n_orb, precision=prec, storage=lbks.STORE_PSI)
        if n_orb == 5:
            mol = W.methane()
            s.set_geometry(mol.xyz, mol.Z)
        else:  # two Z = 10 centres: ten doubly occupied orbitals
            s.set_geometry(np.array([[-2.0, 0.0, 0.0], [2.0, 0.0, 0.0]]), np.array([10.0, 10.0]))
        got = lbks.lbks_get_relax_variant(s.handle)
    finally:
        lbks.lbks_set_relax_variant(prev)
    names = lbks.RELAX_VARIANTS
    tma_ok = nx % (4 if prec == 1 else 2) == 0
    if n_orb > 8 and not tma_ok:  # nothing to choose: the tiled step
        assert got["index"] == 0
    else:
        ms = {k: got["ms_" + names[k]] for k in range(4)}
        timed = [k for k in range(4) if ms[k] >= 0]
        assert (2 in timed) == tma_ok and 0 in timed and (1 in timed) == (n_orb <= 8)
        assert (3 in timed) == (n_orb <= 8)
        assert got["index"] == min(timed, key=lambda k: ms[k])
    s.close()
