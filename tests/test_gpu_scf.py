"""GPU parity of the full self-consistent solve against the oracle, through
the C ABI (lbks_create_system / lbks_set_geometry / lbks_scf / lbks_energy).

Tolerances: |Delta E_total| <= 1e-5 Ha, Ritz eigenvalues
<= 1e-5 Ha, relative density L2 <= 1e-5.  The FP64 path reproduces the
oracle's trajectory to round-off; FP32 populations stay within the same
tolerances."""
import numpy as np
import pytest

import workloads as W
from oracle import scf

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

E_TOL, EIG_TOL, RHO_TOL = 1e-5, 1e-5, 1e-5


def _gpu_system(lbks, w, prec, **kw):
    params = dict(precision=prec, n_inner=w.n_inner, e_tol=w.e_tol, theta=w.theta, omega=w.omega, mix=w.mix,
                  max_cycles=w.max_cycles, poisson_rtol=1e-12)
    params.update(kw)
    s = lbks.System(w.n, w.h, w.n_orb, **params)
    s.set_geometry(w.molecule.xyz, w.molecule.Z)
    return s


def _rho_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _compare(g, ref, gpu_rho, ref_rho, e_tol=E_TOL):
    assert abs(g["E_total"] - ref["E_total"]) <= e_tol, (g["E_total"], ref["E_total"])
    np.testing.assert_allclose(np.sort(g["eigenvalues"]), np.sort(ref["eigenvalues"]), atol=EIG_TOL)
    assert _rho_l2(gpu_rho, ref_rho) <= RHO_TOL


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_initial_state_matches_oracle(prec):
    torch, lbks = require_gpu()
    w = W.ch4_small(32, 0.35)
    s = _gpu_system(lbks, w, prec)
    st = scf.State(w.n, w.h, w.molecule.xyz, w.molecule.Z, w.n_orb, w.theta, w.omega, poisson_rtol=1e-12)
    e = s.energy()
    for k in ("T_s", "E_ext", "E_H", "E_xc", "E_nn", "E_total", "n_electrons"):
        assert e[k] == pytest.approx(st.terms[k], abs=1e-9 if prec == 0 else 1e-5), k
    _compare(e, st.terms, s.density(), st.rho)
    np.testing.assert_allclose(s.potential(3), st.v_ext, rtol=1e-13)
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_helium_scf_matches_oracle(prec):
    torch, lbks = require_gpu()
    w = W.he_24()
    st, ref = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 1, n_inner=w.n_inner, e_tol=w.e_tol,
                      poisson_rtol=1e-12)
    s = _gpu_system(lbks, w, prec)
    g = s.scf()
    assert g["converged"]
    if prec == 0:
        assert g["cycles"] == ref["cycles"]
    _compare(g, ref, s.density(), st.rho)
    # FP32 orbitals carry ~1e-7 relative rounding into the density's norm
    assert g["n_electrons"] == pytest.approx(2.0, abs=1e-10 if prec == 0 else 1e-6)
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_methane_trajectory_matches_oracle(prec):
    """Five orbitals (W source active, degenerate t2 level), three fixed cycles."""
    torch, lbks = require_gpu()
    w = W.ch4_small(32, 0.35)
    w.n_inner = 20
    st, ref = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 5, n_inner=20, poisson_rtol=1e-12, fixed_cycles=3)
    s = _gpu_system(lbks, w, prec)
    g = s.scf_cycles(3)
    assert g["steps"] == ref["steps"]
    _compare(g, ref, s.density(), st.rho, e_tol=1e-8 if prec == 0 else E_TOL)
    np.testing.assert_allclose(s.potential(1), st.v_out, atol=1e-8 if prec == 0 else 1e-5)
    s.close()


def test_population_memory_omega_below_one():
    """omega = 0.8: the populations keep a memory term (1 - omega) f."""
    torch, lbks = require_gpu()
    w = W.he_24()
    w.omega = 0.8
    st, ref = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 1, n_inner=w.n_inner, omega=0.8, poisson_rtol=1e-12,
                      fixed_cycles=4)
    s = _gpu_system(lbks, w, 0)
    g = s.scf_cycles(4)
    _compare(g, ref, s.density(), st.rho, e_tol=1e-9)
    s.close()


def test_two_orbital_molecule_odd_cycle_length():
    """LiH with an odd cycle length exercises both graph start buffers."""
    torch, lbks = require_gpu()
    w = W.Workload("LiH", W.lih(3.0), (30, 28, 36), 0.3, n_inner=11)
    st, ref = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 2, n_inner=11, poisson_rtol=1e-12, fixed_cycles=5)
    s = _gpu_system(lbks, w, 0)
    g = s.scf_cycles(5)
    _compare(g, ref, s.density(), st.rho, e_tol=1e-8)
    s.close()


def test_scf_is_deterministic():
    torch, lbks = require_gpu()
    w = W.he_24()
    out = []
    for _ in range(2):
        s = _gpu_system(lbks, w, 1)
        out.append((s.scf()["E_total"], s.density()))
        s.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


def test_geometry_errors():
    torch, lbks = require_gpu()
    s = lbks.System((16, 16, 16), 0.3, 1)
    with pytest.raises(lbks.LbksError) as e:
        s.set_geometry([[10.0, 0.0, 0.0]], [2.0])  # outside the 4.5 bohr half-box
    assert e.value.code == lbks.EINVAL
    with pytest.raises(lbks.LbksError):
        s.set_geometry([[0.0, 0.0, 0.0]], [1.0])  # one electron for one doubly occupied orbital
    with pytest.raises(lbks.LbksError):
        s.scf()  # no geometry yet
    s.close()


def test_bf16_storage_with_fp32_polish():
    """bfloat16 populations until |dE| < 1e-4 Ha, then FP32 to convergence:
    within the stated tolerances of the oracle's self-consistent solution.

    The bfloat16 phase leaves the oracle's trajectory, so both sides are run
    to the fixed point (oracle |dE| < 1e-10, GPU < 1e-8): stopped at
    |dE| < 1e-6 the oracle's own eigenvalue is still ~3e-5 Ha from it (the
    energy is second order in the orbital error, the eigenvalue first order).
    Without the polish, bfloat16 rounding bounds the accuracy; its error is
    reported."""
    torch, lbks = require_gpu()
    w = W.he_24()
    st, ref = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 1, n_inner=w.n_inner, e_tol=1e-10,
                      poisson_rtol=1e-12)
    s = _gpu_system(lbks, w, 2, e_tol=1e-8, max_cycles=120)
    g = s.scf()
    assert g["converged"]
    _compare(g, ref, s.density(), st.rho)
    s.close()
    s = _gpu_system(lbks, w, 2, polish_tol=0.0, max_cycles=40)
    g = s.scf(allow_notconv=True)
    err = abs(g["E_total"] - ref["E_total"])
    rho_err = _rho_l2(s.density(), st.rho)
    print(f"bf16 without polish: |dE_total| = {err:.2e} Ha, density L2 = {rho_err:.2e}")
    assert err < 5e-3 and rho_err < 5e-2
    s.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_water_dimer_ten_orbitals_trajectory(prec):
    """Ten orbitals take the wide path (separate Gram, W-field, orthonormalisation
    and energy kernels); three fixed cycles against the oracle."""
    torch, lbks = require_gpu()
    mol = W.water_cluster(2, seed=3, box=11.0, min_oo=5.0, margin=2.5)
    n, h = (36, 32, 34), 0.35
    st, ref = scf.scf(n, h, mol.xyz, mol.Z, 10, n_inner=15, poisson_rtol=1e-12, fixed_cycles=3)
    s = lbks.System(n, h, 10, precision=prec, n_inner=15, poisson_rtol=1e-12)
    s.set_geometry(mol.xyz, mol.Z)
    g = s.scf_cycles(3)
    _compare(g, ref, s.density(), st.rho, e_tol=1e-8 if prec == 0 else E_TOL)
    s.close()


@pytest.mark.parametrize("mode", [1, 2, 3, 4], ids=["sites", "pairs", "prefetch", "bulk"])
def test_stream_collide_variants_give_the_oracle_trajectory(mode):
    """Both stream-collide kernels (one site or two x-neighbouring sites per
    thread), forced, follow the oracle's SCF trajectory; the tuner (mode 0)
    reports the variant it chose and both timings."""
    torch, lbks = require_gpu()
    mol = W.water(1.8, 104.0)
    n, h = (30, 26, 28), 0.4
    st, ref = scf.scf(n, h, mol.xyz, mol.Z, 5, n_inner=12, poisson_rtol=1e-12, fixed_cycles=2)
    prev = lbks.lbks_set_relax_variant(mode)
    try:
        for prec in (0, 1, 2):
            s = lbks.System(n, h, 5, precision=prec, n_inner=12, poisson_rtol=1e-12, polish_tol=0.0)
            s.set_geometry(mol.xyz, mol.Z)
            assert lbks.lbks_get_relax_variant(s.handle)["variant"] == lbks.RELAX_VARIANTS[mode - 1]
            g = s.scf_cycles(2)
            tol = {0: 1e-8, 1: 1e-5, 2: 2e-3}[prec]
            assert abs(g["E_total"] - ref["E_total"]) <= tol, (prec, g["E_total"], ref["E_total"])
            s.close()
    finally:
        lbks.lbks_set_relax_variant(prev)
    lbks.lbks_set_relax_variant(0)
    s = lbks.System((34 + 2 * mode, 22, 18), h, 5, precision=1, n_inner=12)  # a shape no other test uses
    s.set_geometry(mol.xyz, mol.Z)
    t = lbks.lbks_get_relax_variant(s.handle)
    assert t["variant"] in lbks.RELAX_VARIANTS and min(t[f"ms_{v}"] for v in lbks.RELAX_VARIANTS) > 0
    s.close()
    lbks.lbks_set_relax_variant(prev)
