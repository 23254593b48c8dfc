"""Pins of the oracle's orbital-storage form (oracle.psi) against its
population form (oracle.lb): at omega = 1 the post-collision populations
are xi_p a - dt chi_p b of the site's orbital values (Sec. 3), so keeping
(psi, Lambda, Vc) and pulling the populations formed from them must give
the same steps and SCF cycles to rounding."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice, lb, psi as P, scf


def test_steps_equal_population_steps():
    n, h, theta = (7, 6, 8), 0.4, 0.5
    dt = lattice.time_step(theta, 1.0, h)
    rng = np.random.default_rng(3)
    psi0 = lb.orthonormalize(rng.uniform(-1, 1, size=(3, 8, 6, 7)), h)
    f, sig = lb.equilibrium(psi0, theta), np.ones(3)
    st, sig2 = P.PsiState(psi0.copy()), np.ones(3)
    for t in range(9):
        V = rng.uniform(-3, 1, size=(8, 6, 7))  # a new potential every step
        ortho = t in (3, 7)
        r = lb.step(f, sig, V, 1.0, theta, dt, h, orthonormalize=ortho)
        q = P.step(st, sig2, V, theta, dt, h, orthonormalize=ortho)
        f, sig, sig2 = r["fstar"], r["sigma"], q["sigma"]
        np.testing.assert_allclose(q["psi"], r["psi"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(q["S"], r["S"], rtol=0, atol=1e-14)
        np.testing.assert_allclose(sig2, sig, rtol=1e-14)


@pytest.mark.parametrize("n_orb,mol", [(1, W.helium()), (2, W.lih(3.0))])
def test_scf_cycles_equal_population_cycles(n_orb, mol):
    n, h = (18, 16, 20), 0.4
    st_a, a = scf.scf(n, h, mol.xyz, mol.Z, n_orb, n_inner=9, fixed_cycles=3)
    st_b, b = scf.scf(n, h, mol.xyz, mol.Z, n_orb, n_inner=9, fixed_cycles=3, storage="psi")
    assert a["E_total"] == pytest.approx(b["E_total"], abs=1e-12)
    np.testing.assert_allclose(a["eigenvalues"], b["eigenvalues"], atol=1e-12)
    np.testing.assert_allclose(st_a.rho, st_b.rho, atol=1e-13)


def test_orbital_storage_needs_omega_one():
    mol = W.helium()
    with pytest.raises(ValueError):
        scf.State((8, 8, 8), 0.5, mol.xyz, mol.Z, 1, omega=0.9, storage="psi")
