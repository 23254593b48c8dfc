"""Born-Oppenheimer extension: Hellmann-Feynman forces (lbks_forces), atom
moves with warm-started orbitals (lbks_move_atoms) and geometry relaxation
(lbks_relax_geometry), against the oracle (oracle.forces, oracle.scf)."""
import numpy as np
import pytest

import workloads as W
from oracle import forces, md, scf

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

H2_GRID, H2_H = (18, 18, 22), 0.35  # H2 lies along z


def _h2(d):
    return np.array([[0.0, 0.0, -d / 2], [0.0, 0.0, d / 2]]), np.array([1.0, 1.0])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("waters", [1, 3, 6])  # 3, 9 and 18 nuclei: one, two and three chunks of the reduction
def test_forces_match_the_oracle_at_the_solver_density(prec, waters):
    """The device reduction against oracle.forces on the density the handle holds."""
    torch, lbks = require_gpu()
    if waters == 1:
        mol, n, h = W.water(1.8, 104.0), (30, 26, 28), 0.4
    else:
        mol, n, h = W.water_cluster(waters, seed=2, box=14.0, min_oo=4.0, margin=3.0), (36, 36, 36), 0.4
    s = lbks.System(n, h, 4 * waters + waters, precision=prec, n_inner=8)
    s.set_geometry(mol.xyz, mol.Z)
    s.scf_cycles(1)
    rho = s.density()
    F = s.forces()
    ref = forces.hf_forces(rho, h, mol.xyz, mol.Z, h)  # the default softening a = h
    np.testing.assert_allclose(F, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())
    s.close()


def test_batch_forces_match_the_oracle_per_system():
    """Every system of a batch, converged or still running, at its own density."""
    torch, lbks = require_gpu()
    n, h = (28, 26, 30), 0.4
    mols = W.water_scan(3, 5)
    b = lbks.Batch(n, h, 5, len(mols), precision=0, n_inner=10)
    b.set_geometries([(m.xyz, m.Z) for m in mols])
    b.scf_cycles(1)
    for i, m in enumerate(mols):
        ref = forces.hf_forces(b.density(i), h, m.xyz, m.Z, h)
        np.testing.assert_allclose(b.forces(i, len(m.Z)), ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())
    b.close()


def test_forces_follow_the_oracle_scf():
    """Three fixed cycles of H2 in FP64 on both sides: same density, same forces."""
    torch, lbks = require_gpu()
    xyz, Z = _h2(1.3)
    st, _ = scf.scf(H2_GRID, H2_H, xyz, Z, 1, n_inner=20, poisson_rtol=1e-12, fixed_cycles=3)
    ref = forces.hf_forces(st.rho, H2_H, xyz, Z, st.a)
    s = lbks.System(H2_GRID, H2_H, 1, precision=0, n_inner=20, poisson_rtol=1e-12)
    s.set_geometry(xyz, Z)
    s.scf_cycles(3)
    np.testing.assert_allclose(s.forces(), ref, rtol=1e-7, atol=1e-9)
    s.close()


@pytest.mark.parametrize("storage", ["populations", "psi"])
def test_move_atoms_then_scf_matches_a_fresh_solve(storage):
    torch, lbks = require_gpu()
    """Both converged far (|dE| < 1e-10 per cycle: a stop at 1e-6 can sit
    some 1e-5 Ha from the fixed point) from different starts."""
    st = lbks.STORE_PSI if storage == "psi" else lbks.STORE_POPULATIONS
    kw = dict(precision=0, n_inner=30, storage=st, e_tol=1e-10, max_cycles=400)
    s = lbks.System(H2_GRID, H2_H, 1, **kw)
    xyz, Z = _h2(1.3)
    s.set_geometry(xyz, Z)
    s.scf()
    xyz2, _ = _h2(1.5)
    s.move_atoms(xyz2)
    moved = s.scf()
    f = lbks.System(H2_GRID, H2_H, 1, **kw)
    f.set_geometry(xyz2, Z)
    fresh = f.scf()
    assert moved["converged"] and fresh["converged"]
    assert moved["cycles"] < fresh["cycles"]  # the warm start pays
    assert abs(moved["E_total"] - fresh["E_total"]) < 1e-7
    np.testing.assert_allclose(s.forces(), f.forces(), atol=1e-5)
    s.close()
    f.close()


def test_relax_geometry_finds_the_oracle_force_zero():
    """H2 from 1.1 bohr: the relaxed bond has no force on the oracle's side
    either (one oracle solve at the returned geometry), and the energy is the
    oracle's there."""
    torch, lbks = require_gpu()
    s = lbks.System(H2_GRID, H2_H, 1, precision=0, n_inner=30, e_tol=1e-9)
    xyz, Z = _h2(1.1)
    s.set_geometry(xyz, Z)
    e0 = s.scf()["E_total"]
    r = s.relax_geometry(max_steps=40, fmax=1e-3, step=1.0)
    assert r["relaxed"] and r["E_total"] < e0
    R = r["xyz"]
    # stays on the axis and centred (the start orbitals' offsets break the
    # symmetry at the 1e-8 level)
    np.testing.assert_allclose(R[:, :2], 0.0, atol=1e-5)
    np.testing.assert_allclose(R[0, 2], -R[1, 2], atol=1e-4)
    assert np.abs(s.forces()).max() < 1e-3
    st, ref = scf.scf(H2_GRID, H2_H, R, Z, 1, n_inner=30, e_tol=1e-10, max_cycles=400)
    Fo = forces.hf_forces(st.rho, H2_H, R, Z, st.a)
    assert np.abs(Fo).max() < 2e-3, Fo
    assert abs(r["E_total"] - ref["E_total"]) < 1e-5
    d = R[1, 2] - R[0, 2]
    assert 1.5 < d < 2.3, d  # softened nuclei (a = h = 0.35) bind H2 longer than 1.4 bohr
    s.close()


def test_relax_geometry_keeps_fixed_nuclei():
    """One H2 nucleus fixed: it does not move, the other relaxes to zero force."""
    torch, lbks = require_gpu()
    s = lbks.System(H2_GRID, H2_H, 1, precision=0, n_inner=30, e_tol=1e-9)
    xyz, Z = _h2(1.1)
    s.set_geometry(xyz, Z)
    r = s.relax_geometry(max_steps=40, fmax=1e-3, step=1.0, fixed=[1, 0])
    assert r["relaxed"]
    np.testing.assert_array_equal(r["xyz"][0], xyz[0])
    F = s.forces()
    assert np.linalg.norm(F[1]) < 1e-3 and np.linalg.norm(F[0]) > 1e-3  # the held nucleus still feels a force
    s.close()


M_H = 1836.15267  # proton mass in electron masses


def test_md_follows_the_oracle_and_conserves_energy():
    """H2 released from a stretched bond, FP64, velocity Verlet with dt = 10:
    the first three steps against the oracle's integrator driven by oracle
    SCF forces; over 20 steps E_total + E_kin stays within 6e-5 Ha while
    E_kin grows to 6.5e-4 Ha (the bond contracts).  The Hellmann-Feynman
    force is -dE/dR only up to the scheme's non-variational terms, and the
    energy has a grid ripple as the nuclei cross grid planes (R20): the
    measured excursion is 3.7e-5 Ha and returns towards zero."""
    torch, lbks = require_gpu()
    xyz, Z = _h2(2.2)
    m, dt = [M_H, M_H], 10.0
    s = lbks.System(H2_GRID, H2_H, 1, precision=0, n_inner=30, e_tol=1e-11, max_cycles=600)
    s.set_geometry(xyz, Z)
    v, e, traj = s.md(20, dt, m, np.zeros((2, 3)))
    tot = e.sum(axis=1)
    assert e[-1, 1] > 3e-4
    assert np.abs(tot - tot[0]).max() < 6e-5, tot - tot[0]

    def force(R):
        st, r = scf.scf(H2_GRID, H2_H, R, Z, 1, n_inner=30, e_tol=1e-11, max_cycles=600)
        return forces.hf_forces(st.rho, H2_H, R, Z, st.a), r["E_total"]

    Ro, vo, eo = md.velocity_verlet(force, xyz, np.zeros((2, 3)), m, dt, 3)
    np.testing.assert_allclose(traj[:4], Ro, atol=1e-7)
    np.testing.assert_allclose(e[:4, 0], eo[:, 0], atol=1e-6)
    s.close()


def test_force_and_move_errors():
    torch, lbks = require_gpu()
    s = lbks.System(H2_GRID, H2_H, 1, precision=0)
    with pytest.raises(lbks.LbksError):  # no geometry yet
        lbks.lbks_forces(s.handle, 2)
    xyz, Z = _h2(1.4)
    s.set_geometry(xyz, Z)
    with pytest.raises(lbks.LbksError):  # capacity below 3 n_atoms
        lbks.lbks_forces(s.handle, 1)
    with pytest.raises(lbks.LbksError):  # outside the box
        s.move_atoms(xyz + np.array([0.0, 0.0, 50.0]))
    with pytest.raises(lbks.LbksError):
        lbks.lbks_relax_geometry(s.handle, 2, 10, -1.0, 0.5)
    with pytest.raises(lbks.LbksError):  # a non-positive mass
        s.md(2, 10.0, [1836.0, 0.0], np.zeros((2, 3)))
    with pytest.raises(lbks.LbksError):  # a non-positive time step
        s.md(2, 0.0, [1836.0, 1836.0], np.zeros((2, 3)))
    s.close()
