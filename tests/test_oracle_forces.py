"""Pins of the oracle's Hellmann-Feynman forces (oracle.forces) against what
the mathematics fixes: central differences of the electron-nucleus energy
through the solver-side V_ext routine (scf.external_potential) and of the
nucleus-nucleus energy (energy.nuclear_repulsion), mirror symmetry, Newton's
third law for the nuclear term, and -dE_total/dR from two self-consistent
oracle solves of H2."""
import numpy as np

from oracle import energy, forces, scf


def _blob_density(n, h, seed):
    """A positive density of a few Gaussian blobs on an n grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = scf.grid_coords(n, h)
    rho = np.zeros_like(X)
    for _ in range(3):
        c = rng.uniform(-1.0, 1.0, 3)
        w = rng.uniform(0.6, 1.2)
        rho += rng.uniform(0.2, 1.0) * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * w * w))
    return rho


def test_electron_nucleus_force_is_minus_the_energy_gradient():
    n, h, a = (14, 12, 11), 0.35, 0.35
    rho = _blob_density(n, h, 3)
    xyz = np.array([[0.3, -0.2, 0.1], [-0.9, 0.4, -0.3], [0.5, 0.8, 0.6]])
    Z = np.array([8.0, 1.0, 1.0])

    def e_ext(R):
        return h ** 3 * (rho * scf.external_potential(n, h, R, Z, a)).sum()

    F = forces.electron_nucleus(rho, h, xyz, Z, a)
    d = 1e-5
    for I in range(len(Z)):
        for c in range(3):
            Rp, Rm = xyz.copy(), xyz.copy()
            Rp[I, c] += d
            Rm[I, c] -= d
            fd = -(e_ext(Rp) - e_ext(Rm)) / (2 * d)
            assert abs(F[I, c] - fd) <= 1e-7 * max(1.0, abs(fd)), (I, c, F[I, c], fd)


def test_nuclear_force_is_minus_the_repulsion_gradient_and_sums_to_zero():
    xyz = np.array([[0.0, 0.0, 0.0], [1.8, 0.2, -0.1], [-0.5, 1.7, 0.4], [0.3, -0.6, 1.9]])
    Z = np.array([6.0, 1.0, 1.0, 1.0])
    F = forces.nuclear(xyz, Z)
    d = 1e-6
    for I in range(len(Z)):
        for c in range(3):
            Rp, Rm = xyz.copy(), xyz.copy()
            Rp[I, c] += d
            Rm[I, c] -= d
            fd = -(energy.nuclear_repulsion(Rp, Z) - energy.nuclear_repulsion(Rm, Z)) / (2 * d)
            assert abs(F[I, c] - fd) <= 1e-7 * max(1.0, abs(fd))
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)


def test_mirror_symmetric_density_pulls_a_centred_nucleus_nowhere():
    """rho(x) = rho(-x) about a nucleus on the mirror plane: no x force."""
    n, h = (16, 13, 12), 0.3  # x coordinates symmetric about 0
    rho = _blob_density(n, h, 5)
    rho = rho + rho[:, :, ::-1]
    F = forces.electron_nucleus(rho, h, np.array([[0.0, 0.2, -0.1]]), np.array([3.0]), h)
    assert abs(F[0, 0]) < 1e-13 * np.abs(F).max()
    assert np.abs(F[0, 1:]).max() > 1e-3


def test_hf_force_matches_the_scf_energy_difference_for_h2():
    """-dE_total/dd by a central difference of two converged oracle solves
    against the Hellmann-Feynman force at d: agreement to 3e-3 relative (the
    lattice scheme's fixed point is not exactly a minimum of the energy
    functional -- the source carries the chi-weighted potential -- and the
    difference has an O(dd^2) error; measured 1.1e-3)."""
    n, h, d, dd = (22, 18, 18), 0.35, 1.4, 0.02
    Z = np.array([1.0, 1.0])

    def solve(sep):
        xyz = np.array([[-sep / 2, 0.0, 0.0], [sep / 2, 0.0, 0.0]])
        st, r = scf.scf(n, h, xyz, Z, 1, n_inner=40, e_tol=1e-10, max_cycles=400)
        assert r["converged"]
        return st, r, xyz

    st, _, xyz = solve(d)
    F = forces.hf_forces(st.rho, h, xyz, Z, st.a)
    fd = -(solve(d + dd)[1]["E_total"] - solve(d - dd)[1]["E_total"]) / (2 * dd)  # force on the +x nucleus
    assert abs(F[1, 0] - fd) <= 3e-3 * abs(fd), (F[1, 0], fd)
    np.testing.assert_allclose(F[0], -F[1], atol=1e-6)  # the two nuclei, mirror images
    assert np.abs(F[:, 1:]).max() < 1e-6


def test_velocity_verlet_follows_the_harmonic_oscillator():
    """F = -k x: the closed form x(t) = x0 cos(w t), w = sqrt(k/m), to
    O(dt^2); the energy stays within O(dt^2) of its start; reversing the
    final velocity retraces the path (time reversibility)."""
    from oracle import md

    k, m, x0, dt, n = 2.0, 3.0, 0.7, 0.01, 2000
    w = np.sqrt(k / m)

    def force(R):
        return -k * R, 0.5 * k * float((R * R).sum())

    R, v, e = md.velocity_verlet(force, np.array([[x0, 0.0, 0.0]]), np.zeros((1, 3)), [m], dt, n)
    t = dt * np.arange(n + 1)
    np.testing.assert_allclose(R[:, 0, 0], x0 * np.cos(w * t), atol=2e-4)
    tot = e.sum(axis=1)
    assert np.abs(tot - tot[0]).max() < 1e-4 * tot[0]
    Rb, _, _ = md.velocity_verlet(force, R[-1], -v[-1], [m], dt, n)
    np.testing.assert_allclose(Rb[-1], R[0], atol=1e-9)
