"""Pins of the concurrent-dynamics oracle (oracle/cd.py, Eq. KSLBCD of Sec. 3)
against closed forms, exact invariants of the two-step scheme and the
Born-Oppenheimer limit."""
import numpy as np
import pytest

from oracle import cd, forces, lattice, scf

THETA = 0.5


def _box_mode(n, m):
    """Product sine mode sin(pi m_a (i + 1) / (n_a + 1)): it vanishes one cell
    outside the box, so every symmetric stencil of the lattice maps it onto a
    multiple of itself, the stencil's symbol at k_a = pi m_a / (n_a + 1)."""
    s = [np.sin(np.pi * m[a] * (np.arange(n[a]) + 1) / (n[a] + 1)) for a in range(3)]
    k = [np.pi * m[a] / (n[a] + 1) for a in range(3)]
    return np.einsum("z,y,x->zyx", s[2], s[1], s[0]), k


def _symbol(w, k):
    return sum(w[p] * np.cos(k[0] * vx + k[1] * vy + k[2] * vz) for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES))


def _mode_energy(k, V0, dt):
    """eps of H = (1 - K_xi)/dt + K_chi V on a box mode at constant V."""
    return (1.0 - _symbol(lattice.xi(THETA), k)) / dt + V0 * _symbol(lattice.chi(), k)


@pytest.mark.parametrize("m,V0", [((1, 1, 1), -0.7), ((1, 2, 1), 0.3), ((3, 1, 2), -2.0)])
def test_box_mode_rotates_at_the_two_step_frequency(m, V0):
    """A box mode is an eigenvector of H at constant V; the exact solution of
    phi(t + tau) = phi(t - tau) - 2 i tau eps phi(t) is exp(-i Omega t) v with
    sin(Omega tau) = eps tau, at constant norm."""
    n, h = (9, 7, 6), 0.4
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.5 * dt
    mode, k = _box_mode(n, m)
    eps = _mode_energy(k, V0, dt)
    omega = np.arcsin(eps * tau) / tau
    V = np.full(mode.shape, V0)
    prev = mode[None].astype(complex)
    cur = prev * np.exp(-1j * omega * tau)
    for _ in range(80):
        prev, cur = cur, cd.cd_step(prev, cur, V, THETA, dt, h, tau)
    ref = mode * np.exp(-1j * omega * 81 * tau)
    assert np.abs(cur[0] - ref).max() < 1e-12 * np.abs(mode).max()


def test_two_orthogonal_box_modes_rotate_independently():
    """Two box modes of different m are orthogonal: Lambda = 0, the W source
    vanishes and each orbital keeps its own frequency."""
    n, h, V0 = (8, 7, 6), 0.35, -0.4
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.5 * dt
    modes, omegas = [], []
    for m in ((1, 1, 1), (2, 1, 1)):
        v, k = _box_mode(n, m)
        modes.append(v)
        omegas.append(np.arcsin(_mode_energy(k, V0, dt) * tau) / tau)
    V = np.full(modes[0].shape, V0)
    prev = np.array(modes, dtype=complex)
    cur = np.array([v * np.exp(-1j * w * tau) for v, w in zip(modes, omegas)])
    for _ in range(40):
        prev, cur = cur, cd.cd_step(prev, cur, V, THETA, dt, h, tau)
    for j in range(2):
        assert np.abs(cur[j] - modes[j] * np.exp(-1j * omegas[j] * 41 * tau)).max() < 1e-12


def test_start_is_the_second_order_taylor_step():
    """On an eigenvector the start is (1 - i x - x^2 / 2) v, x = eps tau."""
    n, h, V0 = (7, 6, 5), 0.4, -0.9
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.5 * dt
    mode, k = _box_mode(n, (1, 2, 1))
    x = _mode_energy(k, V0, dt) * tau
    got = cd.start(mode[None], np.full(mode.shape, V0), THETA, dt, h, tau)[0]
    np.testing.assert_allclose(got, (1 - 1j * x - 0.5 * x * x) * mode, atol=1e-14)


def test_hermitian_case_keeps_the_two_step_invariant():
    """At constant V, H is real symmetric and the scheme conserves
    Re <phi(t + tau)|phi(t)> exactly for any start: a dropped i, a streamed
    older level or a wrong factor breaks it."""
    rng = np.random.default_rng(3)
    n, h, V0 = (8, 6, 7), 0.3, -1.3
    dt = lattice.time_step(THETA, 1.0, h)
    tau = 0.5 * dt
    shape = (1, n[2], n[1], n[0])
    prev = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    cur = prev + 0.01 * (rng.normal(size=shape) + 1j * rng.normal(size=shape))
    V = np.full(shape[1:], V0)
    inv0 = cd.inner(cur, prev, h).real
    for _ in range(60):
        prev, cur = cur, cd.cd_step(prev, cur, V, THETA, dt, h, tau)
        assert abs(cd.inner(cur, prev, h).real - inv0) < 1e-12 * abs(inv0)


def test_u_source_adds_no_density_and_no_momentum():
    """sum_p w_p q_p = 0 and sum_p w_p q_p v_p = 0; the second moment is
    sum_p w_p q_p |v_p|^2 = 3 per unit of phi (lattice units)."""
    rng = np.random.default_rng(5)
    n = (11, 10, 9)
    g = np.zeros((n[2], n[1], n[0]))
    g[2:-2, 2:-2, 2:-2] = rng.normal(size=(n[2] - 4, n[1] - 4, n[0] - 4))
    kq = cd.pulled(g, cd.u_weights())
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    scale = np.abs(g).sum()
    assert abs(kq.sum()) < 1e-13 * scale
    for r in (x, y, z):
        assert abs((r * kq).sum()) < 1e-12 * scale * max(n)
    r2 = x * x + y * y + z * z
    assert abs((r2 * kq).sum() - 3.0 * g.sum()) < 1e-11 * scale * max(n) ** 2
    np.testing.assert_allclose(cd.u_weights()[[0, 1, 7]], [-1.5, 0.0, 0.125], atol=1e-15)


def test_lambda_removes_the_lower_orbitals_component():
    """a_j = phi_j - sum_k Lambda_jk phi_k is orthogonal to phi_k when the
    lower orbitals are orthogonal: the complex projection coefficient is
    <phi_k|phi_j> / <phi_k|phi_k> (a conjugated or transposed Lambda fails)."""
    rng = np.random.default_rng(11)
    n, h = (6, 5, 4), 0.5
    shape = (3, n[2], n[1], n[0])
    phi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    # make the two lower orbitals orthogonal, leave the top one general
    phi[1] -= cd.inner(phi[0], phi[1], h) / cd.inner(phi[0], phi[0], h) * phi[0]
    lam = cd.lambda_matrix(cd.overlap(phi, h))
    a = phi - np.tensordot(lam, phi, axes=(1, 0))
    for j in range(3):
        for k in range(j):
            scale = np.sqrt(cd.inner(phi[k], phi[k], h).real * cd.inner(phi[j], phi[j], h).real)
            assert abs(cd.inner(phi[k], a[j], h)) < 1e-13 * scale
    assert abs(lam[2, 0]) > 0.05 and abs(lam[2, 0].imag) > 0.01  # a general complex coefficient


def _h2(d):
    n, h = (22, 18, 18), 0.35
    Z = np.array([1.0, 1.0])
    xyz = np.array([[-d / 2, 0.0, 0.0], [d / 2, 0.0, 0.0]])
    st, r = scf.scf(n, h, xyz, Z, 1, n_inner=40, e_tol=1e-10, eig_tol=1e-8, rho_tol=1e-8, max_cycles=400)
    assert r["converged"]
    return n, h, xyz, Z, st, r


def test_ground_state_is_stationary():
    """The converged ground state rotates at Omega = arcsin(eps tau)/tau (eps
    its Rayleigh quotient of H) with density and energy unchanged, the
    potential rebuilt every ten steps."""
    n, h, xyz, Z, st, _ = _h2(1.4)
    run = cd.Run(st.psi, n, h, xyz, Z, theta=st.theta, v_h=st.v_h.copy())
    g = st.psi[0].astype(complex)
    hg = (g - cd.pulled(g, lattice.xi(st.theta))) / run.dt + cd.pulled(run.V * g, lattice.chi())
    eps = cd.inner(g, hg, h).real / cd.inner(g, g, h).real
    omega = np.arcsin(eps * run.tau) / run.tau
    rho0, e0 = run.rho.copy(), run.energies()["E_total"]
    for _ in range(20):
        run.block(10)
    assert run.steps == 201
    ov = cd.inner(g, run.cur[0], h)
    assert abs(abs(ov) - 1.0) < 1e-8
    assert abs(np.angle(ov * np.exp(1j * omega * run.steps * run.tau))) < 1e-6
    assert np.linalg.norm(run.rho - rho0) / np.linalg.norm(rho0) < 1e-8
    assert abs(run.energies()["E_total"] - e0) < 1e-8


def test_slowly_moving_h2_follows_born_oppenheimer():
    """Stretched H2 (d = 1.7 bohr, protons at rest) let go: over 61 a.u. the
    electrons follow the nuclei adiabatically.  E_KS + E_kin(nuclei) stays
    within 5e-6 Ha while 5e-3 Ha turns into nuclear kinetic energy (measured
    1.7e-6), and at the end the force and energy equal a converged
    Born-Oppenheimer solve at the same geometry within 1 % and 2e-5 Ha
    (measured 0.25 % and 6.7e-6 Ha)."""
    n, h, xyz, Z, st, _ = _h2(1.7)
    M = 1836.15267
    run = cd.Run(st.psi, n, h, xyz, Z, theta=st.theta, v_h=st.v_h.copy(), masses=[M, M])
    e = run.energies()
    total0 = e["E_total"] + e["E_kin_nuclei"]
    drift = 0.0
    for _ in range(200):
        run.block(10)
        e = run.energies()
        drift = max(drift, abs(e["E_total"] + e["E_kin_nuclei"] - total0))
    assert e["E_kin_nuclei"] > 4e-3
    assert drift < 5e-6
    d_end = run.xyz[1, 0] - run.xyz[0, 0]
    assert d_end > 1.8
    _, _, _, _, st2, r2 = _h2(d_end)
    f_bo = forces.hf_forces(st2.rho, h, run.xyz, Z, st2.a)
    assert abs(run.F[1, 0] - f_bo[1, 0]) < 0.01 * abs(f_bo[1, 0])
    assert abs(e["E_total"] - r2["E_total"]) < 2e-5
