"""Pins of the oracle's lattice tables and collision against what Sec. 3 of the
paper states: normalised weights, the equilibrium's moments, the source's
vanishing first and second moments, and the collision invariants."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice, lb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q19_weights.json")


def _cls(v):
    v2 = int((v ** 2).sum())
    return {0: "rest", 1: "axis", 2: "diagonal"}[v2]


def _frac(pair):
    return float(Fraction(pair[0], pair[1]))


def test_weights_and_tables_match_hand_derived_rationals():
    g = json.load(open(GOLDEN))
    w, q, chi = lattice.weights(), lattice.hermite2(), lattice.chi()
    for p, v in enumerate(lattice.VELOCITIES):
        c = _cls(v)
        assert w[p] == pytest.approx(_frac(g["w"][c]), abs=1e-15)
        assert q[p] == pytest.approx(_frac(g["q"][c]), abs=1e-14)
        assert chi[p] == pytest.approx(_frac(g["chi"][c]), abs=1e-15)
        assert lattice.xi(0.5)[p] == pytest.approx(_frac(g["xi_theta_1_2"][c]), abs=1e-15)
        # theta = c_s^2 reduces the equilibrium weights to the lattice weights
        assert lattice.xi(1.0 / 3.0)[p] == pytest.approx(_frac(g["xi_theta_1_3"][c]), abs=1e-15)


def test_velocity_set_is_d3q19_with_opposites():
    v = lattice.VELOCITIES
    assert v.shape == (19, 3)
    assert len({tuple(x) for x in v}) == 19
    for x in v:
        assert any((y == -x).all() for y in v)
    assert sorted((v ** 2).sum(1).tolist()) == [0] + [1] * 6 + [2] * 12


@pytest.mark.parametrize("theta", [0.2, 1.0 / 3.0, 0.5, 0.8])
def test_equilibrium_moments(theta):
    """sum xi = 1, sum xi v = 0, sum xi v v = theta I: f^e = xi psi has density
    psi, no momentum, and second moment theta psi (Sec. 3)."""
    v = lattice.VELOCITIES.astype(float)
    xi = lattice.xi(theta)
    assert xi.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(xi @ v, 0.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("p,pa,pb->ab", xi, v, v), theta * np.eye(3), atol=1e-15)


def test_lattice_weight_isotropy():
    v = lattice.VELOCITIES.astype(float)
    w = lattice.weights()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(np.einsum("p,pa,pb->ab", w, v, v), lattice.CS2 * np.eye(3), atol=1e-15)
    m4 = np.einsum("p,pa,pb,pc,pd->abcd", w, v, v, v, v)
    d = np.eye(3)
    iso = lattice.CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                              + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(m4, iso, atol=1e-15)


def test_source_weights_moments():
    """sum chi = 1 and zero first and second moments (Sec. 3, definition of V_p)."""
    v = lattice.VELOCITIES.astype(float)
    chi = lattice.chi()
    assert chi.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(chi @ v, 0.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("p,pa,pb->ab", chi, v, v), 0.0, atol=1e-15)


def test_time_step_matches_diffusivity_relation():
    """theta (1/omega - 1/2) = dt / (2 h^2) (Sec. 3, relation between omega and D)."""
    for theta, omega, h in [(0.5, 1.0, 0.2), (0.3, 0.8, 0.4), (0.6, 1.3, 0.25)]:
        dt = lattice.time_step(theta, omega, h)
        assert theta * (1.0 / omega - 0.5) == pytest.approx(dt / (2 * h * h), rel=1e-14)


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.4])
def test_collision_invariants(omega):
    """Without sources the BGK collision keeps psi = sum_p f at every site,
    damps the first moment by (1 - omega) and relaxes the second moment
    towards theta psi I (Eq. LBeq)."""
    rng = np.random.default_rng(3)
    theta, dt = 0.45, 0.07
    f = rng.uniform(-1, 1, size=(2, 19, 3, 4, 5))
    psi = f.sum(1)
    V = np.zeros(psi.shape[1:])
    out = lb.collide(f, psi, V, omega, theta, dt, None)
    v = lattice.VELOCITIES.astype(float)
    np.testing.assert_allclose(out.sum(1), psi, atol=1e-14)
    np.testing.assert_allclose(np.einsum("jpzyx,pa->jazyx", out, v),
                               (1 - omega) * np.einsum("jpzyx,pa->jazyx", f, v), atol=1e-14)
    m2_in = np.einsum("jpzyx,pa,pb->jabzyx", f, v, v)
    m2_out = np.einsum("jpzyx,pa,pb->jabzyx", out, v, v)
    target = theta * np.einsum("ab,jzyx->jabzyx", np.eye(3), psi)
    np.testing.assert_allclose(m2_out, (1 - omega) * m2_in + omega * target, atol=1e-13)


def test_potential_and_orthogonalisation_source_moments():
    """The potential source changes only the zeroth moment, by -dt V psi; the
    W source changes the zeroth moment by -omega sum_k Lambda_jk psi_k and
    leaves the first moment alone (Sec. 3)."""
    rng = np.random.default_rng(4)
    theta, dt, omega = 0.5, 0.05, 0.9
    f = rng.uniform(-1, 1, size=(3, 19, 3, 4, 5))
    psi = f.sum(1)
    V = rng.uniform(-2, 1, size=psi.shape[1:])
    lam = np.tril(rng.uniform(-0.5, 0.5, size=(3, 3)), -1)
    base = lb.collide(f, psi, np.zeros_like(V), omega, theta, dt, None)
    withv = lb.collide(f, psi, V, omega, theta, dt, None)
    withw = lb.collide(f, psi, np.zeros_like(V), omega, theta, dt, lam)
    v = lattice.VELOCITIES.astype(float)
    dv = withv - base
    np.testing.assert_allclose(dv.sum(1), -dt * V * psi, atol=1e-14)
    np.testing.assert_allclose(np.einsum("jpzyx,pa->jazyx", dv, v), 0.0, atol=1e-14)
    np.testing.assert_allclose(np.einsum("jpzyx,pa,pb->jabzyx", dv, v, v), 0.0, atol=1e-14)
    dw = withw - base
    np.testing.assert_allclose(dw.sum(1), -omega * np.tensordot(lam, psi, axes=(1, 0)), atol=1e-14)
    np.testing.assert_allclose(np.einsum("jpzyx,pa->jazyx", dw, v), 0.0, atol=1e-14)


def test_streaming_moves_each_population_along_its_velocity():
    """A single population at site r with velocity v_p arrives at r + v_p; one
    that would leave the box is gone (Eq. LBeq, left-hand side)."""
    n = (5, 6, 7)
    for p, vel in enumerate(lattice.VELOCITIES):
        f = np.zeros((1, 19, n[2], n[1], n[0]))
        x, y, z = 2, 3, 3
        f[0, p, z, y, x] = 1.0
        g = lb.pull_stream(f)
        assert g.sum() == 1.0
        assert g[0, p, z + vel[2], y + vel[1], x + vel[0]] == 1.0
        # at a face the outgoing population leaves the box
        f2 = np.zeros_like(f)
        f2[0, p, 0, 0, 0] = 1.0
        expect_inside = (vel >= 0).all()
        assert lb.pull_stream(f2).sum() == (1.0 if expect_inside else 0.0)
