"""Closed-form physics pins of the oracle's potentials and energies.

* Hartree potential of a Gaussian charge: V = q erf(r / (sqrt(2) s)) / r,
  E_H = q^2 / (2 sqrt(pi) s); second-order convergence in h.
* Slater exchange of the hydrogen 1s density rho = exp(-2r)/pi:
  E_x = -(81/256) 3^(1/3) pi^(-2/3) (worked out by hand from the LDA formula).
* PZ81 correlation: its two branches meet at r_s = 1 in value and slope, and
  v = d(rho eps)/d rho holds against finite differences.
* Kinetic operator of the equilibrium stencil on a normalised Gaussian of
  width s: <T> = 3 / (4 s^2) as h -> 0.
* Harmonic oscillator V = w^2 r^2 / 2 (w = 1): the relaxed orbital's energy tends to
  3w/2 (second order in h).
"""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle import energy, lattice, lb, lda, poisson


def _grid(nn, h):
    X, Y, Z = poisson.coords((nn, nn, nn), h)
    return X, Y, Z


def _gauss_rho(X, Y, Z, s, q=1.0, c=(0.0, 0.0, 0.0)):
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    return q * (2 * math.pi * s * s) ** -1.5 * np.exp(-r2 / (2 * s * s))


@pytest.mark.parametrize("c", [(0.0, 0.0, 0.0), (0.9, -0.6, 0.4)])
def test_hartree_of_gaussian_charge(c):
    s, L = 0.8, 12.0
    errs_v, errs_e = [], []
    for nn in (24, 48):
        h = L / nn
        X, Y, Z = _grid(nn, h)
        rho = _gauss_rho(X, Y, Z, s, 1.0, c)
        rho *= 1.0 / (rho.sum() * h ** 3)  # exactly unit lattice charge
        vh, it, res = poisson.hartree(rho, h, rtol=1e-12)
        assert res <= 1e-12
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        exact = np.where(r > 1e-12, erf(r / (math.sqrt(2) * s)) / np.maximum(r, 1e-300),
                         math.sqrt(2 / math.pi) / s)
        errs_v.append(float(np.abs(vh - exact).max()))
        eh = 0.5 * h ** 3 * float((vh * rho).sum())
        errs_e.append(abs(eh - 1.0 / (2 * math.sqrt(math.pi) * s)))
    # second order: halving h cuts the error by about four
    assert errs_v[1] < 0.35 * errs_v[0]
    assert errs_e[1] < 0.35 * errs_e[0]
    assert errs_v[1] < 6e-3 and errs_e[1] < 1e-3


def test_hartree_multipole_boundary_values_are_exact_for_point_like_charges():
    """Far from a compact charge the ghost-layer values equal the Coulomb sum
    of the lattice charges to O((d/R)^3): compare against the direct sum."""
    nn, h = 16, 0.5
    X, Y, Z = _grid(nn, h)
    rng = np.random.default_rng(5)
    rho = np.zeros_like(X)
    m = (np.abs(X) < 1.0) & (np.abs(Y) < 1.0) & (np.abs(Z) < 1.0)
    rho[m] = rng.uniform(0, 1, size=int(m.sum()))
    q, p, Q = poisson.multipoles(rho, h)
    R = np.array([[4.25, 0.25, -1.75], [-0.75, -4.25, 2.25], [3.0, 3.0, 3.0]])
    direct = [h ** 3 * float((rho / np.sqrt((X - a) ** 2 + (Y - b) ** 2 + (Z - cc) ** 2)).sum())
              for a, b, cc in R]
    mp = poisson.multipole_potential(q, p, Q, R[:, 0], R[:, 1], R[:, 2])
    np.testing.assert_allclose(mp, direct, rtol=3e-3)
    # without the dipole and quadrupole terms the error is an order larger
    mono = q / np.linalg.norm(R, axis=1)
    assert np.abs(mono - direct).max() > 5 * np.abs(mp - direct).max()


def test_hartree_energy_of_hydrogen_1s_density():
    """E_H of rho = exp(-2r)/pi is 5/16 Ha."""
    L, nn = 16.0, 64
    h = L / nn
    X, Y, Z = _grid(nn, h)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = np.exp(-2 * r) / math.pi
    vh, _, _ = poisson.hartree(rho, h, rtol=1e-12)
    eh = 0.5 * h ** 3 * float((vh * rho).sum())
    assert eh == pytest.approx(5.0 / 16.0, abs=4e-3)


def test_slater_exchange_of_hydrogen_1s_density():
    exact = -(81.0 / 256.0) * 3 ** (1 / 3) * math.pi ** (-2 / 3)
    assert exact == pytest.approx(-0.21275, abs=1e-5)
    vals = []
    for nn in (60, 120):
        h = 14.0 / nn
        X, Y, Z = _grid(nn, h)
        rho = np.exp(-2 * np.sqrt(X * X + Y * Y + Z * Z)) / math.pi
        ex, _ = lda.exchange(rho)
        vals.append(h ** 3 * float((rho * ex).sum()))
    assert abs(vals[1] - exact) < abs(vals[0] - exact)
    assert vals[1] == pytest.approx(exact, abs=2e-3)


def test_exchange_of_uniform_gas():
    """eps_x = -0.458165 / r_s (Slater exchange per electron)."""
    for rs in (0.5, 1.0, 2.0, 5.0):
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        ex, vx = lda.exchange(np.array([rho]))
        assert ex[0] == pytest.approx(-0.4581652932831429 / rs, rel=1e-12)
        assert vx[0] == pytest.approx(4.0 / 3.0 * ex[0], rel=1e-14)


def test_pz81_branches_meet_at_rs_one():
    e_hi, v_hi = lda.correlation(np.array([1.0]))
    e_lo, v_lo = lda.correlation(np.array([1.0 - 1e-12]))
    assert abs(e_hi[0] - e_lo[0]) < 5e-5
    assert abs(v_hi[0] - v_lo[0]) < 5e-5
    d = 1e-6
    slope_hi = (lda.correlation(np.array([1.0 + d]))[0] - e_hi)[0] / d
    slope_lo = (e_lo - lda.correlation(np.array([1.0 - d]))[0])[0] / d
    assert abs(slope_hi - slope_lo) < 5e-5


def test_xc_potential_is_derivative_of_energy_density():
    rho = np.logspace(-6, 2, 57)
    eps, v = lda.lda_xc(rho)
    d = 1e-6 * rho
    ep, _ = lda.lda_xc(rho + d)
    em, _ = lda.lda_xc(rho - d)
    fd = ((rho + d) * ep - (rho - d) * em) / (2 * d)
    np.testing.assert_allclose(v, fd, rtol=1e-7, atol=1e-12)
    # correlation is negative and smaller in size than exchange
    ec, _ = lda.correlation(np.cbrt(3 / (4 * math.pi * rho)))
    ex, _ = lda.exchange(rho)
    assert (ec < 0).all() and (np.abs(ec) < np.abs(ex)).all()


def test_xc_floor():
    eps, v = lda.lda_xc(np.array([0.0, 1e-20, lda.RHO_FLOOR * 0.5]))
    assert (eps == 0).all() and (v == 0).all()


def test_kinetic_operator_on_gaussian():
    s = 1.0
    errs = []
    for nn, h in ((24, 0.5), (48, 0.25)):
        X, Y, Z = _grid(nn, h)
        g = np.exp(-(X * X + Y * Y + Z * Z) / (2 * s * s))
        g /= math.sqrt(h ** 3 * float((g * g).sum()))
        t = h ** 3 * float((g * energy.apply_kinetic(g, 0.5, h)).sum())
        errs.append(abs(t - 3.0 / (4 * s * s)))
    assert errs[1] < 0.3 * errs[0]
    assert errs[1] < 0.011


def test_harmonic_oscillator_ground_state():
    """Box of half-width 3.9 bohr keeps the wall's effect below 1e-6 and
    dt * max V below one (the explicit scheme is unstable beyond)."""
    w = 1.0
    res = {}
    for nn, h in ((32, 0.25), (40, 0.2)):
        X, Y, Z = _grid(nn, h)
        V = 0.5 * w * w * (X * X + Y * Y + Z * Z)
        theta = 0.5
        dt = lattice.time_step(theta, 1.0, h)
        psi0 = np.exp(-0.4 * (X * X + Y * Y + Z * Z))[None]
        f = lb.equilibrium(lb.orthonormalize(psi0, h), theta)
        sigma = np.ones(1)
        for _ in range(900):
            r = lb.step(f, sigma, V, 1.0, theta, dt, h)
            f, sigma = r["fstar"], r["sigma"]
        psi = lb.orthonormalize(r["psi"], h)[0]
        e_rq = h ** 3 * float((psi * (energy.apply_kinetic(psi, theta, h) + V * psi)).sum())
        e_lam = (1.0 - math.sqrt(r["S"][0, 0])) / dt
        res[h] = (e_rq, e_lam)
    (a1, l1), (a2, l2) = res[0.25], res[0.2]
    for e1, e2 in ((a1, a2), (l1, l2)):
        assert abs(e2 - 1.5 * w) < abs(e1 - 1.5 * w)
        rich = (e2 * 0.25 ** 2 - e1 * 0.2 ** 2) / (0.25 ** 2 - 0.2 ** 2)
        assert rich == pytest.approx(1.5 * w, abs=2e-3)
    assert a2 == pytest.approx(1.5 * w, abs=0.02)
