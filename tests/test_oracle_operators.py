"""Pins of the oracle's relaxation against brute force and closed forms.

* At omega = 1 the populations collapse onto psi and one step is the
  psi-only operator T = K_xi - dt M_chi V.  A dense T assembled site by site
  (independently of the oracle's array shifting) must give the eigenpair the
  relaxation converges to (Sec. 3, eigen-expansion argument: upon
  normalisation the ground state survives).
* With V = 0 (or constant) in a box with zero boundary values the
  eigenvectors of every stencil are products of sines, with eigenvalues in
  closed form; the orthogonalisation source of Eq. KSLB must make orbital j
  converge to the j-th mode (Sec. 3, time-dependent Gram-Schmidt).
* For any omega the second moment of a free pulse must grow at twice the diffusivity
  theta (1/omega - 1/2) (Sec. 3, relation between omega and D).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lattice, lb


def _dense_T(n, V, theta, dt):
    """psi(t+1)(r) = sum_p [xi_p psi(r - v_p) - dt chi_p V(r - v_p) psi(r - v_p)],
    assembled entry by entry."""
    nx, ny, nz = n
    N = nx * ny * nz
    T = np.zeros((N, N))
    xi, chi = lattice.xi(theta), lattice.chi()
    idx = lambda x, y, z: x + nx * (y + ny * z)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(x, y, z)
                for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES):
                    sx, sy, sz = x - vx, y - vy, z - vz
                    if 0 <= sx < nx and 0 <= sy < ny and 0 <= sz < nz:
                        j = idx(sx, sy, sz)
                        T[i, j] += xi[p] - dt * chi[p] * V[sz, sy, sx]
    return T


def _relax(psi0, V, omega, theta, dt, h, steps, ortho_every=None):
    f = lb.equilibrium(lb.orthonormalize(psi0, h), theta)
    sigma = np.ones(psi0.shape[0])
    r = None
    for t in range(steps):
        ortho = ortho_every is not None and (t + 1) % ortho_every == 0
        r = lb.step(f, sigma, V, omega, theta, dt, h, orthonormalize=ortho)
        f, sigma = r["fstar"], r["sigma"]
    return r


def _angle(a, b):
    """Sine of the angle between two grid functions, from the residual of the
    projection (accurate down to round-off, unlike 1 - cos^2)."""
    a = a.ravel() / np.linalg.norm(a)
    b = b.ravel() / np.linalg.norm(b)
    return float(np.linalg.norm(a - (a @ b) * b))


def test_single_orbital_converges_to_dense_dominant_eigenpair():
    n, h, theta = (5, 6, 7), 0.5, 0.5
    dt = lattice.time_step(theta, 1.0, h)
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz) - 3.0, np.arange(ny) - 2.5, np.arange(nx) - 2.0, indexing="ij")
    V = -3.0 / np.sqrt((h * X) ** 2 + (h * Y) ** 2 + (h * Z) ** 2 + h * h) + 0.3 * (h * X)
    T = _dense_T(n, V, theta, dt)
    w, U = np.linalg.eig(T)
    k = int(np.argmax(w.real))
    lam0, u0 = float(w[k].real), U[:, k].real
    rng = np.random.default_rng(0)
    r = _relax(rng.uniform(0.5, 1.0, size=(1,) + V.shape), V, 1.0, theta, dt, h, 600)
    psi = r["psi"][0]
    assert _angle(psi, u0) < 1e-10
    # the norm of the scaled orbital settles at the dominant eigenvalue
    assert math.sqrt(r["S"][0, 0]) == pytest.approx(lam0, abs=1e-12)


def test_omega_one_step_equals_psi_only_operator():
    """At omega = 1 two consecutive oracle steps satisfy
    psi(t+1) = sigma(t+1) T psi(t) to round-off."""
    n, h, theta = (4, 5, 6), 0.4, 0.45
    dt = lattice.time_step(theta, 1.0, h)
    rng = np.random.default_rng(1)
    V = rng.uniform(-4, 1, size=(n[2], n[1], n[0]))
    T = _dense_T(n, V, theta, dt)
    f = rng.uniform(-1, 1, size=(1, 19, n[2], n[1], n[0]))
    sigma = np.array([0.7])
    r1 = lb.step(f, sigma, V, 1.0, theta, dt, h)
    r2 = lb.step(r1["fstar"], r1["sigma"], V, 1.0, theta, dt, h)
    np.testing.assert_allclose(r2["psi"][0].ravel(), r1["sigma"][0] * (T @ r1["psi"][0].ravel()),
                               rtol=1e-13, atol=1e-13)


def _box_modes(n, count, value):
    """Top `count` sine modes of the box, by the closed-form eigenvalue `value(c)`."""
    nx, ny, nz = n
    cands = []
    for m in itertools.product(range(1, nx + 1), range(1, ny + 1), range(1, nz + 1)):
        c = [math.cos(math.pi * m[a] / (n[a] + 1)) for a in range(3)]
        cands.append((value(c), m))
    cands.sort(key=lambda t: -t[0])
    return cands[:count]


def _sine_mode(n, m):
    nx, ny, nz = n
    sx = np.sin(math.pi * m[0] * (np.arange(nx) + 1) / (nx + 1))
    sy = np.sin(math.pi * m[1] * (np.arange(ny) + 1) / (ny + 1))
    sz = np.sin(math.pi * m[2] * (np.arange(nz) + 1) / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def _stencil_symbol(wts, c):
    """sum_p w_p prod_a cos(k_a v_pa) for a weight vector that depends only
    on |v|^2: w0 + 2 w1 (cx+cy+cz) + 4 w2 (cx cy + cy cz + cz cx)."""
    w0, w1, w2 = wts[0], wts[1], wts[7]
    return w0 + 2 * w1 * (c[0] + c[1] + c[2]) + 4 * w2 * (c[0] * c[1] + c[1] * c[2] + c[2] * c[0])


@pytest.mark.parametrize("v0,ortho_every", [(0.0, None), (-1.5, None), (0.0, 25)])
def test_box_modes_with_gram_schmidt_source(v0, ortho_every):
    n, h, theta = (4, 5, 6), 0.5, 0.5
    dt = lattice.time_step(theta, 1.0, h)
    xi, chi = lattice.xi(theta), lattice.chi()
    lam = lambda c: _stencil_symbol(xi, c) - dt * v0 * _stencil_symbol(chi, c)
    modes = _box_modes(n, 4, lam)
    assert modes[2][0] - modes[3][0] > 1e-3  # top three are separated from the rest
    V = np.full((n[2], n[1], n[0]), v0)
    rng = np.random.default_rng(2)
    r = _relax(rng.uniform(-1, 1, size=(3,) + V.shape), V, 1.0, theta, dt, h, 3000, ortho_every)
    for j in range(3):
        assert _angle(r["psi"][j], _sine_mode(n, modes[j][1])) < 1e-8
        if ortho_every is None:
            assert math.sqrt(r["S"][j, j]) == pytest.approx(modes[j][0], abs=1e-10)


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.3])
def test_second_moment_grows_at_twice_the_diffusivity(omega):
    """Without potential, a pulse far from the faces spreads with
    d<x_a^2>/dt = 2 D per step in every direction, D = theta (1/omega - 1/2)
    (Sec. 3, relation between omega and the diffusivity)."""
    D = 0.15
    theta = D / (1.0 / omega - 0.5)
    nn, h = 40, 1.0
    dt = lattice.time_step(theta, omega, h)
    c = np.arange(nn) - (nn - 1) / 2.0
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    psi0 = np.exp(-((X - 0.3) ** 2 + (Y + 0.2) ** 2 + Z ** 2) / (2 * 1.5 ** 2))[None]
    f = lb.equilibrium(psi0, theta)
    sigma = np.ones(1)
    V = np.zeros_like(X)
    m2 = []
    for t in range(24):  # transients have decayed, the pulse has not reached the faces
        r = lb.step(f, sigma, V, omega, theta, dt, h)
        f, sigma = r["fstar"], r["sigma"]
        psi = r["psi"][0]
        mass = psi.sum()
        mx = (X * psi).sum() / mass
        m2.append([((X - mx) ** 2 * psi).sum() / mass, (Y ** 2 * psi).sum() / mass,
                   (Z ** 2 * psi).sum() / mass])
    m2 = np.array(m2)
    growth = (m2[-1] - m2[-11]) / 10.0
    np.testing.assert_allclose(growth, 2 * D, rtol=1e-4)
