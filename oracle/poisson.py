"""Hartree potential by a lattice Poisson solve (oracle; test infrastructure only).

The Kohn-Sham Hamiltonian of Sec. 2 contains the Hartree integral
int rho(r') / |r - r'| dr'.  The paper does not say how it evaluates it.
Reading taken here: V_H solves the 7-point finite-difference Poisson equation

    (sum_{6 face neighbours} V - 6 V) / h^2 = -4 pi rho

on the n^3 grid, with V on the one-cell layer outside the faces fixed to the
multipole expansion (monopole, dipole, quadrupole about the box centre) of
the lattice charge.  The discrete system is solved by textbook conjugate
gradients to a relative residual tolerance.
"""
from __future__ import annotations

import numpy as np


def coords(n, h):
    nx, ny, nz = n
    x = (np.arange(nx) - (nx - 1) / 2.0) * h
    y = (np.arange(ny) - (ny - 1) / 2.0) * h
    z = (np.arange(nz) - (nz - 1) / 2.0) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def multipoles(rho, h):
    """q = h^3 sum rho, p_a = h^3 sum rho r_a, Q_ab = h^3 sum rho (3 r_a r_b - r^2 d_ab)."""
    nz, ny, nx = rho.shape
    X, Y, Z = coords((nx, ny, nz), h)
    w = rho * h ** 3
    r = [X, Y, Z]
    q = w.sum()
    p = np.array([(w * r[a]).sum() for a in range(3)])
    r2 = X * X + Y * Y + Z * Z
    Q = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            Q[a, b] = (w * (3.0 * r[a] * r[b] - (r2 if a == b else 0.0))).sum()
    return q, p, Q


def multipole_potential(q, p, Q, X, Y, Z):
    """V(R) = q/|R| + p.R/|R|^3 + (1/2) sum_ab Q_ab R_a R_b / |R|^5."""
    R = [X, Y, Z]
    r2 = X * X + Y * Y + Z * Z
    r = np.sqrt(r2)
    v = q / r
    for a in range(3):
        v = v + p[a] * R[a] / (r2 * r)
    quad = np.zeros_like(X)
    for a in range(3):
        for b in range(3):
            quad = quad + Q[a, b] * R[a] * R[b]
    return v + 0.5 * quad / (r2 * r2 * r)


def laplacian_operator(v):
    """A v = 6 v - sum of the six face neighbours (zero outside the grid)."""
    out = 6.0 * v
    out[1:, :, :] -= v[:-1, :, :]
    out[:-1, :, :] -= v[1:, :, :]
    out[:, 1:, :] -= v[:, :-1, :]
    out[:, :-1, :] -= v[:, 1:, :]
    out[:, :, 1:] -= v[:, :, :-1]
    out[:, :, :-1] -= v[:, :, 1:]
    return out


def boundary_values(rho, h):
    """Multipole values on the ghost layer, summed into the right-hand side of
    each boundary site (one entry per outward face)."""
    nz, ny, nx = rho.shape
    q, p, Q = multipoles(rho, h)
    X, Y, Z = coords((nx, ny, nz), h)
    g = np.zeros_like(rho)
    # x faces: ghost at x0 - h and x_{n-1} + h
    for axis, n, arr in ((2, nx, X), (1, ny, Y), (0, nz, Z)):
        for side in (0, -1):
            idx = [slice(None)] * 3
            idx[axis] = slice(0, 1) if side == 0 else slice(n - 1, n)
            Xs, Ys, Zs = X[tuple(idx)].copy(), Y[tuple(idx)].copy(), Z[tuple(idx)].copy()
            shift = -h if side == 0 else h
            if axis == 2:
                Xs = Xs + shift
            elif axis == 1:
                Ys = Ys + shift
            else:
                Zs = Zs + shift
            g[tuple(idx)] += multipole_potential(q, p, Q, Xs, Ys, Zs)
    return g


def conjugate_gradient(apply_a, b, x0, rtol, max_iter=100000):
    """Textbook CG for a symmetric positive definite operator."""
    x = x0.copy()
    r = b - apply_a(x)
    p = r.copy()
    rr = float((r * r).sum())
    bnorm = float(np.sqrt((b * b).sum()))
    it = 0
    while np.sqrt(rr) > rtol * bnorm and it < max_iter:
        ap = apply_a(p)
        alpha = rr / float((p * ap).sum())
        x += alpha * p
        r -= alpha * ap
        rr_new = float((r * r).sum())
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / bnorm


def hartree(rho, h, x0=None, rtol=1e-12):
    """V_H on the grid; returns (V_H, iterations, final relative residual)."""
    b = 4.0 * np.pi * h * h * rho + boundary_values(rho, h)
    if x0 is None:
        x0 = np.zeros_like(rho)
    return conjugate_gradient(laplacian_operator, b, x0, rtol)
