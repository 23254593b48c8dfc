"""Lattice-Boltzmann relaxation of the Kohn-Sham orbitals (oracle; test
infrastructure only).

Array layout: populations f[j, p, z, y, x] (orbital, velocity, grid), float64.

One step follows Eq. KSLB of Sec. 3:

    f_jp(r + v_p, t+1) = f_jp(r,t) - omega (f_jp - xi_p psi_j) + V_jp + W_jp
    V_jp = -dt chi_p V psi_j
    W_jp = -xi_p omega sum_{k<j} Lambda_jk psi_k,
    Lambda_jk = <psi_j|psi_k> / <psi_k|psi_k>,   psi_j = sum_p f_jp.

Readings taken where the paper is silent or garbled:
  * The source V_p carries a minus sign and the factor dt: the Wick-rotated
    equation (Sec. 3, first equation) has -V psi, so bound states (V < 0) grow.
  * Streaming is 'pull': the stored state is the post-collision f*, and the
    populations arriving at r are f*_jp(r - v_p).  Nothing streams in from
    outside the box (zero populations beyond the faces; the paper's open
    boundaries with extrapolation are not specified).
  * Normalisation (Sec. 3, 'upon normalisation'): before the collision of
    step t each orbital's arriving populations are scaled by
    sigma_j(t) = 1 / ||psi_j(t-1)||, the norm of that orbital at the previous
    step (h^3 measure).  At the fixed point the norm settles at the step
    operator's eigenvalue, which keeps the values bounded.
  * Lambda is evaluated at the same time t as the psi_k it multiplies.
  * Every n-th step (the end of a self-consistent cycle) the
    time-dependent Gram-Schmidt source is replaced by an exact Cholesky
    orthonormalisation of that step's orbitals: S = L L^T,
    f* <- L^{-1} f*_(no W), psi <- L^{-1} psi.  The lower-triangular L^{-1}
    keeps the paper's ordering (orbital j is orthogonalised against k < j).
"""
from __future__ import annotations

import numpy as np

from . import lattice


def shifted(a: np.ndarray, vx: int, vy: int, vz: int) -> np.ndarray:
    """out[..., z, y, x] = a[..., z - vz, y - vy, x - vx], zero where the source
    lies outside the grid."""
    out = np.zeros_like(a)
    nz, ny, nx = a.shape[-3:]

    def sl(v, n):
        if v >= 0:
            return slice(v, n), slice(0, n - v)
        return slice(0, n + v), slice(-v, n)

    dz, sz = sl(vz, nz)
    dy, sy = sl(vy, ny)
    dx, sx = sl(vx, nx)
    out[..., dz, dy, dx] = a[..., sz, sy, sx]
    return out


def pull_stream(fstar: np.ndarray) -> np.ndarray:
    """Streaming half of Eq. LBeq: f_p(r, t+1) = f*_p(r - v_p, t)."""
    out = np.empty_like(fstar)
    for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES):
        out[:, p] = shifted(fstar[:, p], int(vx), int(vy), int(vz))
    return out


def gram(psi: np.ndarray, h: float) -> np.ndarray:
    """Overlap matrix S_jk = <psi_j|psi_k> = h^3 sum_r psi_j psi_k
    (Eq. ORTOG as a lattice sum)."""
    m = psi.reshape(psi.shape[0], -1)
    return (h ** 3) * (m @ m.T)


def lambda_matrix(S: np.ndarray) -> np.ndarray:
    """Lambda_jk = S_jk / S_kk for k < j, zero elsewhere (Sec. 3, below Eq. KSLB)."""
    n = S.shape[0]
    lam = np.zeros_like(S)
    for j in range(n):
        for k in range(j):
            lam[j, k] = S[j, k] / S[k, k]
    return lam


def collide(f, psi, V, omega, theta, dt, lam=None):
    """BGK collision with potential and orthogonalisation sources (Eq. KSLB).

    f: arriving (already scaled) populations [j, p, z, y, x]; psi = sum_p f.
    lam: strictly lower triangular Lambda, or None for no W term."""
    xi = lattice.xi(theta)[None, :, None, None, None]
    chi = lattice.chi()[None, :, None, None, None]
    ps = psi[:, None]
    out = f - omega * (f - xi * ps) - dt * chi * V[None, None] * ps
    if lam is not None:
        w = np.tensordot(lam, psi, axes=(1, 0))  # sum_{k<j} Lambda_jk psi_k
        out = out - omega * xi * w[:, None]
    return out


def step(fstar, sigma, V, omega, theta, dt, h, orthonormalize=False):
    """One relaxation step of all orbitals.

    Returns a dict with the new post-collision populations ``fstar``, the
    orbitals ``psi`` of this step (after scaling; orthonormalised when
    ``orthonormalize``), their overlap ``S`` (before orthonormalisation), the
    Lambda used, and ``sigma`` for the next step."""
    f = pull_stream(fstar) * sigma[:, None, None, None, None]
    psi = f.sum(axis=1)
    S = gram(psi, h)
    if not orthonormalize:
        lam = lambda_matrix(S)
        fnew = collide(f, psi, V, omega, theta, dt, lam)
        return {"fstar": fnew, "psi": psi, "S": S, "lam": lam,
                "sigma": 1.0 / np.sqrt(np.diag(S))}
    L = np.linalg.cholesky(S)
    Linv = np.linalg.inv(L)
    fnew = np.tensordot(Linv, collide(f, psi, V, omega, theta, dt, None), axes=(1, 0))
    psi_o = np.tensordot(Linv, psi, axes=(1, 0))
    return {"fstar": fnew, "psi": psi_o, "S": S, "lam": None, "L": L,
            "sigma": np.ones(psi.shape[0])}


def orthonormalize(psi: np.ndarray, h: float) -> np.ndarray:
    """Cholesky orthonormalisation psi <- L^{-1} psi with h^3 psi psi^T = L L^T."""
    L = np.linalg.cholesky(gram(psi, h))
    return np.tensordot(np.linalg.inv(L), psi, axes=(1, 0))


def equilibrium(psi: np.ndarray, theta: float) -> np.ndarray:
    """f^e_jp = xi_p psi_j (Sec. 3)."""
    return lattice.xi(theta)[None, :, None, None, None] * psi[:, None]
