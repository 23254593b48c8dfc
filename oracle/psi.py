"""Orbital-storage form of the relaxation at omega = 1 (oracle; test
infrastructure only).

At omega = 1 the collision of Eq. KSLB forgets the arriving populations:
every post-collision population of orbital j at site r is

    f*_jp(r) = xi_p a_j(r) - dt chi_p Vc(r) psi_j(r),
    a_j = psi_j - sum_{k<j} Lambda_jk psi_k          (the W source, Sec. 3),

a fixed combination of the site's orbital values, the potential Vc of that
collision and Lambda of that step.  The next step's pull-and-sum is then a
19-point stencil on psi alone:

    psi_j(t+1)(r) = sigma_j(t+1) sum_p f*_jp(r - v_p),   zero outside the box,

with sigma_j(t+1) = 1 / sqrt(S_jj(t)) as in ``lb.step``.  This module keeps
(psi, Lambda, Vc) instead of the 19 populations, forms each step's
populations from them and pulls them exactly as ``lb.pull_stream`` does; the
trajectory equals the population form of ``lb`` up to rounding (pinned in
the tests against ``lb.step``).  Only the memory differs: two orbital arrays
instead of 19 population arrays per orbital, which lets the oracle solve the
grids of the benchmark workloads.
"""
from __future__ import annotations

import numpy as np

from . import lattice
from .lb import gram, lambda_matrix


def _pull_add(out, src, vx, vy, vz):
    """out[z, y, x] += src[z - vz, y - vy, x - vx] where the source lies inside."""
    nz, ny, nx = src.shape

    def sl(v, n):
        if v >= 0:
            return slice(v, n), slice(0, n - v)
        return slice(0, n + v), slice(-v, n)

    dz, sz = sl(vz, nz)
    dy, sy = sl(vy, ny)
    dx, sx = sl(vx, nx)
    out[dz, dy, dx] += src[sz, sy, sx]


def pull_sum(a, b, theta, dt):
    """sum_p [xi_p a - dt chi_p b](r - v_p) for one orbital: the pulled sum of
    the populations xi_p a - dt chi_p b."""
    xi, chi = lattice.xi(theta), lattice.chi()
    out = np.zeros_like(a)
    pops = {}  # the population of each distinct (xi_p, chi_p): rest, axis and diagonal velocities
    for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES):
        key = (xi[p], chi[p])
        if key not in pops:
            pops[key] = xi[p] * a - dt * chi[p] * b
        _pull_add(out, pops[key], int(vx), int(vy), int(vz))
    return out


class PsiState:
    """State between steps: orbitals psi (after the step's scaling), Lambda of
    that step (None after an orthonormalising step or at the start) and the
    potential Vc of the collision that produced the stored populations (None:
    the start f* = xi psi, which has no potential term)."""

    def __init__(self, psi):
        self.psi = psi
        self.lam = None
        self.vc = None


def populations_a_b(st: PsiState):
    """(a_j, b_j) of every orbital: f*_jp = xi_p a_j - dt chi_p b_j."""
    a = st.psi.copy()
    if st.lam is not None:
        a = a - np.tensordot(st.lam, st.psi, axes=(1, 0))
    b = np.zeros_like(st.psi) if st.vc is None else st.vc[None] * st.psi
    return a, b


def step(st: PsiState, sigma, V, theta, dt, h, orthonormalize=False):
    """One step of Eq. KSLB at omega = 1 in orbital storage; the counterpart
    of ``lb.step(..., omega=1)``.  Returns the same keys except ``fstar``
    (the new state is written into ``st``)."""
    a, b = populations_a_b(st)
    psi = np.empty_like(st.psi)
    for j in range(psi.shape[0]):
        psi[j] = sigma[j] * pull_sum(a[j], b[j], theta, dt)
    S = gram(psi, h)
    st.vc = V
    if not orthonormalize:
        st.psi, st.lam = psi, lambda_matrix(S)
        return {"psi": psi, "S": S, "lam": st.lam, "sigma": 1.0 / np.sqrt(np.diag(S))}
    L = np.linalg.cholesky(S)
    st.psi, st.lam = np.tensordot(np.linalg.inv(L), psi, axes=(1, 0)), None
    return {"psi": st.psi, "S": S, "lam": None, "L": L, "sigma": np.ones(psi.shape[0])}
