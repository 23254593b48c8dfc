"""Self-consistent Kohn-Sham ground state by lattice-kinetic relaxation
(oracle; test infrastructure only).

Born-Oppenheimer scenario of Sec. 3.1: nuclei fixed, the orbitals relax in
imaginary time (Eq. KSLB) while the density, the Hartree potential and the
exchange-correlation potential are rebuilt from them.

Cycle structure (a reading; the paper interleaves the potential update with
the relaxation without saying how often):

  init   psi0_j on the grid (see initial_orbitals), Cholesky-orthonormalised;
         f*_jp = xi_p psi_j; sigma = 1; rho = 2 sum_j psi_j^2;
         V = V_ext + V_H[rho] + v_xc[rho]; E_0 from these orbitals.
  cycle  n_inner - 1 steps of Eq. KSLB at fixed V, then one step whose
         orthogonalisation source is replaced by Cholesky orthonormalisation;
         rho, V_H (warm-started), v_xc, V_out and the energies from the
         orthonormal orbitals of that step; stop when |E_c - E_{c-1}| < e_tol;
         otherwise V <- mix V_out + (1 - mix) V.
"""
from __future__ import annotations

import math

import numpy as np

from . import energy, lattice, lb, lda, poisson


def grid_coords(n, h):
    return poisson.coords(n, h)


def external_potential(n, h, xyz, Z, a):
    """Softened Coulomb nuclei: V_ext(r) = -sum_I Z_I / sqrt(|r - R_I|^2 + a^2)."""
    X, Y, Zc = grid_coords(n, h)
    v = np.zeros_like(X)
    for I in range(len(Z)):
        d2 = (X - xyz[I, 0]) ** 2 + (Y - xyz[I, 1]) ** 2 + (Zc - xyz[I, 2]) ** 2
        v -= Z[I] / np.sqrt(d2 + a * a)
    return v


def initial_orbitals(n, h, xyz, Z, n_orb):
    """Gaussian initial orbitals (a reading of 'Gaussian initial orbital').

    Nuclei are ordered by decreasing charge (stable).  Orbital j sits on
    nucleus I = order[j mod n_atoms], shell m = j div n_atoms:
        c_j = R_I + 0.25 (sin(1 + 2.1 j), sin(2 + 3.3 j), sin(3 + 4.7 j))
        s_j = 1.2 (1 + 0.35 m)
        psi0_j(r) = exp(-|r - c_j|^2 / (2 s_j^2))
    The small offsets break the molecule's point symmetry so that every
    symmetry component is present in every start vector."""
    X, Y, Zc = grid_coords(n, h)
    order = sorted(range(len(Z)), key=lambda i: -Z[i])
    out = np.empty((n_orb,) + X.shape)
    for j in range(n_orb):
        I = order[j % len(Z)]
        m = j // len(Z)
        c = xyz[I] + 0.25 * np.array([math.sin(1.0 + 2.1 * j), math.sin(2.0 + 3.3 * j),
                                      math.sin(3.0 + 4.7 * j)])
        s = 1.2 * (1.0 + 0.35 * m)
        d2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Zc - c[2]) ** 2
        out[j] = np.exp(-d2 / (2.0 * s * s))
    return out


def density(psi):
    """rho = sum_j 2 |psi_j|^2 (Sec. 2, closed shell)."""
    return 2.0 * (psi * psi).sum(axis=0)


class State:
    """Everything the loop carries between cycles."""

    def __init__(self, n, h, xyz, Z, n_orb, theta=0.5, omega=1.0, softening=0.0,
                 poisson_rtol=1e-12):
        self.n, self.h = tuple(n), float(h)
        self.xyz, self.Z = np.asarray(xyz, float), np.asarray(Z, float)
        self.n_orb = n_orb
        self.theta, self.omega = float(theta), float(omega)
        self.dt = lattice.time_step(theta, omega, h)
        self.a = softening if softening > 0 else h
        self.poisson_rtol = poisson_rtol
        self.v_ext = external_potential(self.n, h, self.xyz, self.Z, self.a)
        psi = lb.orthonormalize(initial_orbitals(self.n, h, self.xyz, self.Z, n_orb), h)
        self.fstar = lb.equilibrium(psi, theta)
        self.sigma = np.ones(n_orb)
        self.v_h = np.zeros(psi.shape[1:])
        self.steps = 0
        self.terms = self.evaluate(psi)
        self.v_in = self.v_out.copy()

    def evaluate(self, psi):
        """Density, potentials and energies of orthonormal orbitals psi."""
        self.psi = psi
        self.rho = density(psi)
        self.v_h, self.poisson_iters, _ = poisson.hartree(self.rho, self.h, self.v_h, self.poisson_rtol)
        self.eps_xc, v_xc = lda.lda_xc(self.rho)
        self.v_out = self.v_ext + self.v_h + v_xc
        return energy.energies(psi, self.rho, self.v_ext, self.v_h, self.eps_xc, self.v_out,
                               self.theta, self.h, self.xyz, self.Z)

    def relax(self, n_inner):
        """n_inner - 1 steps of Eq. KSLB, then one orthonormalising step."""
        for _ in range(n_inner - 1):
            r = lb.step(self.fstar, self.sigma, self.v_in, self.omega, self.theta, self.dt, self.h)
            self.fstar, self.sigma = r["fstar"], r["sigma"]
        r = lb.step(self.fstar, self.sigma, self.v_in, self.omega, self.theta, self.dt, self.h,
                    orthonormalize=True)
        self.fstar, self.sigma = r["fstar"], r["sigma"]
        self.last_S = r["S"]
        self.steps += n_inner
        return r["psi"]

    def cycle(self, n_inner):
        prev = self.terms["E_total"]
        self.terms = self.evaluate(self.relax(n_inner))
        de = abs(self.terms["E_total"] - prev)
        return de

    def mix(self, alpha):
        self.v_in = alpha * self.v_out + (1.0 - alpha) * self.v_in


def scf(n, h, xyz, Z, n_orb, n_inner=50, e_tol=1e-6, max_cycles=200, mix=0.5,
        theta=0.5, omega=1.0, softening=0.0, poisson_rtol=1e-12, fixed_cycles=None):
    """Run the loop; returns (State, result dict)."""
    st = State(n, h, xyz, Z, n_orb, theta, omega, softening, poisson_rtol)
    history = [st.terms["E_total"]]
    converged = False
    cycles = 0
    de = float("inf")
    limit = fixed_cycles if fixed_cycles is not None else max_cycles
    for c in range(limit):
        de = st.cycle(n_inner)
        cycles += 1
        history.append(st.terms["E_total"])
        if fixed_cycles is None and de < e_tol:
            converged = True
            break
        st.mix(mix)
    res = dict(st.terms)
    res.update({"cycles": cycles, "steps": st.steps, "converged": converged,
                "dE": de, "history": history})
    return st, res
