"""Concurrent dynamics of electrons and nuclei, Eq. KSLBCD of Sec. 3
("Concurrent Dynamics") -- oracle; test infrastructure only.

The paper prints the update

    f_jp(r + v_p h; t + h) = f_jp(r - v_p h; t - h) + 2h (U_jp + i V_jp + i W_jp),
    U_jp = kappa w_p q_p E_j phi_j,

a two-step, time-centred scheme on complex populations, and says that it is
the relaxation of Eq. KSLB "augmented" by U, with the electrons and the
nuclei moved together.  It gives no kinetic term (taken literally the
populations would stream freely, coupled only through the sources, and
psi = sum_p f_p would not obey a wave equation), no value or rule for kappa,
and no start.  Readings taken here:

  * Real time from imaginary time.  The scheme is the Wick rotation
    (Sec. 3, first equation) of the ground-state step at omega = 1, where the
    populations carry no memory and every post-collision population is
    xi_p a_j - dt chi_p V phi_j (module ``psi``).  One ground-state step maps
    phi_j to G_j(phi) = sum_p [xi_p a_j - dt chi_p V phi_j](r - v_p); its
    change G_j - phi_j = -dt H phi_j (+ the W source) is the Euler step of
    d phi / d t' = -H phi in imaginary time, with
        H = (1 - K_xi) / dt + K_chi V,   K_w g(r) = sum_p w_p g(r - v_p).
    Time-centred in real time with the paper's step (here tau),
    d phi / d t = -i H phi becomes

        phi_j(t + tau) = phi_j(t - tau) + 2i (tau / dt) [G_j(phi(t)) - phi_j(t)]
                         + 2 tau kappa E_j (K_q phi_j)(t),          K_q = K_{w q}.

    The two-step scheme is stable only while tau |eps| < 1 over the spectrum
    of H, a tighter bound than the ground-state step's 0 < dt eps < 2: at
    theta = 1/2, 1 - K_xi reaches 11/9 at the lattice's shortest waves, so
    tau = dt / 2 is the default (tau |eps| <= 11/18 from the kinetic part).

    The i multiplies the potential source and the W source, as printed, and
    also the kinetic part of the step (streaming and relaxation).  The older
    level enters at the site itself: streaming it over two links, as a
    literal reading of the left-hand side would, adds the real smoothing
    K_xi(2 links) to phi(t - tau), which is dissipative and has no
    Schroedinger limit.
  * W source: a_j = phi_j - sum_{k<j} Lambda_jk phi_k with the complex
    projection coefficient Lambda_jk = <phi_k|phi_j> / <phi_k|phi_k>
    (<a|b> = h^3 sum conj(a) b), evaluated at time t.  It vanishes for
    mutually orthogonal orbitals.
  * U: E_j is the orbital's target energy (given by the caller) and kappa a
    dimensionless constant of the run, 0 by default; 2h U_jp is read as
    2 tau kappa w_p q_p E_j phi_j.
    sum_p w_p q_p = 0 and sum_p w_p q_p v_p = 0, so U adds neither density nor
    momentum; its second moment (3 per unit of phi) changes the kinetic
    energy, which is the control the paper describes.
  * Start: the second level from the first by Taylor expansion to second
    order, phi(tau) = phi + i s D(phi) - s^2 D0(D0(phi)) / 2 + tau kappa E K_q phi,
    s = tau / dt, with D = G - 1 (W source included) and D0 its linear part
    (no W).
  * Nuclei (Ehrenfest form of "electrons and ions moved simultaneously"):
    every n_pot electron steps the nuclei make one velocity-Verlet step of
    n_pot tau under the Hellmann-Feynman forces of the current density
    rho = 2 sum_j |phi_j|^2 (module ``forces``); then V_ext is rebuilt at the
    new positions and V = V_ext + V_H[rho] + v_xc[rho] (no mixing) is used
    by the next n_pot electron steps.

Stationary states: for an eigenvector v of H with real eigenvalue eps, the
levels phi(n tau) = exp(-i Omega n tau) v with sin(Omega tau) = eps tau
solve the two-step update exactly, with constant norm.
"""
from __future__ import annotations

import numpy as np

from . import energy, forces, lattice, lda, poisson, scf
from .lb import shifted


def inner(a, b, h):
    """<a|b> = h^3 sum conj(a) b."""
    return (h ** 3) * complex(np.vdot(a.ravel(), b.ravel()))


def overlap(phi, h):
    """S[k, j] = <phi_k|phi_j>."""
    m = phi.reshape(phi.shape[0], -1)
    return (h ** 3) * (np.conj(m) @ m.T)


def lambda_matrix(S):
    """Lambda_jk = <phi_k|phi_j> / <phi_k|phi_k> for k < j, zero elsewhere."""
    n = S.shape[0]
    lam = np.zeros((n, n), dtype=complex)
    for j in range(n):
        for k in range(j):
            lam[j, k] = S[k, j] / S[k, k].real
    return lam


def pulled(g, w):
    """sum_p w_p g(r - v_p), zero outside the box (one grid function)."""
    out = np.zeros_like(g)
    for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES):
        out += w[p] * shifted(g, int(vx), int(vy), int(vz))
    return out


def u_weights():
    """w_p q_p, the weights of the U source."""
    return lattice.weights() * lattice.hermite2()


def ground_step(phi, V, theta, dt, lam=None):
    """G_j(phi): one omega = 1 ground-state step of every orbital without the
    normalisation; lam (Lambda) None means no W source."""
    xi, chi = lattice.xi(theta), lattice.chi()
    a = phi if lam is None else phi - np.tensordot(lam, phi, axes=(1, 0))
    out = np.empty_like(phi)
    for j in range(phi.shape[0]):
        out[j] = pulled(a[j], xi) - dt * pulled(V * phi[j], chi)
    return out


def increment(phi, V, theta, dt, h, w_source=True):
    """D(phi) = G(phi) - phi, with the W source of phi's own Lambda if asked."""
    lam = lambda_matrix(overlap(phi, h)) if w_source else None
    return ground_step(phi, V, theta, dt, lam) - phi


def u_term(phi, kappa, E, tau):
    """tau kappa E_j K_q phi_j for every orbital (zero when kappa = 0)."""
    out = np.zeros_like(phi)
    if kappa == 0.0:
        return out
    wq = u_weights()
    for j in range(phi.shape[0]):
        out[j] = kappa * tau * E[j] * pulled(phi[j], wq)
    return out


def cd_step(phi_prev, phi, V, theta, dt, h, tau, kappa=0.0, E=None):
    """phi(t + tau) from phi(t - tau) and phi(t) (Eq. KSLBCD as read above);
    dt is the ground-state step theta h^2 that G takes."""
    D = increment(phi, V, theta, dt, h, w_source=True)
    return phi_prev + 2j * (tau / dt) * D + 2.0 * u_term(phi, kappa, E, tau)


def start(phi0, V, theta, dt, h, tau, kappa=0.0, E=None):
    """Second time level from the first (Taylor, second order)."""
    phi0 = np.asarray(phi0, dtype=complex)
    s = tau / dt
    d = increment(phi0, V, theta, dt, h, w_source=True)
    d0 = increment(phi0, V, theta, dt, h, w_source=False)
    dd = ground_step(d0, V, theta, dt, None) - d0
    return phi0 + 1j * s * d - 0.5 * s * s * dd + u_term(phi0, kappa, E, tau)


def density(phi):
    """rho = 2 sum_j |phi_j|^2."""
    return 2.0 * (phi.real ** 2 + phi.imag ** 2).sum(axis=0)


def ks_energy(phi, rho, v_ext, v_h, eps_xc, v_ks, theta, h, xyz, Z):
    """Kohn-Sham energy terms of complex orbitals: T_h is real and symmetric,
    so <phi|T_h|phi> = <Re phi|T_h|Re phi> + <Im phi|T_h|Im phi> and the real
    and imaginary parts enter energy.energies as separate rows."""
    rows = np.concatenate([phi.real, phi.imag], axis=0)
    t = energy.energies(rows, rho, v_ext, v_h, eps_xc, v_ks, theta, h, xyz, Z)
    return {k: t[k] for k in ("T_s", "E_ext", "E_H", "E_xc", "E_nn", "E_total", "n_electrons")}


class Run:
    """Electrons and nuclei moved together (readings above).  Holds the two
    complex levels, the potential in use, the nuclei and their velocities."""

    def __init__(self, phi0, n, h, xyz, Z, theta=0.5, softening=0.0, kappa=0.0, E=None,
                 masses=None, velocities=None, poisson_rtol=1e-12, v_h=None, tau=None):
        self.n, self.h, self.theta = tuple(n), float(h), float(theta)
        self.dt = lattice.time_step(theta, 1.0, h)
        self.tau = 0.5 * self.dt if tau is None else float(tau)
        self.a = softening if softening > 0 else h
        self.xyz, self.Z = np.array(xyz, float), np.asarray(Z, float)
        self.kappa = float(kappa)
        self.E = None if E is None else np.asarray(E, float)
        self.masses = None if masses is None else np.asarray(masses, float)
        self.vel = np.zeros_like(self.xyz) if velocities is None else np.array(velocities, float)
        self.poisson_rtol = poisson_rtol
        self.v_h = v_h
        self.steps = 0
        phi0 = np.asarray(phi0, dtype=complex)
        self.rebuild(phi0)
        self.F = forces.hf_forces(self.rho, self.h, self.xyz, self.Z, self.a)
        self.prev = phi0
        self.cur = start(phi0, self.V, self.theta, self.dt, self.h, self.tau, self.kappa, self.E)
        self.steps = 1

    def rebuild(self, phi):
        """Density of phi, then V = V_ext(R) + V_H + v_xc (no mixing)."""
        self.rho = density(phi)
        self.v_ext = scf.external_potential(self.n, self.h, self.xyz, self.Z, self.a)
        self.v_h, _, _ = poisson.hartree(self.rho, self.h, self.v_h, self.poisson_rtol)
        self.eps_xc, v_xc = lda.lda_xc(self.rho)
        self.V = self.v_ext + self.v_h + v_xc

    def electron_steps(self, k):
        for _ in range(k):
            nxt = cd_step(self.prev, self.cur, self.V, self.theta, self.dt, self.h, self.tau, self.kappa, self.E)
            self.prev, self.cur = self.cur, nxt
            self.steps += 1

    def block(self, n_pot):
        """n_pot electron steps at fixed V, then the nuclei's velocity-Verlet
        step of n_pot tau (skipped without masses) and the potential rebuilt
        from the current level."""
        self.electron_steps(n_pot)
        tau = n_pot * self.tau
        moving = self.masses is not None
        if moving:
            m = self.masses[:, None]
            self.xyz = self.xyz + tau * self.vel + 0.5 * tau * tau * self.F / m
        self.rebuild(self.cur)
        Fn = forces.hf_forces(self.rho, self.h, self.xyz, self.Z, self.a)
        if moving:
            self.vel = self.vel + 0.5 * tau * (self.F + Fn) / self.masses[:, None]
        self.F = Fn

    def energies(self):
        """Kohn-Sham terms of the current level at the current nuclei, and the
        nuclei's kinetic energy."""
        t = ks_energy(self.cur, self.rho, self.v_ext, self.v_h, self.eps_xc, self.V, self.theta, self.h,
                      self.xyz, self.Z)
        m = np.zeros(len(self.Z)) if self.masses is None else self.masses
        t["E_kin_nuclei"] = 0.5 * float((m[:, None] * self.vel ** 2).sum())
        return t
