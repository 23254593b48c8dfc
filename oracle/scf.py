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
         orthonormal orbitals of that step; stop by the rule below;
         otherwise V <- mix V_out + (1 - mix) V.

Stop rule (a reading: the paper stops once the orbital energies no longer
change, Sec. 4, without a threshold or a bound).  A change between two
cycles does not bound the distance to the fixed point when a cycle contracts
the error slowly: the time-dependent Gram-Schmidt of Eq. KSLB separates two
occupied orbitals at the rate of their eigenvalue ratio, and the part of the
orthogonalisation source that the potential term does not carry leaks that
slow rotation into the occupied span, hence into the density.  Cycles are
grouped in blocks of STOP_BLOCK; at the end of each block three changes since
the previous block end are watched -- the total energy, the eigenvalues
(largest change) and the density (relative L2 change) -- and for each the
last block change D_m is extended by its geometric tail D_m r / (1 - r), r
the larger of the last two ratios D_m / D_{m-1}, D_{m-1} / D_{m-2}, capped at
Q_CAP (a sequence that does not contract counts as contracting at Q_CAP).
The loop stops once, for every quantity with a positive tolerance, both D_m
and that tail are within the tolerance, or D_m is below the rounding floor
FLOOR_ULPS u s (u the unit roundoff of the orbital values, 2^-53 here; s =
|E|, max_j |eps_j| and 1 for the three quantities); at least three blocks
run.  Blocks let a slow drift stand out of the rounding noise of
single-precision orbitals, which does not grow with the block length.
"""
from __future__ import annotations

import math

import numpy as np

from . import energy, lattice, lb, lda, poisson
from . import psi as psi_form


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


STOP_BLOCK = 4
Q_CAP = 0.92  # per block of four cycles: 0.98 per cycle
FLOOR_ULPS = 8.0
UNIT_ROUNDOFF = 2.0 ** -53


def _ratio(a, b):
    if b > 0.0:
        return a / b
    return math.inf if a > 0.0 else 0.0


def tail_estimate(d0, d1, d2):
    """Geometric tail d0 q / (1 - q) of the changes d0 (last), d1, d2: q is the
    larger of d0/d1 and d1/d2, capped at Q_CAP."""
    q = min(max(_ratio(d0, d1), _ratio(d1, d2)), Q_CAP)
    return d0 * q / (1.0 - q)


def settled(changes, tol, scale=1.0):
    """changes: the per-cycle changes of one quantity, oldest first.  True when
    the last change and its tail are both within tol, or the last change is
    below the rounding floor FLOOR_ULPS u scale (tol <= 0: not watched)."""
    if tol <= 0.0:
        return True
    if len(changes) < 3:
        return False
    d0, d1, d2 = changes[-1], changes[-2], changes[-3]
    if d0 <= FLOOR_ULPS * UNIT_ROUNDOFF * scale:
        return True
    return d0 <= tol and tail_estimate(d0, d1, d2) <= tol


def splitmix64(state):
    """SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014): returns (next state, 64-bit output)."""
    M = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & M
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return state, z ^ (z >> 31)


def start_offsets(n_orb, seed=0):
    """Offsets (bohr) of the Gaussian centres from their nuclei.
    seed 0: 0.25 (sin(1 + 2.1 j), sin(2 + 3.3 j), sin(3 + 4.7 j)).
    seed != 0: 0.25 (2 u - 1) per component, u = top 53 bits of successive
    SplitMix64 outputs from state = seed, drawn x, y, z for j = 0, 1, ..."""
    out = np.empty((n_orb, 3))
    if seed == 0:
        for j in range(n_orb):
            out[j] = 0.25 * np.array([math.sin(1.0 + 2.1 * j), math.sin(2.0 + 3.3 * j), math.sin(3.0 + 4.7 * j)])
        return out
    state = seed & ((1 << 64) - 1)
    for j in range(n_orb):
        for k in range(3):
            state, z = splitmix64(state)
            out[j, k] = 0.25 * (2.0 * ((z >> 11) * 2.0 ** -53) - 1.0)
    return out


def initial_orbitals(n, h, xyz, Z, n_orb, seed=0):
    """Gaussian initial orbitals (a reading of 'Gaussian initial orbital').

    Nuclei are ordered by decreasing charge (stable).  Orbital j sits on
    nucleus I = order[j mod n_atoms], shell m = j div n_atoms:
        c_j = R_I + o_j   (o_j from start_offsets(n_orb, seed))
        s_j = 1.2 (1 + 0.35 m)
        psi0_j(r) = exp(-|r - c_j|^2 / (2 s_j^2))
    The small offsets break the molecule's point symmetry so that every
    symmetry component is present in every start vector."""
    X, Y, Zc = grid_coords(n, h)
    order = sorted(range(len(Z)), key=lambda i: -Z[i])
    off = start_offsets(n_orb, seed)
    out = np.empty((n_orb,) + X.shape)
    for j in range(n_orb):
        I = order[j % len(Z)]
        m = j // len(Z)
        c = xyz[I] + off[j]
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
                 poisson_rtol=1e-12, seed=0, storage="populations"):
        self.n, self.h = tuple(n), float(h)
        self.xyz, self.Z = np.asarray(xyz, float), np.asarray(Z, float)
        self.n_orb = n_orb
        self.theta, self.omega = float(theta), float(omega)
        self.dt = lattice.time_step(theta, omega, h)
        self.a = softening if softening > 0 else h
        self.poisson_rtol = poisson_rtol
        self.v_ext = external_potential(self.n, h, self.xyz, self.Z, self.a)
        psi = lb.orthonormalize(initial_orbitals(self.n, h, self.xyz, self.Z, n_orb, seed), h)
        # storage "psi" (omega = 1 only): the same steps in orbital storage (module psi)
        if storage not in ("populations", "psi") or (storage == "psi" and self.omega != 1.0):
            raise ValueError("orbital storage needs omega = 1")
        self.storage = storage
        if storage == "psi":
            self.pstate = psi_form.PsiState(psi.copy())
        else:
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
        if self.storage == "psi":
            for t in range(n_inner):
                r = psi_form.step(self.pstate, self.sigma, self.v_in, self.theta, self.dt, self.h,
                                  orthonormalize=(t == n_inner - 1))
                self.sigma = r["sigma"]
            self.last_S = r["S"]
            self.steps += n_inner
            return r["psi"]
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
        theta=0.5, omega=1.0, softening=0.0, poisson_rtol=1e-12, fixed_cycles=None,
        eig_tol=2e-6, rho_tol=2e-6, seed=0, state=None, storage="populations"):
    """Run the loop (stop rule in the module docstring); returns (State,
    result dict).  state: continue an existing State instead of starting.
    storage "psi": the orbital-storage form of the steps (omega = 1)."""
    st = state if state is not None else State(n, h, xyz, Z, n_orb, theta, omega, softening, poisson_rtol, seed,
                                               storage)
    history = [st.terms["E_total"]]
    d_e, d_eig, d_rho = [], [], []  # block changes
    ref_E, ref_eig, ref_rho = st.terms["E_total"], st.terms["eigenvalues"].copy(), st.rho.copy()
    converged = False
    cycles = 0
    de = math.inf
    limit = fixed_cycles if fixed_cycles is not None else max_cycles
    for c in range(limit):
        de = st.cycle(n_inner)
        cycles += 1
        history.append(st.terms["E_total"])
        if cycles % STOP_BLOCK == 0:
            E, eig = st.terms["E_total"], st.terms["eigenvalues"]
            d_e.append(abs(E - ref_E))
            d_eig.append(float(np.abs(eig - ref_eig).max()))
            d_rho.append(float(np.linalg.norm(st.rho - ref_rho) / np.linalg.norm(st.rho)))
            ref_E, ref_eig, ref_rho = E, eig.copy(), st.rho.copy()
            if (fixed_cycles is None and settled(d_e, e_tol, abs(E))
                    and settled(d_eig, eig_tol, float(np.abs(eig).max())) and settled(d_rho, rho_tol)):
                converged = True
                break
        st.mix(mix)
    tails = [tail_estimate(*d[-1:-4:-1]) if len(d) >= 3 else math.inf for d in (d_e, d_eig, d_rho)]
    res = dict(st.terms)
    res.update({"cycles": cycles, "steps": st.steps, "converged": converged,
                "dE": de, "d_eig": d_eig[-1] if d_eig else math.inf,
                "d_rho": d_rho[-1] if d_rho else math.inf, "err_E": tails[0], "err_eig": tails[1],
                "err_rho": tails[2], "history": history})
    return st, res
