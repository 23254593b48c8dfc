"""Energies of a set of orthonormal lattice orbitals (oracle; test
infrastructure only).

The paper stops on the change of the orbital energies (Sec. 4) but prints no
formula for them or for the total energy.  Readings taken here:

  * Kinetic operator: the equilibrium stencil K_xi psi(r) = sum_p xi_p
    psi(r - v_p) (zero outside the box) satisfies K_xi = 1 + (theta/2)
    Lap_lattice + O(lap^2), so T_h = (1 - K_xi) / (theta h^2) approximates
    -(1/2) Lap in atomic units.
  * Orbital energies: the Rayleigh-Ritz values of the occupied subspace,
    i.e. the eigenvalues of the N_O x N_O matrix H_jk = <psi_j| T_h + V |psi_k>
    for orthonormal psi (h^3 measure), V the Kohn-Sham potential built from
    the same density.  They do not depend on how a degenerate level's
    orbitals are rotated among themselves; the diagonal H_jj (each orbital's
    own Rayleigh quotient) is reported beside them.
  * Total energy (standard Kohn-Sham expression, doubly occupied orbitals):
      E = 2 sum_j <psi_j|T_h|psi_j> + int V_ext rho + 1/2 int V_H rho
          + int rho eps_xc(rho) + sum_{I<J} Z_I Z_J / |R_I - R_J|
    with integrals as h^3 sums; the nucleus-nucleus term is the bare
    Coulomb one.
"""
from __future__ import annotations

import numpy as np

from . import lattice
from .lb import shifted


def apply_k_xi(psi, theta):
    """K_xi psi for a single grid function psi[z, y, x]."""
    xi = lattice.xi(theta)
    out = np.zeros_like(psi)
    for p, (vx, vy, vz) in enumerate(lattice.VELOCITIES):
        out += xi[p] * shifted(psi, int(vx), int(vy), int(vz))
    return out


def apply_kinetic(psi, theta, h):
    """T_h psi = (psi - K_xi psi) / (theta h^2)."""
    return (psi - apply_k_xi(psi, theta)) / (theta * h * h)


def nuclear_repulsion(xyz, Z):
    e = 0.0
    for i in range(len(Z)):
        for j in range(i):
            e += Z[i] * Z[j] / float(np.linalg.norm(xyz[i] - xyz[j]))
    return e


def energies(psi, rho, v_ext, v_h, eps_xc, v_ks, theta, h, xyz, Z):
    """All energy terms and the orbital eigenvalues.  psi orthonormal."""
    dv = h ** 3
    n = psi.shape[0]
    tpsi = np.array([apply_kinetic(psi[j], theta, h) for j in range(n)])
    hpsi = tpsi + v_ks[None] * psi
    H = np.array([[dv * float((psi[j] * hpsi[k]).sum()) for k in range(n)] for j in range(n)])
    kin = np.array([dv * float((psi[j] * tpsi[j]).sum()) for j in range(n)])
    t_s = 2.0 * kin.sum()
    e_ext = dv * float((v_ext * rho).sum())
    e_h = 0.5 * dv * float((v_h * rho).sum())
    e_xc = dv * float((rho * eps_xc).sum())
    e_nn = nuclear_repulsion(xyz, Z)
    return {
        "T_s": t_s, "E_ext": e_ext, "E_H": e_h, "E_xc": e_xc, "E_nn": e_nn,
        "E_total": t_s + e_ext + e_h + e_xc + e_nn,
        "eigenvalues": np.linalg.eigvalsh(0.5 * (H + H.T)),
        "orbital_energies": np.diag(H).copy(),
        "n_electrons": dv * float(rho.sum()),
    }
