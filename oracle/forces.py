"""Hellmann-Feynman forces on the nuclei (oracle; test infrastructure only).

Born-Oppenheimer extension of Sec. 3.1 (nuclei fixed while the orbitals relax;
here they are then moved along the forces).  Of the energy terms (kinetic,
electron-nucleus, Hartree, exchange-correlation, nucleus-nucleus) only two
depend on the nuclear positions explicitly:

  E_ext = h^3 sum_r rho(r) V_ext(r),  V_ext(r) = -sum_I Z_I / sqrt(|r - R_I|^2 + a^2)
          (softened nuclei, the same V_ext as the solver),
  E_nn  = sum_{I<J} Z_I Z_J / |R_I - R_J|   (bare Coulomb between nuclei).

With the orbitals at self-consistency the force is minus the explicit
derivative of the total energy (Hellmann-Feynman; the grid basis does not
move with the nuclei, so no basis term appears):

  F_I = Z_I h^3 sum_r rho(r) (r - R_I) / (|r - R_I|^2 + a^2)^(3/2)
        + sum_{J != I} Z_I Z_J (R_I - R_J) / |R_I - R_J|^3.

Parity pinned by the tests against central differences of E_ext (through the
solver's own V_ext routine, scf.external_potential) and of
energy.nuclear_repulsion, and by symmetry.
"""
from __future__ import annotations

import numpy as np

from . import poisson


def electron_nucleus(rho, h, xyz, Z, a):
    """-dE_ext/dR_I at fixed density rho: one row (Fx, Fy, Fz) per nucleus."""
    X, Y, Zc = poisson.coords(rho.shape[::-1], h)
    xyz = np.asarray(xyz, float)
    out = np.zeros((len(Z), 3))
    for I in range(len(Z)):
        dx, dy, dz = X - xyz[I, 0], Y - xyz[I, 1], Zc - xyz[I, 2]
        w = rho * Z[I] / (dx * dx + dy * dy + dz * dz + a * a) ** 1.5
        out[I] = h ** 3 * np.array([(w * dx).sum(), (w * dy).sum(), (w * dz).sum()])
    return out


def nuclear(xyz, Z):
    """-dE_nn/dR_I: one row per nucleus."""
    xyz = np.asarray(xyz, float)
    out = np.zeros((len(Z), 3))
    for I in range(len(Z)):
        for J in range(len(Z)):
            if J != I:
                d = xyz[I] - xyz[J]
                out[I] += Z[I] * Z[J] * d / np.linalg.norm(d) ** 3
    return out


def hf_forces(rho, h, xyz, Z, a):
    """Total Hellmann-Feynman force on each nucleus (Ha/bohr)."""
    return electron_nucleus(rho, h, xyz, Z, a) + nuclear(xyz, Z)
