"""Born-Oppenheimer molecular dynamics of the nuclei (oracle; test
infrastructure only).

The nuclei move on the ground-state energy surface of Sec. 3.1 (the orbitals
relaxed to self-consistency at every position) under the Hellmann-Feynman
forces of oracle.forces.  Time integration: velocity Verlet,

  R(t + dt) = R(t) + dt v(t) + dt^2 F(t) / (2 m)
  v(t + dt) = v(t) + dt (F(t) + F(t + dt)) / (2 m),

atomic units (masses in electron masses, dt in hbar/Ha).  Pinned by the
tests against the closed-form harmonic oscillator.
"""
from __future__ import annotations

import numpy as np


def velocity_verlet(force, R0, v0, masses, dt, n_steps):
    """force(R) -> (F, E_pot).  Returns positions [n+1, n_atoms, 3],
    velocities [n+1, n_atoms, 3] and energies [n+1, 2] (E_pot, E_kin)."""
    m = np.asarray(masses, float)[:, None]
    R = np.array(R0, float)
    v = np.array(v0, float)
    F, E = force(R)
    Rs, vs, es = [R.copy()], [v.copy()], [(E, 0.5 * (m * v * v).sum())]
    for _ in range(n_steps):
        R = R + dt * v + 0.5 * dt * dt * F / m
        Fn, E = force(R)
        v = v + 0.5 * dt * (F + Fn) / m
        F = Fn
        Rs.append(R.copy())
        vs.append(v.copy())
        es.append((E, 0.5 * (m * v * v).sum()))
    return np.array(Rs), np.array(vs), np.array(es)
