"""D3Q19 lattice of the oracle (test infrastructure only).

The paper does not name its velocity set; it needs a set whose weights make
the source term's first and second moments vanish (Sec. 3, definition of
chi_p) and whose equilibrium carries an adjustable second moment.  D3Q19 --
rest, 6 axis and 12 face-diagonal velocities with weights 1/3, 1/18, 1/36
and sound speed c_s^2 = 1/3 -- is the smallest standard set with that
isotropy.

Velocity order (shared with the C ABI as a data layout, not as code):
    0: ( 0, 0, 0)
    1: (+1, 0, 0)   2: (-1, 0, 0)   3: ( 0,+1, 0)   4: ( 0,-1, 0)
    5: ( 0, 0,+1)   6: ( 0, 0,-1)
    7: (+1,+1, 0)   8: (-1,-1, 0)   9: (+1,-1, 0)  10: (-1,+1, 0)
   11: (+1, 0,+1)  12: (-1, 0,-1)  13: (+1, 0,-1)  14: (-1, 0,+1)
   15: ( 0,+1,+1)  16: ( 0,-1,-1)  17: ( 0,+1,-1)  18: ( 0,-1,+1)
"""
import numpy as np

Q = 19
CS2 = 1.0 / 3.0

VELOCITIES = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
], dtype=np.int64)


def weights() -> np.ndarray:
    """Lattice weights w_p, normalised to one (Sec. 3, 'lattice weights
    normalised to unity')."""
    v2 = (VELOCITIES ** 2).sum(axis=1)
    return np.where(v2 == 0, 1.0 / 3.0, np.where(v2 == 1, 1.0 / 18.0, 1.0 / 36.0))


def hermite2() -> np.ndarray:
    """Second-order lattice Hermite polynomial q_p = (v_p^2 - 3 c_s^2)/(2 c_s^4)
    (Sec. 3, definition of the equilibrium)."""
    v2 = (VELOCITIES ** 2).sum(axis=1).astype(np.float64)
    return (v2 - 3.0 * CS2) / (2.0 * CS2 * CS2)


def xi(theta: float) -> np.ndarray:
    """Equilibrium weights xi_p = w_p (1 + (theta - c_s^2) q_p), f^e_p = xi_p psi.

    Sec. 3 prints xi_p = (1 + (D - c_s^2) q_p) and then speaks of w_p; the
    factor w_p is read as lost from the printed formula (without it sum_p xi_p
    is not 1 and the collision does not conserve psi).  The coefficient in
    front of q_p is the equilibrium's second moment, called theta here:
    sum_p xi_p v_p v_p = theta I.
    """
    return weights() * (1.0 + (theta - CS2) * hermite2())


def chi() -> np.ndarray:
    """Source weights chi_p = w_p [1 - (v_p^2 - 3 c_s^2)/(2 c_s^2)]
    (Sec. 3, definition of V_p).  With D3Q19 this is {5/6, 1/18, -1/72}."""
    v2 = (VELOCITIES ** 2).sum(axis=1).astype(np.float64)
    return weights() * (1.0 - (v2 - 3.0 * CS2) / (2.0 * CS2))


def time_step(theta: float, omega: float, h: float) -> float:
    """Imaginary-time step delta_t of one lattice update.

    Sec. 3 relates the relaxation frequency to the diffusivity,
    D = c_s^2 (1/omega - 1/2) in lattice units; with an equilibrium of second
    moment theta the diffusivity is theta (1/omega - 1/2).  The Wick-rotated
    Schroedinger equation (Sec. 3, first equation) has diffusivity hbar/2m,
    i.e. 1/2 in atomic units, which on a lattice of spacing h with step
    delta_t is delta_t / (2 h^2) in lattice units.  Equating the two:
        delta_t = 2 h^2 theta (1/omega - 1/2) = theta h^2 (2 - omega) / omega.
    """
    return theta * h * h * (2.0 - omega) / omega
