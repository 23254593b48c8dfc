"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds inputs only: nuclear geometries, grid sizes, seeded random
draws (geometry scans, request arrival streams, random population states for
one-step parity tests).  It contains none of the method's arithmetic -- no
lattice tables, no equilibria, no potentials, no energies -- so that the
oracle and the CUDA path share nothing but the numbers they are fed.

Units are atomic units (bohr, Hartree).  Coordinates are relative to the box
centre; a grid of n sites at spacing h spans [-(n-1)h/2, +(n-1)h/2].

The molecules are the paper's kind of workload (atoms and small molecules
built from nuclear charges, Sec. 4 "Results"): He, CH4, H2O, H2, LiH and a
cluster of water molecules.  No dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

Z_OF = {"H": 1.0, "He": 2.0, "Li": 3.0, "C": 6.0, "O": 8.0}


@dataclasses.dataclass
class Molecule:
    """Nuclei of a closed-shell neutral system."""
    name: str
    symbols: List[str]
    xyz: np.ndarray  # (n_atoms, 3) bohr, relative to box centre

    @property
    def Z(self) -> np.ndarray:
        return np.array([Z_OF[s] for s in self.symbols], dtype=np.float64)

    @property
    def n_electrons(self) -> int:
        return int(round(self.Z.sum()))

    @property
    def n_orb(self) -> int:
        ne = self.n_electrons
        if ne % 2:
            raise ValueError("closed-shell systems only")
        return ne // 2


@dataclasses.dataclass
class Workload:
    """One single-system solve: molecule + grid + relaxation controls."""
    name: str
    molecule: Molecule
    n: Tuple[int, int, int]  # (nx, ny, nz)
    h: float
    n_inner: int = 50
    e_tol: float = 1e-6
    max_cycles: int = 200
    theta: float = 0.5
    omega: float = 1.0
    mix: float = 0.5
    softening: float = 0.0  # <= 0 means a = h

    @property
    def n_orb(self) -> int:
        return self.molecule.n_orb

    @property
    def sites(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def helium() -> Molecule:
    return Molecule("He", ["He"], np.zeros((1, 3)))


def hydrogen_atom() -> Molecule:
    """Not closed shell; used only by single-orbital physics pins."""
    return Molecule("H", ["H"], np.zeros((1, 3)))


def methane(r_ch: float = 2.05) -> Molecule:
    """C at the origin, four H on alternate cube corners (tetrahedral)."""
    d = r_ch / math.sqrt(3.0)
    corners = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    xyz = np.vstack([np.zeros((1, 3)), d * corners])
    return Molecule("CH4", ["C", "H", "H", "H", "H"], xyz)


def water(r_oh: float = 1.81, angle_deg: float = 104.5, r_oh2: float | None = None) -> Molecule:
    """O at the origin, molecule in the xz plane, HOH bisector along +z."""
    r2 = r_oh if r_oh2 is None else r_oh2
    half = math.radians(angle_deg) / 2.0
    h1 = [r_oh * math.sin(half), 0.0, r_oh * math.cos(half)]
    h2 = [-r2 * math.sin(half), 0.0, r2 * math.cos(half)]
    return Molecule("H2O", ["O", "H", "H"], np.array([[0.0, 0.0, 0.0], h1, h2]))


def h2(r: float = 1.4) -> Molecule:
    return Molecule("H2", ["H", "H"], np.array([[0, 0, -r / 2], [0, 0, r / 2]], dtype=np.float64))


def lih(r: float = 3.0) -> Molecule:
    return Molecule("LiH", ["Li", "H"], np.array([[0, 0, -r / 2], [0, 0, r / 2]], dtype=np.float64))


def water_scan(count: int = 64, seed: int = 0) -> List[Molecule]:
    """Seeded water geometries: one O-H length ~ U[1.6, 2.0] bohr shared by both
    bonds, HOH angle ~ U[95, 115] degrees."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(1.6, 2.0, size=count)
    a = rng.uniform(95.0, 115.0, size=count)
    return [water(float(r[i]), float(a[i])) for i in range(count)]


def _rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly random rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def water_cluster(count: int = 8, seed: int = 0, box: float = 51.2, min_oo: float = 5.0,
                  margin: float = 6.0) -> Molecule:
    """`count` waters (r_OH = 1.81 bohr, 104.5 deg) at seeded random positions
    and orientations: O-O distances >= min_oo, every O at least `margin` from
    the faces of a cubic box of edge `box` centred on the origin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    unit = water()
    half = box / 2.0 - margin
    centres = []
    while len(centres) < count:
        c = rng.uniform(-half, half, size=3)
        if all(np.linalg.norm(c - o) >= min_oo for o in centres):
            centres.append(c)
    symbols, xyz = [], []
    for c in centres:
        rot = _rotation(rng)
        for s, p in zip(unit.symbols, unit.xyz):
            symbols.append(s)
            xyz.append(c + rot @ p)
    return Molecule(f"(H2O){count}", symbols, np.array(xyz))


def cluster_256() -> Workload:
    """Eight waters in a 256^3 grid at h = 0.2 bohr, 40 doubly occupied orbitals."""
    return Workload("(H2O)8 256^3 h=0.2", water_cluster(8, 0), (256, 256, 256), 0.2, n_inner=100)


def cluster_sample() -> Workload:
    """The cluster of cluster_256 on a 64^3 grid spanning the same box
    (h = 0.8 bohr): a host-sized sample of its relaxation steps."""
    return Workload("(H2O)8 64^3 h=0.8", water_cluster(8, 0), (64, 64, 64), 0.8, n_inner=100)


def perturb(mol: Molecule, sigma: float, rng: np.random.Generator) -> Molecule:
    return Molecule(mol.name, list(mol.symbols), mol.xyz + rng.normal(0.0, sigma, size=mol.xyz.shape))


# ---------------------------------------------------------------- workloads
def he_24() -> Workload:
    """Helium, 24^3 grid at h = 0.4 bohr, one doubly occupied orbital."""
    return Workload("He 24^3 h=0.4", helium(), (24, 24, 24), 0.4, n_inner=20, e_tol=1e-6)


def ch4_128() -> Workload:
    """Methane single solve, 128^3 grid at h = 0.2 bohr, five orbitals."""
    return Workload("CH4 128^3 h=0.2", methane(), (128, 128, 128), 0.2, n_inner=100, e_tol=1e-6)


def ch4_cd_128() -> Workload:
    """Methane with its C-H bonds stretched to 2.25 bohr (a breathing-mode
    start), 128^3 grid at h = 0.2 bohr: the start of the concurrent dynamics."""
    return Workload("CH4 (r_CH 2.25) 128^3 h=0.2", methane(2.25), (128, 128, 128), 0.2, n_inner=100, e_tol=1e-6)


# nuclear masses in electron masses (1 u = 1822.888 m_e; H 1.008 u, He 4.0026 u, C 12.011 u, O 15.999 u)
MASS_ME = {"H": 1.008 * 1822.888, "He": 4.0026 * 1822.888, "Li": 6.94 * 1822.888, "C": 12.011 * 1822.888,
           "O": 15.999 * 1822.888}


def masses(mol: Molecule) -> np.ndarray:
    return np.array([MASS_ME[s] for s in mol.symbols])


def ch4_small(n: int = 40, h: float = 0.4) -> Workload:
    """Reduced methane case that the oracle finishes in tens of seconds."""
    return Workload(f"CH4 {n}^3 h={h}", methane(), (n, n, n), h, n_inner=40, e_tol=1e-6)


def water_96(mol: Molecule | None = None) -> Workload:
    return Workload("H2O 96^3 h=0.2", mol or water(), (96, 96, 96), 0.2, n_inner=100, e_tol=1e-6)


SERVING_MIX = (
    ("H2", 48), ("He", 48), ("LiH", 64), ("H2O", 96), ("CH4", 128),
)


def serving_stream(n_requests: int, rate_hz: float = 200.0, seed: int = 0):
    """Poisson arrivals of a uniform mix of {H2 48^3, He 48^3, LiH 64^3,
    H2O 96^3, CH4 128^3}, h ~ U[0.2, 0.25], atom jitter N(0, 0.05^2) bohr.
    Returns a list of (arrival_time_s, Workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = {"H2": h2(), "He": helium(), "LiH": lih(), "H2O": water(), "CH4": methane()}
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        kind, n = SERVING_MIX[int(rng.integers(0, len(SERVING_MIX)))]
        h = float(rng.uniform(0.2, 0.25))
        mol = perturb(base[kind], 0.05, rng)
        out.append((t, Workload(f"{kind} {n}^3", mol, (n, n, n), h, n_inner=50)))
    return out


# --------------------------------------------------- random states for unit parity
def random_state(n: Sequence[int], n_orb: int, seed: int, q: int = 19):
    """Seeded random populations f[j][p][z][y][x] (fp64), potential V[z][y][x],
    per-orbital scales and a strictly lower triangular coupling matrix.
    Values are O(1) with a smooth part so that physical magnitudes are mimicked."""
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.uniform(-0.5, 1.0, size=(n_orb, q, nz, ny, nx))
    v = rng.uniform(-3.0, 1.0, size=(nz, ny, nx))
    sigma = rng.uniform(0.5, 2.0, size=n_orb)
    lam = np.tril(rng.uniform(-0.3, 0.3, size=(n_orb, n_orb)), -1)
    u = rng.uniform(-0.2, 0.2, size=(n_orb, nz, ny, nx))
    u[0] = 0.0
    return f, v, sigma, lam, u


# ------------------------------------------------ converged reference solves
def converged_cases():
    """Solves whose oracle fixed points are stored under tests/golden (written
    by tests/golden/make_goldens.py): small grids the oracle converges in
    minutes, a served mix of five molecules, and the 128^3 methane and 96^3
    water (first geometry of the scan) bench workloads."""
    scan0 = water_scan(64, 0)[0]
    return {
        "he_24": Workload("He 24^3 h=0.4", helium(), (24, 24, 24), 0.4, n_inner=20),
        "h2_24": Workload("H2 24^3 h=0.4", h2(), (24, 24, 24), 0.4, n_inner=20),
        "lih_28": Workload("LiH 28x28x32 h=0.35", lih(), (28, 28, 32), 0.35, n_inner=30),
        # at h = 0.35 two of water's occupied levels lie only 0.002 Ha apart, which the
        # time-dependent Gram-Schmidt separates over thousands of cycles; at h = 0.3 they
        # are 0.027 Ha apart
        "h2o_38": Workload("H2O 38^3 h=0.3", water(), (38, 38, 38), 0.3, n_inner=60),
        "ch4_32": Workload("CH4 32^3 h=0.35", methane(), (32, 32, 32), 0.35, n_inner=40),
        "dimer_36": Workload("(H2O)2 36x32x34 h=0.35", water_cluster(2, seed=3, box=11.0, min_oo=5.0, margin=2.5),
                             (36, 32, 34), 0.35, n_inner=40),
        "ch4_128": ch4_128(),
        "h2o_96": water_96(scan0),
    }
