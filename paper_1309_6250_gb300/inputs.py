"""Seeded synthetic inputs: cells, planewave coefficient sets and positions.

This module is shared by the CUDA path, the oracle tests and the benchmark. It holds
the *workload recipe* only (which G vectors exist, which random numbers are drawn,
where the electrons sit) and none of the spline method's arithmetic.

The paper's orbitals are LDA/Troullier-Martins planewave orbitals of Si, Al and MgO
(Sec. III, Gamma point).  Those orbitals are not available, so seeded synthetic
planewave sets with the same shapes stand in for them:

* the G set is every reciprocal-lattice vector with |G|^2/2 <= E_cut (the spherical
  cutoff of Eq. (pw_orbital) and the memory footnote of Sec. III C);
* per orbital, over the half-space of G in lexicographic Miller order,
  x, y ~ N(0,1) and c_G = (x + i y)/sqrt(2) * exp(-|G|^2/d), c_{-G} = conj(c_G),
  c_0 = x (real), so every orbital is real (Gamma point);
* positions are uniform in the cell (crystal coordinates uniform in [0,1)^3).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Cell:
    """One synthetic workload: cubic cell, grid, planewave cutoff and positions."""

    name: str
    a: float                 # cubic lattice constant, bohr
    n_orb: int               # number of real orbitals
    grid: Tuple[int, int, int]
    ecut: float              # Hartree: keep G with |G|^2/2 <= ecut
    decay: float             # c_G envelope exp(-|G|^2/decay)
    n_walkers: int
    n_elec: int
    coef_seed: int
    pos_seed: int

    @property
    def n_pos(self) -> int:
        return self.n_walkers * self.n_elec

    @property
    def lattice(self) -> np.ndarray:
        """3x3 lattice matrix whose COLUMNS are the lattice vectors a_i (bohr)."""
        return np.eye(3) * self.a


# The five workloads.  Cell sizes, cutoffs and decays not fixed by the workload
# statement are proposed readings (documented in the design notes); the shapes
# (orbitals, grid, walkers x electrons) are as stated.
CELLS: Dict[str, Cell] = {
    # 8 real orbitals on 16^3, Ecut 15 Ha, decay 4, 1000 positions.
    "c1": Cell("c1-fp64-interp-16", 10.26, 8, (16, 16, 16), 15.0, 4.0, 1, 1000, 1001, 2001),
    # Si-like 8-atom cubic cell, 16 orbitals on 48^3, 1024 walkers x 32 electrons.
    "c2": Cell("c2-si8-48", 10.26, 16, (48, 48, 48), 15.0, 4.0, 1024, 32, 1002, 2002),
    # MgO-like 64-atom cell, 128 orbitals on 96^3, Ecut 40 Ha, decay 8,
    # 2048 walkers x 256 electrons.
    "c3": Cell("c3-mgo64-96", 15.9, 128, (96, 96, 96), 40.0, 8.0, 2048, 256, 1003, 2003),
    # Uneven multi-cell batch: Al-like 32-atom, Si-like 64-atom, MgO-like 16-atom.
    "c4-al32": Cell("c4-al32-64", 15.3, 48, (64, 64, 64), 15.0, 4.0, 512, 96, 1041, 2041),
    "c4-si64": Cell("c4-si64-80", 20.52, 128, (80, 80, 80), 15.0, 4.0, 1024, 256, 1042, 2042),
    "c4-mgo16": Cell("c4-mgo16-64", 10.02, 32, (64, 64, 64), 40.0, 8.0, 2048, 64, 1043, 2043),
    # Backward workload: Si-like 64-atom cell, 128 orbitals, 72^3, 4096 positions.
    "c5": Cell("c5-si64-72-bwd", 20.52, 128, (72, 72, 72), 15.0, 4.0, 1, 4096, 1005, 2005),
}


def miller_set(lattice: np.ndarray, ecut: float, kpoint=None) -> np.ndarray:
    """All integer Miller triples n with |k + G|^2/2 <= ecut, G = 2*pi*a^{-T} n.

    k = 2*pi*a^{-T} kpoint (kpoint in units of the reciprocal vectors; None = Gamma).
    Returned as an int32 array [n_pw, 3] in lexicographic (n1, n2, n3) order.
    """
    lat = np.asarray(lattice, dtype=np.float64)
    bmat = 2.0 * np.pi * np.linalg.inv(lat).T          # columns: reciprocal vectors
    kf = np.zeros(3) if kpoint is None else np.asarray(kpoint, dtype=np.float64)
    gmax = math.sqrt(2.0 * ecut)
    # |n_i + kf_i| <= gmax * |a_i| / (2 pi) bounds every component.
    nmax = [int(math.floor(gmax * np.linalg.norm(lat[:, i]) / (2.0 * np.pi) + abs(kf[i]))) + 1
            for i in range(3)]
    r = [np.arange(-m, m + 1) for m in nmax]
    n = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    g = (n + kf[None, :]) @ bmat.T
    keep = 0.5 * np.einsum("ij,ij->i", g, g) <= ecut * (1.0 + 1e-14)
    return np.ascontiguousarray(n[keep].astype(np.int32))


def _half_space(n: np.ndarray) -> np.ndarray:
    """Mask of Miller triples lexicographically greater than (0,0,0)."""
    return (n[:, 0] > 0) | ((n[:, 0] == 0) & (n[:, 1] > 0)) | \
           ((n[:, 0] == 0) & (n[:, 1] == 0) & (n[:, 2] > 0))


def pw_coefficients(lattice: np.ndarray, miller: np.ndarray, n_orb: int,
                    decay: float, seed: int) -> np.ndarray:
    """Hermitian-symmetric random coefficients c[n_orb, n_pw] (complex128)."""
    lat = np.asarray(lattice, dtype=np.float64)
    bmat = 2.0 * np.pi * np.linalg.inv(lat).T
    g = miller.astype(np.float64) @ bmat.T
    g2 = np.einsum("ij,ij->i", g, g)
    env = np.exp(-g2 / decay)
    rng = np.random.default_rng(seed)
    half = np.nonzero(_half_space(miller))[0]
    zero = np.nonzero(np.all(miller == 0, axis=1))[0]
    draws = rng.standard_normal((n_orb, half.size, 2))
    c0 = rng.standard_normal(n_orb)
    # index of -G for every G of the half space
    lookup = {tuple(m): i for i, m in enumerate(miller.tolist())}
    neg = np.array([lookup[(-m[0], -m[1], -m[2])] for m in miller[half].tolist()],
                   dtype=np.int64)
    c = np.zeros((n_orb, miller.shape[0]), dtype=np.complex128)
    ch = (draws[..., 0] + 1j * draws[..., 1]) / math.sqrt(2.0) * env[half]
    c[:, half] = ch
    c[:, neg] = np.conj(ch)
    if zero.size:
        c[:, zero[0]] = c0 * env[zero[0]]
    return c


def bloch_coefficients(lattice: np.ndarray, miller: np.ndarray, n_band: int, kpoint,
                       decay: float, seed: int) -> np.ndarray:
    """Coefficients c[n_band, n_pw] (complex128) of Bloch orbitals at k != 0.

    phi_nk(r) = sum_G c_G exp(i (k + G).r) has no Hermitian symmetry: every c_G is drawn
    independently, c_G = (x + i y)/sqrt(2) * exp(-|k + G|^2/d) with x, y ~ N(0,1).
    """
    lat = np.asarray(lattice, dtype=np.float64)
    bmat = 2.0 * np.pi * np.linalg.inv(lat).T
    kf = np.asarray(kpoint, dtype=np.float64)
    g = (miller.astype(np.float64) + kf[None, :]) @ bmat.T
    env = np.exp(-np.einsum("ij,ij->i", g, g) / decay)
    rng = np.random.default_rng(seed)
    draws = rng.standard_normal((n_band, miller.shape[0], 2))
    return (draws[..., 0] + 1j * draws[..., 1]) / math.sqrt(2.0) * env[None, :]


def positions(lattice: np.ndarray, n_pos: int, seed: int,
              lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Cartesian positions [n_pos, 3] with crystal coordinates uniform in [lo, hi)^3."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(lo, hi, size=(n_pos, 3))
    return np.ascontiguousarray(s @ np.asarray(lattice, dtype=np.float64).T)


def upstream_weights(n_pos: int, n_orb: int, seed: int) -> Tuple[np.ndarray, ...]:
    """N(0,1) upstream weights (gv [P,O], gg [P,3,O], gl [P,O]) for the backward pass."""
    rng = np.random.default_rng(seed)
    gv = rng.standard_normal((n_pos, n_orb))
    gg = rng.standard_normal((n_pos, 3, n_orb))
    gl = rng.standard_normal((n_pos, n_orb))
    return gv, gg, gl


@dataclasses.dataclass
class Workload:
    cell: Cell
    lattice: np.ndarray
    miller: np.ndarray       # int32 [n_pw, 3]
    coef: np.ndarray         # complex128 [n_orb, n_pw]
    pos: np.ndarray          # float64 [n_pos, 3]


def make_workload(key: str, n_pos: Optional[int] = None,
                  n_orb: Optional[int] = None) -> Workload:
    """Build the seeded workload of cell `key`, optionally truncated in P or O."""
    cell = CELLS[key]
    lat = cell.lattice
    mil = miller_set(lat, cell.ecut)
    no = cell.n_orb if n_orb is None else n_orb
    coef = pw_coefficients(lat, mil, no, cell.decay, cell.coef_seed)
    npos = cell.n_pos if n_pos is None else n_pos
    pos = positions(lat, npos, cell.pos_seed)
    return Workload(cell, lat, mil, coef, pos)


def random_cell(seed: int, dims: Tuple[int, int, int], n_orb: int, ecut: float,
                decay: float, lattice: Optional[np.ndarray] = None) -> Tuple[np.ndarray, ...]:
    """Small random workload for tests: (lattice, miller, coef)."""
    if lattice is None:
        lattice = np.eye(3) * 6.0
    mil = miller_set(lattice, ecut)
    coef = pw_coefficients(lattice, mil, n_orb, decay, seed)
    return np.asarray(lattice, dtype=np.float64), mil, coef


# k points in units of the reciprocal vectors of the (simple cubic) synthetic cells: the
# zone-boundary points X and R of the cubic Brillouin zone and a point of no symmetry.
# Sec. III reports the same conclusions at several k points, so any of them will do.
KPOINTS: Dict[str, Tuple[float, float, float]] = {
    "gamma": (0.0, 0.0, 0.0),
    "X": (0.5, 0.0, 0.0),
    "R": (0.5, 0.5, 0.5),
    "generic": (0.137, -0.291, 0.412),
}


def random_bloch_cell(seed: int, n_band: int, ecut: float, decay: float, kpoint,
                      lattice: Optional[np.ndarray] = None) -> Tuple[np.ndarray, ...]:
    """Small random k != 0 workload for tests: (lattice, miller, coef)."""
    if lattice is None:
        lattice = np.eye(3) * 6.0
    mil = miller_set(lattice, ecut, kpoint)
    coef = bloch_coefficients(lattice, mil, n_band, kpoint, decay, seed)
    return np.asarray(lattice, dtype=np.float64), mil, coef


def make_bloch_workload(key: str, kpoint, n_pos: Optional[int] = None,
                        n_band: Optional[int] = None) -> Workload:
    """Cell `key` with complex orbitals at `kpoint`: half as many bands as the cell has
    real orbitals (the same table bytes), the same grid, cutoff and positions."""
    cell = CELLS[key]
    lat = cell.lattice
    mil = miller_set(lat, cell.ecut, kpoint)
    nb = cell.n_orb // 2 if n_band is None else n_band
    coef = bloch_coefficients(lat, mil, nb, kpoint, cell.decay, cell.coef_seed + 500)
    npos = cell.n_pos if n_pos is None else n_pos
    pos = positions(lat, npos, cell.pos_seed)
    return Workload(cell, lat, mil, coef, pos)


def graded_knots(n: int, amplitude: float = 0.5, phase: float = 0.0) -> np.ndarray:
    """Non-uniform periodic grid points of one axis in reduced coordinates [0, 1):
    x_l = u + amplitude/(2 pi) (sin(2 pi (u + phase)) - sin(2 pi phase)), u = l/n, strictly
    increasing for |amplitude| < 1 (spacing varies by a factor (1+a)/(1-a) along the axis)."""
    u = np.arange(n) / n
    x = u + amplitude / (2.0 * np.pi) * (np.sin(2.0 * np.pi * (u + phase)) - np.sin(2.0 * np.pi * phase))
    return np.ascontiguousarray(x - np.floor(x))


def all_cells() -> List[str]:
    return list(CELLS.keys())
