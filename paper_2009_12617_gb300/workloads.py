"""Seeded synthetic inputs: water-like charge boxes for the reciprocal-space SPME evaluation.

This module only draws random positions and charges. It holds none of the SPME arithmetic, so both the
CUDA path and the FP64 oracle can be fed from it.

The paper measures a "65536 atom simulation" with a 64^3 grid (Abstract; Sec. V-E) but does not say what
the system is. These generators stand in for it with liquid-water-like boxes: oxygen sites uniform in a
cubic box, two hydrogens at TIP3P-like geometry (r_OH = 0.9572 A, H-O-H angle 104.52 deg) with a uniform
random orientation, charges O -0.834 e and H +0.417 e, and +-1 counter-ion pairs that make the atom count
come out exactly while keeping the box neutral. Density is about 0.1 atoms/A^3 as in liquid water.

Atom-count reading: with t = N // 3, N % 3 == 0 gives t triplets; N % 3 == 2 gives t triplets plus one
+-1 pair; N % 3 == 1 gives t - 1 triplets plus two pairs (so 65536 atoms = 21844 triplets + 2 pairs).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Q_O = -0.834
Q_H = 0.417
R_OH = 0.9572
ANGLE_HOH_DEG = 104.52
DENSITY = 0.1  # atoms / A^3
GRID_CHOICES = (32, 40, 48, 64, 80)
MAX_SPACING = 1.4  # A


@dataclasses.dataclass
class System:
    """One periodic box: positions (N,3) float32 in A, charges (N,) float32 in e, cubic box edge L."""

    pos: np.ndarray
    q: np.ndarray
    box: np.ndarray  # (3,3) float64, rows are the cell vectors a, b, c
    K: tuple
    p: int
    beta: float

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


def composition(n: int) -> tuple[int, int]:
    """(triplets, ion pairs) for an n-atom neutral water-like box."""
    if n < 0:
        raise ValueError("n must be >= 0")
    t = n // 3
    r = n % 3
    if r == 0:
        return t, 0
    if r == 2:
        return t, 1
    if t == 0:
        raise ValueError("n = 1 cannot be made neutral")
    return t - 1, 2


def _random_rotations(rng: np.random.Generator, m: int) -> np.ndarray:
    """m uniform random rotation matrices from uniform unit quaternions (Shoemake's method)."""
    u1, u2, u3 = rng.random((3, m))
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qw = a * np.sin(2 * math.pi * u2)
    qx = a * np.cos(2 * math.pi * u2)
    qy = b * np.sin(2 * math.pi * u3)
    qz = b * np.cos(2 * math.pi * u3)
    R = np.empty((m, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def water_box(n: int, L: float, seed: int, independent: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Positions (n,3) float32 wrapped into [0, L)^3 and charges (n,) float32 of a neutral water-like box.

    independent=True places every atom uniformly and independently (same composition and charges).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t, pairs = composition(n)
    pos = np.empty((n, 3))
    q = np.empty(n)
    if t:
        o = rng.random((t, 3)) * L
        half = math.radians(ANGLE_HOH_DEG) / 2
        local = np.array([[0.0, 0.0, 0.0],
                          [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                          [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])
        rot = _random_rotations(rng, t)
        trip = o[:, None, :] + np.einsum("tij,aj->tai", rot, local)
        pos[: 3 * t] = trip.reshape(-1, 3)
        q[: 3 * t] = np.tile([Q_O, Q_H, Q_H], t)
    if pairs:
        pos[3 * t:] = rng.random((2 * pairs, 3)) * L
        q[3 * t:] = np.tile([1.0, -1.0], pairs)
    if independent:
        pos = rng.random((n, 3)) * L
    pos = np.mod(pos, L)
    pos32 = pos.astype(np.float32)
    pos32[pos32 >= np.float32(L)] = 0.0  # rounding up to L wraps to 0
    return pos32, q.astype(np.float32)


def jitter(pos: np.ndarray, L: float, base_seed: int, step: int, sigma: float = 0.01) -> np.ndarray:
    """One step of the jittered random walk: pos + N(0, sigma) per coordinate, wrapped into the box.

    Step s draws from seed (base_seed, s), so any step can be regenerated on its own given the previous one.
    """
    rng = np.random.Generator(np.random.PCG64([base_seed, step]))
    out = np.mod(pos.astype(np.float64) + rng.normal(0.0, sigma, pos.shape), L).astype(np.float32)
    out[out >= np.float32(L)] = 0.0
    return out


def cubic_box(L: float) -> np.ndarray:
    return np.diag([L, L, L]).astype(np.float64)


# The five workloads. Sizes follow the paper's 64^3 / 65536-atom case (Abstract; Sec. V-E) and grid range
# 32^3..128^3 (Abstract), with beta = 0.34 / A.
def parity_system(seed: int = 1) -> System:
    """2048 atoms (682 triplets + one +-1 pair), cubic 27.4 A, 32^3, p = 4."""
    L = 27.4
    pos, q = water_box(2048, L, seed)
    return System(pos, q, cubic_box(L), (32, 32, 32), 4, 0.34)


def headline_system(seed: int = 2) -> System:
    """65536 atoms, cubic 86.9 A (1.358 A spacing), 64^3, p = 4."""
    L = 86.9
    pos, q = water_box(65536, L, seed)
    return System(pos, q, cubic_box(L), (64, 64, 64), 4, 0.34)


def large_system(seed: int = 3) -> System:
    """262144 atoms, cubic 137.9 A, 128^3, p = 6."""
    L = 137.9
    pos, q = water_box(262144, L, seed)
    return System(pos, q, cubic_box(L), (128, 128, 128), 6, 0.34)


def grid_for_edge(L: float) -> int:
    """Smallest grid edge from {32, 40, 48, 64, 80} with spacing L/K <= 1.4 A (80 if none qualifies)."""
    for K in GRID_CHOICES:
        if L / K <= MAX_SPACING:
            return K
    return GRID_CHOICES[-1]


def batch_sizes(count: int = 64, seed: int = 4, lo: int = 1024, hi: int = 32768) -> list[int]:
    """Atom counts drawn log-uniformly from [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), count)]


def batch_systems(count: int = 64, seed: int = 4, p: int = 4, beta: float = 0.34) -> list[System]:
    """Uneven independent boxes: N log-uniform in [1024, 32768], edge for 0.1 atoms/A^3, K by spacing."""
    out = []
    for i, n in enumerate(batch_sizes(count, seed)):
        L = (n / DENSITY) ** (1.0 / 3.0)
        K = grid_for_edge(L)
        pos, q = water_box(n, L, seed * 100003 + i)
        out.append(System(pos, q, cubic_box(L), (K, K, K), p, beta))
    return out


def rocksalt(a: float = 5.64, cells: int = 2) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """NaCl rock salt: cells^3 conventional cubic cells of edge a, +1 on Na and -1 on Cl sites.

    Returns positions (8*cells^3, 3) float64, charges float64, box (3,3).
    """
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])
    pos, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k], dtype=float)
                for f in fcc:
                    pos.append((o + f) * a)
                    q.append(1.0)
                    pos.append((o + f + np.array([0.5, 0, 0])) * a)
                    q.append(-1.0)
    return np.array(pos), np.array(q), cubic_box(a * cells)
