"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds the workload definitions (mesh sizes, polynomial orders,
seeds) and the counter-based random generator that draws the right-hand
sides.  It contains none of the spectral-element arithmetic: no quadrature,
no operator, no gather-scatter.  Both sides of every parity test receive the
arrays produced here and nothing else in common.

Random numbers are drawn with SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based generator: the value for (seed, index) is one SplitMix64 output
step applied to the state ``seed * GOLDEN + index``.  A 53-bit mantissa is
taken from the top bits, giving a double in [0, 1) that is mapped to [-1, 1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state: np.ndarray) -> np.ndarray:
    """One SplitMix64 output step for every uint64 entry of ``state``."""
    with np.errstate(over="ignore"):
        z = state.astype(np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1): entry ``i`` depends only on (seed, offset + i)."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed) * GOLDEN
        idx = np.arange(offset, offset + n, dtype=np.uint64)
        z = splitmix64(base + idx)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def draw_u64(seed: int, n: int, stream: int) -> np.ndarray:
    """Raw 64-bit draws for integer choices (``stream`` separates uses)."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed) * GOLDEN + np.uint64(stream) * np.uint64(0xD1B54A32D192ED03)
        return splitmix64(base + np.arange(n, dtype=np.uint64))


@dataclasses.dataclass(frozen=True)
class Box:
    """A box of nx*ny*nz hexahedral elements of order N on the unit cube.

    ``deform`` is the amplitude of the smooth sinusoidal node displacement as
    a fraction of the smallest element width h = 1/max(nx, ny, nz)."""

    nx: int
    ny: int
    nz: int
    N: int
    deform: float = 0.0

    @property
    def E(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return self.N + 1

    @property
    def n_local(self) -> int:
        return self.E * self.n ** 3

    @property
    def n_global(self) -> int:
        return (self.nx * self.N + 1) * (self.ny * self.N + 1) * (self.nz * self.N + 1)


def rhs_global(box: Box, seed: int) -> np.ndarray:
    """Nodal right-hand side: i.i.d. U[-1, 1) per unique (global) node."""
    return uniform_pm1(seed, box.n_global)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow the problem statement of the method's
# Nekbone case study: a Poisson problem on box meshes of hexahedra.
# ---------------------------------------------------------------------------

#: plain FP64 Jacobi-PCG, 2x2x2 affine box, N=7, seed 0
SMALL_FP64 = Box(2, 2, 2, 7, 0.0)
#: mixed precision workload, 16^3 deformed box, N=9, seed 0
MIXED_16CUBE_N9 = Box(16, 16, 16, 9, 0.05)
#: learned-preconditioner workload, 16^3 deformed box, N=7
LEARNED_16CUBE_N7 = Box(16, 16, 16, 7, 0.05)
#: roofline sweep grid: E from 8^3=512 to 32^3=32768 at these orders
SWEEP_ORDERS = (5, 7, 9, 11, 15)
SWEEP_EDGES = (8, 16, 24, 32)


def sweep_boxes():
    """Deformed cubes of the roofline sweep (E = 512 ... 32768)."""
    return [Box(m, m, m, N, 0.05) for m in SWEEP_EDGES for N in SWEEP_ORDERS]


def most_cubic_factorisation(E: int) -> tuple[int, int, int]:
    """nx*ny*nz = E minimising max/min, ties broken lexicographically."""
    best = None
    for nx in range(1, E + 1):
        if E % nx:
            continue
        rest = E // nx
        for ny in range(1, rest + 1):
            if rest % ny:
                continue
            nz = rest // ny
            t = (nx, ny, nz)
            key = (max(t) / min(t), t)
            if best is None or key < best[0]:
                best = (key, t)
    return best[1]


BATCH_ORDERS = (5, 7, 9, 11)


def batched_problems(count: int = 256, deform: float = 0.05):
    """Independent problems of the batched workload: problem p draws its
    element count E ~ U{8..512} and order N ~ U{5,7,9,11} from seed p; its
    right-hand side uses seed p too."""
    out = []
    for p in range(count):
        d = draw_u64(p, 2, stream=7)
        E = 8 + int(d[0] % np.uint64(505))
        N = BATCH_ORDERS[int(d[1] % np.uint64(4))]
        nx, ny, nz = most_cubic_factorisation(E)
        out.append((Box(nx, ny, nz, N, deform), p))
    return out


TRAIN_SEEDS = tuple(range(1000, 1008))
HELDOUT_SEEDS = tuple(range(2000, 2004))


def l2_flush_bytes() -> int:
    """Size of the buffer written between timed repetitions (> 129 MB L2)."""
    return 512 * 1024 * 1024


def describe(box: Box) -> str:
    return (f"box {box.nx}x{box.ny}x{box.nz} (E={box.E}) N={box.N} "
            f"deform={box.deform}h n_local={box.n_local} n_global={box.n_global}")


__all__ = [
    "Box", "rhs_global", "uniform_pm1", "draw_u64", "splitmix64",
    "SMALL_FP64", "MIXED_16CUBE_N9", "LEARNED_16CUBE_N7", "SWEEP_ORDERS",
    "SWEEP_EDGES", "sweep_boxes", "batched_problems", "most_cubic_factorisation",
    "TRAIN_SEEDS", "HELDOUT_SEEDS", "l2_flush_bytes", "describe",
]
