"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module holds no Cholesky, covariance or precision arithmetic: it only draws
spatial locations, orders them, and draws Gaussian vectors, so that both sides can
be fed the same data.  The geospatial workloads follow Section III-D of the paper
(locations s_1..s_n in R^2, Eq. 1-2); the paper generates its own synthetic
locations, so nothing here stands in for a public dataset.

Random numbers come from numpy's PCG64 generator seeded with the workload seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_points", "morton_order", "gaussian", "line_points",
    "MaternWorkload", "WORKLOADS", "batched_workload",
]


def uniform_points(n: int, seed: int, morton: bool = False) -> np.ndarray:
    """n i.i.d. uniform points in the unit square, shape (n, 2), float64.

    With ``morton=True`` the points are re-ordered along a Z-order (Morton) curve:
    each coordinate is quantised to 16 bits, the bits are interleaved (x in the
    even positions) and the points are sorted stably by that key.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 2))
    if morton:
        pts = pts[morton_order(pts)]
    return np.ascontiguousarray(pts)


def _spread16(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0xFFFF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
    v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
    v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
    v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
    return v


def morton_order(pts: np.ndarray) -> np.ndarray:
    """Permutation sorting 2-D points in [0,1)^2 along a 16-bit-per-axis Z-order curve."""
    q = np.clip(np.floor(pts * 65536.0), 0, 65535).astype(np.uint64)
    key = _spread16(q[:, 0]) | (_spread16(q[:, 1]) << np.uint64(1))
    return np.argsort(key, kind="stable")


def line_points(n: int, seed: int) -> np.ndarray:
    """n sorted uniform points on [0,1] embedded in 2-D as (x, 0): a 1-D transect."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.sort(rng.random(n))
    return np.ascontiguousarray(np.stack([x, np.zeros(n)], axis=1))


def gaussian(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Standard normal matrix of shape (n, nrhs), float64, column-major friendly (C order rows)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, nrhs))


@dataclass(frozen=True)
class MaternWorkload:
    """A synthetic Matern covariance problem: locations, theta = (sigma^2, a, nu), nugget, tile."""
    name: str
    n: int
    tile: int
    nu: float
    range_a: float
    sigma2: float = 1.0
    nugget: float = 1e-6
    seed: int = 1
    morton: bool = True
    mixed: bool = False          # four-precision map (else all FP64)
    eps_high: float = 1e-9
    band: int = 2
    prec_set: int = 4            # 1..4 -> {64}, {64,32}, {64,32,16}, {64,32,16,8}

    def points(self) -> np.ndarray:
        return uniform_points(self.n, self.seed, self.morton)


WORKLOADS = {
    # 2048 unsorted points, exponential kernel, plain FP64, tile 256
    "fp64_n2048": MaternWorkload("fp64_n2048", 2048, 256, 0.5, 0.1, 1.0, 1e-6, 1, morton=False),
    # 65536 Morton-sorted points, exponential kernel, plain FP64, tile 1024 (about 17 GB of lower tiles)
    "fp64_n65536": MaternWorkload("fp64_n65536", 65536, 1024, 0.5, 0.05, 1.0, 1e-6, 2),
    # 131072 Morton-sorted points, nu = 1.5, four precisions, eps_high 1e-9, FP64 band of 2 tiles
    "mxp4_n131072": MaternWorkload("mxp4_n131072", 131072, 2048, 1.5, 0.03, 1.0, 1e-4, 3,
                                   mixed=True, eps_high=1e-9, band=2, prec_set=4),
    # out-of-core shape (the full n = 262144 needs 275 GB of pinned host memory)
    "ooc_n262144": MaternWorkload("ooc_n262144", 262144, 2048, 0.5, 0.02, 1.0, 1e-4, 4),
}

# The paper's accuracy study (Section V): exponential kernel, variance 1, range beta for weak,
# medium and strong spatial correlation, and accuracy levels of the precision map.
THETA_SETS = {"weak": (1.0, 0.02627, 0.5), "medium": (1.0, 0.078809, 0.5), "strong": (1.0, 0.210158, 0.5)}
SWEEP_EPS = (1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11)


@dataclass
class BatchedWorkload:
    """Many independent Matern problems of uneven size (log-uniform n in [64, 4096])."""
    ns: list = field(default_factory=list)
    ranges: list = field(default_factory=list)
    nus: list = field(default_factory=list)
    seeds: list = field(default_factory=list)
    nrhs: int = 16

    def points(self, i: int) -> np.ndarray:
        return uniform_points(self.ns[i], self.seeds[i], morton=True)


def batched_workload(count: int = 512, seed: int = 5, lo: int = 64, hi: int = 4096) -> BatchedWorkload:
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(count)
    ns = [int(round(lo * (hi / lo) ** ui)) for ui in u]
    ranges = list(rng.uniform(0.02, 0.2, count))
    nus = [float(v) for v in rng.choice([0.5, 1.5, 2.5], count)]
    seeds = [int(seed * 100003 + i) for i in range(count)]
    return BatchedWorkload(ns, ranges, nus, seeds)



# Out-of-core workload actually run on a 199 GB host: n = 65536, tile 2048 (17.6 GB of tiles in
# pinned host memory), device cache capped at 0.44 of it (the 120 GB / 275 GB ratio of the
# n = 262144 configuration).
OOC_CACHE_FRACTION = 120.0 / 275.0
