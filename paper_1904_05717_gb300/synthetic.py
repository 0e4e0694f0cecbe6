"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

Holds no arithmetic of the method: only a counter-based random generator and
the value distributions of the workloads (uniform[-1,1] matrices, standard
normal matrices, the wide-exponent family (u - 0.5) * exp(phi * g), and
log-uniform problem sizes for the batched workload).

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based hash: the value at
counter c is mix64(seed + (c + 1) * 0x9E3779B97F4A7C15).  Element (i, j) of an
m x n matrix uses counter i + j*m, so the matrix does not depend on the leading
dimension it is stored with.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 0x4D4F4D4D  # workload seed = SEED_BASE + 1000 * workload_index + matrix_id

MATRIX_ID = {"A": 0, "B": 1, "C": 2, "dC": 3, "G": 4}


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw_u64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    c = np.arange(offset, offset + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN
    return mix64(z)


def unit_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each 64-bit word times 2^-53."""
    return (raw_u64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    return 2.0 * unit_uniform(seed, count, offset) - 1.0


def standard_normal(seed: int, count: int) -> np.ndarray:
    """Box-Muller on pairs of counters (2c, 2c+1)."""
    u = raw_u64(seed, 2 * count)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = (u[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _place(vals: np.ndarray, m: int, n: int, ld: int | None) -> np.ndarray:
    """Column-major m x n matrix (Fortran order) with leading dimension ld >= m.

    With ld > m the result is a view into an (ld x n) buffer whose padding rows
    hold NaN, so any read of the padding shows up in the result."""
    vals = vals.reshape(n, m).T  # counter i + j*m -> element (i, j)
    if ld is None or ld == m:
        return np.asfortranarray(vals)
    if ld < m:
        raise ValueError("ld < m")
    buf = np.full((ld, n), np.nan, dtype=np.float64, order="F")
    buf[:m, :] = vals
    return buf[:m, :]


def matrix(kind: str, m: int, n: int, seed: int, ld: int | None = None, phi: float = 0.0) -> np.ndarray:
    """A seeded m x n float64 column-major matrix.

    kind: 'uniform'  i.i.d. uniform[-1, 1]
          'normal'   i.i.d. N(0, 1)
          'phi'      (u - 0.5) * exp(phi * g), u ~ U[0,1), g ~ N(0,1)  (wide exponent range)
          'int'      integers uniform in [-8, 8]
    """
    cnt = m * n
    if kind == "uniform":
        v = uniform_pm1(seed, cnt)
    elif kind == "normal":
        v = standard_normal(seed, cnt)
    elif kind == "phi":
        u = unit_uniform(seed, cnt)
        g = standard_normal(seed ^ 0x5DEECE66D, cnt)
        v = (u - 0.5) * np.exp(phi * g)
    elif kind == "int":
        v = np.floor(unit_uniform(seed, cnt) * 17.0) - 8.0
    else:
        raise ValueError(kind)
    return _place(v, m, n, ld)


def workload_seed(workload_index: int, matrix_name: str) -> int:
    return SEED_BASE + 1000 * workload_index + MATRIX_ID[matrix_name]


def log_uniform_sizes(seed: int, count: int, lo: int = 32, hi: int = 2048) -> np.ndarray:
    """count x 3 integer (m, n, k) triples, each log-uniform in [lo, hi]."""
    u = unit_uniform(seed, 3 * count).reshape(count, 3)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)
