"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method itself: it only draws input data
(arrays, sizes, trip counts, sparse patterns) from a counter-based generator and
writes them to files or returns numpy arrays.  Both sides of a parity test read
the same bytes, so neither re-implements the other's input path.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), in its counter form: draw k of stream `seed`
is mix(seed * GOLDEN + (k + 1) * GOLDEN), where mix is the 64-bit finaliser
(xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).  Uniform
doubles take the top 53 bits: u = (z >> 11) * 2^-53 in [0, 1); the [-1, 1)
map 2u - 1 is exact in binary64.

Log-uniform integers use an integer-only method: draw an octave e uniformly
from the octaves covering [lo, hi], then a uniform integer in [2^e, 2^(e+1)),
clipped to [lo, hi].  This is log-uniform per octave (a stated deviation from a
continuous log-uniform law) and involves no libm call, so every language that
re-implements it gets the same integers.
"""
from __future__ import annotations

import os
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of stream `seed` as uint64."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(base + k * GOLDEN)


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    u = splitmix64(seed, n, offset) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    return 2.0 * uniform01(seed, n, offset) - 1.0


def uniform_int(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] by the multiply-shift (Lemire) map of the top 32 bits."""
    span = np.uint64(hi - lo + 1)
    u = splitmix64(seed, n, offset) >> np.uint64(32)
    return (np.int64(lo) + ((u * span) >> np.uint64(32)).astype(np.int64))


def loguniform_int(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Per-octave log-uniform integers in [lo, hi] (module docstring)."""
    elo = int(lo).bit_length() - 1
    ehi = int(hi).bit_length() - 1
    e = uniform_int(seed, n, elo, ehi, offset=0)
    m = splitmix64(seed, n, offset=n) >> np.uint64(11)       # 53 random bits
    width = np.left_shift(np.int64(1), e)                      # 2^e
    v = width + (m.astype(np.uint64) % width.astype(np.uint64)).astype(np.int64)
    return np.clip(v, lo, hi)


# ---------------------------------------------------------------- workloads

def axpy_inputs(n: int, seed: int = 1):
    """x, y ~ U[-1, 1): FP64 arrays of n elements (two disjoint draws of one stream)."""
    return uniform_pm1(seed, n, 0), uniform_pm1(seed, n, n)


def axpy_closed_form_inputs(n: int):
    """x[i] = i, y[i] = 1: every partial sum of y_new is exact in binary64."""
    return np.arange(n, dtype=np.float64), np.ones(n, dtype=np.float64)


def jacobi_input(n: int, seed: int = 2) -> np.ndarray:
    """n^3 FP64 grid, index (k, j, i) with i fastest; interior ~ U[0, 1), boundary 0."""
    g = uniform01(seed, n * n * n).reshape(n, n, n)
    g[0, :, :] = 0.0
    g[-1, :, :] = 0.0
    g[:, 0, :] = 0.0
    g[:, -1, :] = 0.0
    g[:, :, 0] = 0.0
    g[:, :, -1] = 0.0
    return np.ascontiguousarray(g.reshape(-1))


def write_f64(path: str, a: np.ndarray) -> None:
    np.ascontiguousarray(a, dtype=np.float64).tofile(path)


def write_raw(path: str, a: np.ndarray) -> None:
    np.ascontiguousarray(a).tofile(path)


def ensure_dir(path: str) -> str:
    os.makedirs(path, exist_ok=True)
    return path
