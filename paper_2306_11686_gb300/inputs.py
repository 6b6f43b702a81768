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


def loops_inputs(n: int = 256, seed: int = 3, lo: int = 1 << 10, hi: int = 1 << 22):
    """n independent axpy loops: trip counts log-uniform per octave in [lo, hi],
    coefficients a_k ~ U[-1,1), slices packed back to back in x, y, z.
    Returns (trips int64[n], a float64[n], off int64[n], x, y) with x, y ~ U[-1,1)."""
    trips = loguniform_int(seed, n, lo, hi).astype(np.int64)
    a = uniform_pm1(seed + 1000, n)
    off = np.zeros(n, dtype=np.int64)
    off[1:] = np.cumsum(trips)[:-1]
    total = int(trips.sum())
    x = uniform_pm1(seed + 2000, total)
    y = uniform_pm1(seed + 3000, total)
    return trips, a, off, x, y


def serve_program_inputs(p: int, n: int = 1 << 20, nnz_row: int = 16, passes: int = 10, req_per_pass: int = 64,
                         seed_base: int = 5):
    """Program p of the serving workload: CSR matrix with n rows, nnz_row
    nonzeros per row at uniform random columns, values and x0 ~ U[-1,1)
    (stream seed_base + p), and libc requests at Poisson row positions
    (geometric gaps with mean n / req_per_pass) in every pass, kinds uniform
    over {fwrite, printf, clock, getenv}, fwrite sizes per-octave log-uniform
    in [64 B, 1 MiB].  Returns (rowptr, col, val, x0, req) with req an int64
    array of pairs (pass << 32 | row, kind | size << 8) sorted by key."""
    seed = seed_base + p
    nnz = n * nnz_row
    rowptr = np.arange(0, nnz + 1, nnz_row, dtype=np.int64)
    col = uniform_int(seed, nnz, 0, n - 1).astype(np.int32)
    val = uniform_pm1(seed + 100, nnz)
    x0 = uniform_pm1(seed + 200, n)
    keys, types = [], []
    for r in range(passes):
        u = uniform01(seed * 1000 + r, 4 * req_per_pass + 16)
        q = req_per_pass / n                                     # success probability per row
        gaps = 1 + np.floor(np.log1p(-u) / np.log1p(-q)).astype(np.int64)
        rows = np.cumsum(gaps) - 1
        rows = rows[rows < n]
        kind = uniform_int(seed * 1000 + r + 500, len(rows), 0, 3)
        size = loguniform_int(seed * 1000 + r + 700, len(rows), 64, 1 << 20)
        keys.append((np.int64(r) << 32) | rows)
        types.append(kind.astype(np.int64) | (size.astype(np.int64) << 8))
    key = np.concatenate(keys) if keys else np.zeros(0, dtype=np.int64)
    typ = np.concatenate(types) if types else np.zeros(0, dtype=np.int64)
    req = np.empty(2 * len(key), dtype=np.int64)
    req[0::2], req[1::2] = key, typ
    return rowptr, col, val, x0, req


def write_f64(path: str, a: np.ndarray) -> None:
    np.ascontiguousarray(a, dtype=np.float64).tofile(path)


def write_raw(path: str, a: np.ndarray) -> None:
    np.ascontiguousarray(a).tofile(path)


def ensure_dir(path: str) -> str:
    os.makedirs(path, exist_ok=True)
    return path
