"""Seeded synthetic point clouds for the k-d tree build.

This module only draws numbers: it holds none of the tree-building
arithmetic, so both the CPU oracle's tests and the GPU path may use it.
Every stream is a splitmix64 sequence (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the i-th output
of stream ``seed`` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15) with the
standard 64-bit finaliser.  Independent streams for one workload are made
by hashing (seed, purpose) into a new seed.

The paper measures only "randomly-generated" integer tuples (Section 2.3,
Section 3.2, Appendix "Performance Measurements"); the workloads here follow
that and add the float, mixture, duplicate and batched shapes the build is
exercised on.  Each recipe is written out in its docstring.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` consecutive outputs of the splitmix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN)


def substream(seed: int, purpose: int) -> int:
    """Seed of an independent stream derived from (seed, purpose)."""
    with np.errstate(over="ignore"):
        z = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN
                           + np.uint64(purpose)], dtype=np.uint64))
    return int(z[0])


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles uniform on [0, 1) from the top 53 bits."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """int64 uniform on [lo, hi) (hi - lo a power of two up to 2^62, or any
    range by 128-bit-free multiply-shift on the top 32 bits)."""
    span = hi - lo
    r = splitmix64(seed, count)
    if span & (span - 1) == 0:
        v = (r & np.uint64(span - 1)).astype(np.int64)
    else:
        assert span < (1 << 32)
        v = (((r >> np.uint64(32)) * np.uint64(span)) >> np.uint64(32)).astype(np.int64)
    return v + np.int64(lo)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller on two uniform streams."""
    u1 = uniform01(substream(seed, 1), count)
    u2 = uniform01(substream(seed, 2), count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def add_exact_duplicates(coords: np.ndarray, frac: float, seed: int) -> np.ndarray:
    """Overwrite floor(frac*n) distinct target rows, each with a copy of a
    uniformly chosen non-target row (so every target becomes an exact
    duplicate of some other row)."""
    n = coords.shape[0]
    nd = int(np.floor(frac * n))
    if nd == 0 or n < 2:
        return coords
    order = np.argsort(splitmix64(substream(seed, 11), n), kind="stable")
    targets = order[:nd]
    keep = order[nd:]
    pick = uniform_int(substream(seed, 12), nd, 0, 1 << 31) % len(keep)
    out = coords.copy()
    out[targets] = coords[keep[pick]]
    return out


# ---------------------------------------------------------------- workloads

def cloud_int_uniform(n: int, k: int, bits: int, seed: int, dtype=np.int64,
                      dup_frac: float = 0.0) -> np.ndarray:
    """n x k integers uniform on [0, 2^bits), optionally with exact duplicates."""
    c = uniform_int(seed, n * k, 0, 1 << bits).reshape(n, k).astype(dtype)
    if dup_frac > 0:
        c = add_exact_duplicates(c, dup_frac, seed)
    return np.ascontiguousarray(c)


def cloud_gmm(n: int, k: int, seed: int, components: int = 64,
              mean_lo: float = -1000.0, mean_hi: float = 1000.0,
              sigma_lo: float = 0.1, sigma_hi: float = 10.0) -> np.ndarray:
    """n x k float32 from an isotropic Gaussian mixture: equal weights,
    means uniform in [mean_lo, mean_hi]^k, per-component sigma log-uniform
    in [sigma_lo, sigma_hi]."""
    means = mean_lo + (mean_hi - mean_lo) * uniform01(substream(seed, 21), components * k)
    means = means.reshape(components, k)
    ls = uniform01(substream(seed, 22), components)
    sig = np.exp(np.log(sigma_lo) + (np.log(sigma_hi) - np.log(sigma_lo)) * ls)
    comp = uniform_int(substream(seed, 23), n, 0, 1 << 32) % components
    z = normal(substream(seed, 24), n * k).reshape(n, k)
    pts = means[comp] + sig[comp, None] * z
    return np.ascontiguousarray(pts.astype(np.float32))


def cloud_unit_cube(n: int, k: int, seed: int, dup_frac: float = 0.0) -> np.ndarray:
    """n x k float32 uniform in [0, 1)^k (24-bit mantissa draws)."""
    u = (splitmix64(seed, n * k) >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)
    c = u.reshape(n, k)
    if dup_frac > 0:
        c = add_exact_duplicates(c, dup_frac, seed)
    return np.ascontiguousarray(c)


# Named workloads.  Sizes follow the five build configurations: a small
# int64 cloud with 1% duplicates, a 2^26-point float32 mixture, an int64
# dimension sweep, a batch of 4096 uneven clouds and a served request stream.

def small_int64(seed: int = 1, n: int = 16384, k: int = 3) -> np.ndarray:
    """n=16384, k=3, int64 uniform in [0, 2^20), 1% exact duplicates."""
    return cloud_int_uniform(n, k, 20, seed, np.int64, dup_frac=0.01)


def large_gmm(seed: int = 2, n: int = 1 << 26, k: int = 3) -> np.ndarray:
    """n=2^26, k=3, float32 64-component isotropic Gaussian mixture."""
    return cloud_gmm(n, k, seed)


def sweep_int64(k: int, n: int = 1 << 22, seed: int | None = None) -> np.ndarray:
    """n=2^22 int64 uniform in [0, 2^40) at dimension k (seed 3 + k)."""
    return cloud_int_uniform(n, k, 40, 3 + k if seed is None else seed, np.int64)


def batch_sizes(count: int = 4096, seed: int = 4, lo_log2: float = 6.0,
                hi_log2: float = 16.0) -> np.ndarray:
    """Cloud sizes floor(2^U(lo_log2, hi_log2))."""
    u = uniform01(substream(seed, 31), count)
    return np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def batch_clouds(count: int = 4096, seed: int = 4, k: int = 3,
                 lo_log2: float = 6.0, hi_log2: float = 16.0,
                 dup_frac: float = 0.005) -> list[np.ndarray]:
    """``count`` float32 unit-cube clouds, log-uniform sizes, 0.5% duplicates each."""
    sizes = batch_sizes(count, seed, lo_log2, hi_log2)
    return [cloud_unit_cube(int(s), k, substream(seed, 1000 + i), dup_frac)
            for i, s in enumerate(sizes)]


def serving_requests(count: int = 20000, seed: int = 5, lo_log2: float = 8.0,
                     hi_log2: float = 20.0):
    """Request descriptors for a Poisson stream: (size, k, kind, seed) with
    sizes log-uniform in [2^lo, 2^hi], k uniform in {2,3,4}, kind 0 = int32
    uniform in [0, 2^24), kind 1 = float32 Gaussian mixture.  Coordinates
    are drawn lazily with :func:`serving_cloud`."""
    u = uniform01(substream(seed, 41), count)
    sizes = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    ks = 2 + uniform_int(substream(seed, 42), count, 0, 1 << 32) % 3
    kinds = uniform_int(substream(seed, 43), count, 0, 2)
    return [(int(sizes[i]), int(ks[i]), int(kinds[i]), substream(seed, 5000 + i))
            for i in range(count)]


def serving_cloud(size: int, k: int, kind: int, seed: int) -> np.ndarray:
    if kind == 0:
        return cloud_int_uniform(size, k, 24, seed, np.int32)
    return cloud_gmm(size, k, seed)


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = uniform01(substream(seed, 51), count)
    return np.cumsum(-np.log1p(-u) / rate_per_s)
