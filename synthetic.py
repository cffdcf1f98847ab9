"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds random-number generation and the value distributions of the
workloads only; none of the multiplication methods' arithmetic lives here.

The generator is counter-based splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the i-th draw of a
stream with seed ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` with the
published finaliser (shifts 30/27/31, multipliers 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB).  Everything is generated on the host in numpy and copied
to wherever it is needed, so every consumer sees identical bits.

Distributions (one per workload family):

* ``uniform``       entries in [-1, 1): ``(r >> 11) * 2**-52 - 1`` (53-bit grid).
* ``integers``      entries uniform in [lo, hi] (default [-8, 8]) as ``lo + r mod (hi-lo+1)``;
                    the modulo bias is below 2**-59 for these ranges.
* ``loguniform``    ``sign * 2**E * (1 + f)`` with E a uniform integer in [emin, emax],
                    f uniform on [0, 1) and a uniform random sign: magnitudes
                    log-uniform over 2**emin .. 2**(emax+1).
* ``badly_scaled``  a uniform base with row i of A scaled by 10**u_i and column k
                    of B by 10**v_k, u and v uniform on [-6, 6].
* ``paper_pair``    A uniform, B = 8A (the paper's timing workload, section "Tests").
* ``serving_trace`` products with N, P, M = round(2**(5 + 7U)) (log-uniform on
                    [32, 4096]), Poisson arrivals and a 50/50 accuracy-tier mix.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x11061347
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def stream_seed(config: int, tag: int) -> int:
    """Seed of stream ``tag`` (0 = A, 1 = B, ...) of workload ``config``."""
    return (BASE_SEED + 0x1000 * int(config) + int(tag)) & 0xFFFFFFFFFFFFFFFF


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the counter-based splitmix64 stream ``seed``."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        z = np.arange(offset + lo + 1, offset + hi + 1, dtype=np.uint64)
        z *= _GOLDEN
        z += s
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
        out[lo:hi] = z
    return out


def uniform(rows: int, cols: int, seed: int) -> np.ndarray:
    r = splitmix64(seed, rows * cols)
    x = (r >> np.uint64(11)).astype(np.float64)
    x *= 2.0 ** -52
    x -= 1.0
    return x.reshape(rows, cols)


def integers(rows: int, cols: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    r = splitmix64(seed, rows * cols)
    v = (r % np.uint64(hi - lo + 1)).astype(np.int64) + lo
    return v.astype(np.float64).reshape(rows, cols)


def loguniform(rows: int, cols: int, seed: int, emin: int = -20, emax: int = 19) -> np.ndarray:
    n = rows * cols
    r_exp = splitmix64(seed, n, 0)
    r_frac = splitmix64(seed, n, n)
    e = (r_exp % np.uint64(emax - emin + 1)).astype(np.int64) + emin
    f = (r_frac >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    sign = np.where((r_exp >> np.uint64(63)) == 1, -1.0, 1.0)
    return (sign * np.ldexp(1.0 + f, e.astype(np.int32))).reshape(rows, cols)


def badly_scaled(n: int, seed_a: int, seed_b: int, span: float = 6.0):
    a = uniform(n, n, seed_a)
    b = uniform(n, n, seed_b)
    u = uniform(1, n, seed_a ^ 0x5A5A5A5A).ravel() * span
    v = uniform(1, n, seed_b ^ 0x5A5A5A5A).ravel() * span
    return a * (10.0 ** u)[:, None], b * (10.0 ** v)[None, :]


def paper_pair(n: int, seed: int):
    a = uniform(n, n, seed)
    return a, 8.0 * a


def serving_trace(count: int, seed: int, mean_gap_s: float, tiers=(1e-14, 1e-6)):
    """A list of request dicts: arrival time, N, P, M, tier, and per-request seeds."""
    n = count
    u = splitmix64(seed, 5 * n)
    def unit(x):
        return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    dims = np.rint(2.0 ** (5.0 + 7.0 * unit(u[: 3 * n]))).astype(np.int64).reshape(n, 3)
    gaps = -np.log1p(-unit(u[3 * n: 4 * n])) * mean_gap_s
    arrivals = np.cumsum(gaps)
    tier_idx = (u[4 * n:] >> np.uint64(63)).astype(np.int64)
    out = []
    for i in range(n):
        out.append({"id": i, "arrival_s": float(arrivals[i]), "N": int(dims[i, 0]), "P": int(dims[i, 1]),
                    "M": int(dims[i, 2]), "tier": float(tiers[int(tier_idx[i])]),
                    "seed_a": stream_seed(4, 2 * i + 16), "seed_b": stream_seed(4, 2 * i + 17)})
    return out
