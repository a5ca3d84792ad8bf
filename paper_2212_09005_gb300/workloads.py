"""Seeded synthetic inputs for the filter workloads.

This module only generates keys. It holds none of the filters' arithmetic
(no fingerprinting, no placement), so the CPU oracle and the CUDA path can
both be fed from it without sharing any method code.

The paper's microbenchmarks use 64-bit items taken from hashed cuRAND XORWOW
output, with a different seed for the negative (absent) set (Sec. 6,
"Microbenchmarks setup"). Here a counter-based generator stands in for that
stream: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). Item i of stream `seed` is the SplitMix64
output mix(seed + (i + 1) * golden_gamma), so any index range can be produced
independently, on any machine, with identical results.

Skewed multisets (the counting benchmark of Sec. 6, Table 5) are drawn from a
Zipf law with the rejection-inversion sampler of Hoermann and Derflinger
("Rejection-inversion to generate variates from monotone discrete
distributions", ACM TOMACS 1996), restated below from its published
description.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_ATTEMPT_SALT = 0xD1B54A32D192ED03
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Items start .. start+count-1 of the SplitMix64 stream with this seed."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
    return _mix(state)


def uniform_keys(seed: int, n: int) -> np.ndarray:
    """n uniform 64-bit keys, pairwise distinct (the stream is a bijection of i)."""
    out = np.empty(n, dtype=np.uint64)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        out[s:s + c] = splitmix64(seed, s, c)
    return out


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sample_without_replacement(seed: int, population: int, k: int) -> np.ndarray:
    """k distinct indices of range(population), as int64, in a seed-fixed order.

    Index j is ranked by item j of the stream `seed`; the k smallest ranks are
    taken and returned in rank order.
    """
    if k > population:
        raise ValueError("sample larger than population")
    ranks = uniform_keys(seed, population)
    if k == population:
        return np.argsort(ranks, kind="stable").astype(np.int64)
    sel = np.argpartition(ranks, k - 1)[:k]
    return sel[np.argsort(ranks[sel], kind="stable")].astype(np.int64)


def sample_with_replacement(seed: int, population: int, k: int) -> np.ndarray:
    """k indices of range(population) drawn uniformly with replacement."""
    u = uniform_keys(seed, k)
    return (u % np.uint64(population)).astype(np.int64)


def zipf_ranks(seed: int, n: int, s: float, universe: int) -> np.ndarray:
    """n ranks in 1..universe with P(k) proportional to k**-s (rejection-inversion).

    With H the antiderivative of x**-s and h(x) = x**-s, a proposal x is drawn by
    inverting H between H(universe + 1/2) and H(3/2) - 1, rounded to the nearest
    integer k, and accepted when k - x is within the precomputed squeeze bound or
    when u >= H(k + 1/2) - h(k). Rejected samples redraw from a fresh counter
    stream (attempt a uses seed XOR a * salt), so every sample is reproducible.
    """
    if s <= 0:
        raise ValueError("exponent must be positive")

    def H(x):
        if s == 1.0:
            return np.log(x)
        return (np.power(x, 1.0 - s) - 1.0) / (1.0 - s)

    def H_inv(y):
        if s == 1.0:
            return np.exp(y)
        return np.power(1.0 + y * (1.0 - s), 1.0 / (1.0 - s))

    def h(x):
        return np.power(x, -s)

    h_x1 = H(1.5) - 1.0
    h_n = H(universe + 0.5)
    squeeze = 2.0 - H_inv(H(2.5) - h(2.0))

    out = np.empty(n, dtype=np.int64)
    for c0 in range(0, n, _CHUNK):
        cn = min(_CHUNK, n - c0)
        pending = np.arange(cn, dtype=np.int64)
        res = np.zeros(cn, dtype=np.int64)
        attempt = 0
        while pending.size:
            a_seed = (seed ^ (attempt * _ATTEMPT_SALT)) & 0xFFFFFFFFFFFFFFFF
            # Counter-based: sample (c0 + j) on attempt a uses stream index c0 + j.
            u01 = np.empty(pending.size, dtype=np.float64)
            # Pending indices are sorted; gather from a contiguous draw.
            lo, hi = int(pending[0]), int(pending[-1]) + 1
            draw = uniform01(a_seed, c0 + lo, hi - lo)
            u01[:] = draw[pending - lo]
            u = h_n + u01 * (h_x1 - h_n)
            x = H_inv(u)
            k = np.floor(x + 0.5)
            k = np.clip(k, 1.0, float(universe))
            ok = ((k - x) <= squeeze) | (u >= H(k + 0.5) - h(k))
            res[pending[ok]] = k[ok].astype(np.int64)
            pending = pending[~ok]
            attempt += 1
            if attempt > 64:
                raise RuntimeError("rejection sampler did not converge")
        out[c0:c0 + cn] = res
    return out


def zipf_keys(seed: int, n: int, s: float = 1.0, universe: int = 1 << 32) -> np.ndarray:
    """Zipf-distributed uint64 keys: key = rank - 1, so keys lie in [0, universe)."""
    return (zipf_ranks(seed, n, s, universe) - 1).astype(np.uint64)


# ---------------------------------------------------------------------------
# Named workloads. Sizes follow the paper's filter sizes and load factors.
# ---------------------------------------------------------------------------

def gqf_uniform_workload(q: int = 20, seed: int = 1):
    """GQF, 2^q slots, 8-bit remainders: insert floor(0.9 * 2^q) uniform keys in one
    batch; query those keys plus 2^q fresh keys (stream seed + 1000)."""
    n_ins = int(0.9 * (1 << q))
    ins = uniform_keys(seed, n_ins)
    neg = uniform_keys(seed + 1000, 1 << q)
    return {"q": q, "r": 8, "insert": ins, "negatives": neg}


def tcf_workload(log2_slots: int = 26, seed: int = 2, batch: int = 1 << 22,
                 n_query: int = 1 << 24):
    """TCF, 2^log2_slots slots, 16-bit tags: insert floor(0.9 * slots) uniform keys in
    batches of `batch`; positive queries sample n_query inserted keys without
    replacement (seed*1000 + 2); negatives are n_query fresh keys (seed + 1000);
    a random half of the inserted keys (seed*1000 + 3) is then deleted."""
    slots = 1 << log2_slots
    n_ins = int(0.9 * slots)
    ins = uniform_keys(seed, n_ins)
    nq = min(n_query, n_ins)
    pos_idx = sample_without_replacement(seed * 1000 + 2, n_ins, nq)
    neg = uniform_keys(seed + 1000, n_query)
    del_idx = sample_without_replacement(seed * 1000 + 3, n_ins, n_ins // 2)
    return {"log2_slots": log2_slots, "tag_bits": 16, "batch": batch, "insert": ins,
            "pos_idx": pos_idx, "negatives": neg, "del_idx": del_idx}


def gqf_zipf_workload(q: int = 28, n: int = 240_000_000, seed: int = 3, s: float = 1.0,
                      universe: int = 1 << 32, n_query: int = 1 << 24):
    """Counting GQF, 2^q slots, 8-bit remainders: a Zipf(s) multiset of n keys over
    `universe`; count queries on n_query stream positions drawn uniformly (seed*1000 + 3)."""
    keys = zipf_keys(seed, n, s, universe)
    qpos = sample_with_replacement(seed * 1000 + 3, n, n_query)
    return {"q": q, "r": 8, "insert": keys, "query": keys[qpos]}
