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


def gqf_target_workload(q: int = 28, seed: int = 9, n_query: int = 1 << 24, load: float = 0.9):
    """GQF at the target size, 2^q home slots, 8-bit remainders, filled to
    `load` with uniform keys in one batch (stream seed); positive count
    queries take n_query inserted keys drawn with replacement
    (seed*1000 + 2), negatives are n_query fresh keys (seed + 1000); then
    n_query distinct inserted keys (seed*1000 + 3) are deleted."""
    n_ins = int(load * (1 << q))
    ins = uniform_keys(seed, n_ins)
    nq = min(n_query, n_ins)
    pos_idx = sample_with_replacement(seed * 1000 + 2, n_ins, nq)
    neg = uniform_keys(seed + 1000, n_query)
    del_idx = sample_without_replacement(seed * 1000 + 3, n_ins, nq)
    return {"q": q, "r": 8, "insert": ins, "pos_idx": pos_idx, "negatives": neg, "del_idx": del_idx}


def batched_workload(n_filters: int = 4096, seed: int = 4, emin: int = 10, emax: int = 20,
                     load_lo: float = 0.85, load_hi: float = 0.95, tcf_rounds: int = 8):
    """Many small filters: the first half TCF (16-bit tags, bulk mode), the
    second half GQF (8-bit remainders). Filter i has 2^e_i slots (TCF) or home
    slots (GQF), e_i uniform over the integers emin..emax (stream seed), and
    receives floor(L_i * 2^e_i) distinct uniform keys with L_i uniform in
    [load_lo, load_hi) (stream seed + 1); its hash seed is item i of stream
    seed + 3. Insert keys are consecutive ranges of stream seed + 2 in filter
    order; the negatives, one fresh key per inserted key, are consecutive
    ranges of stream seed + 1000. TCF filters take their keys in `tcf_rounds`
    near-equal consecutive chunks (round j inserts chunk j of every TCF
    filter); GQF filters take theirs in one batch."""
    span = emax - emin + 1
    e = (emin + (splitmix64(seed, 0, n_filters) % np.uint64(span))).astype(np.int64)
    load = load_lo + (load_hi - load_lo) * uniform01(seed + 1, 0, n_filters)
    n_keys = np.floor(load * np.power(2.0, e)).astype(np.int64)
    off = np.zeros(n_filters + 1, dtype=np.int64)
    np.cumsum(n_keys, out=off[1:])
    total = int(off[-1])
    return {
        "n_filters": n_filters, "n_tcf": n_filters // 2, "log2_slots": e, "n_keys": n_keys,
        "offsets": off, "hash_seeds": splitmix64(seed + 3, 0, n_filters),
        "insert": uniform_keys(seed + 2, total), "negatives": uniform_keys(seed + 1000, total),
        "tcf_rounds": tcf_rounds,
    }


def round_chunks(offsets: np.ndarray, rounds: int):
    """Split each filter's key range [offsets[i], offsets[i+1]) into `rounds`
    near-equal consecutive chunks: returns (round, member) -> (start, end)
    as an int64 array of shape (rounds, n, 2)."""
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    lens = off[1:] - off[:-1]
    out = np.empty((rounds, n, 2), dtype=np.int64)
    for j in range(rounds):
        out[j, :, 0] = off[:-1] + (lens * j) // rounds
        out[j, :, 1] = off[:-1] + (lens * (j + 1)) // rounds
    return out


def keys_at(seed: int, pos: np.ndarray) -> np.ndarray:
    """Items at arbitrary positions `pos` of stream `seed`."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(pos).astype(np.uint64) + np.uint64(1)) * _GAMMA
    return _mix(state)


def uniform_keys_range(seed: int, start: int, n: int) -> np.ndarray:
    """Items start .. start+n-1 of stream `seed` (as uniform_keys, from an offset)."""
    out = np.empty(n, dtype=np.uint64)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        out[s:s + c] = splitmix64(seed, start + s, c)
    return out


def serving_workload(n_filters: int = 64, log2_slots: int = 24, seed: int = 5, bmin: int = 10, bmax: int = 24,
                     mix=(0.50, 0.45, 0.05), prefill: float = 0.5, stop_load: float = 0.9,
                     filter_cap: float = 0.95, max_requests: int = 100000):
    """A request stream for a filter server: n_filters filters of 2^log2_slots
    slots, the first half TCF and the second half GQF, each pre-filled to
    `prefill` with distinct uniform keys. Every inserted key is a fresh item of
    stream seed + 2 (consecutive positions). Request j picks a filter uniformly
    (stream seed + 10, item j), an operation by `mix` (insert, query, delete;
    stream seed + 11) and a size 2^u with u uniform in [bmin, bmax] (stream
    seed + 12; log-uniform sizes).
      insert: fresh keys, capped at what keeps the filter at or below
        filter_cap of its slots (a filter already there gets a query instead);
      query: half of the keys drawn uniformly, with replacement, from the keys
        the filter was ever given (stream seed + 3), half fresh keys of stream
        seed + 1000;
      delete: distinct keys drawn from the filter's live keys (inserted, not yet
        deleted), capped at the live count (stream seed + 4, by rejection).
    The stream ends once the live keys of all filters reach stop_load of all
    slots, or after max_requests requests. Returns the prefill batches (one per
    filter) and the requests as (filter, op, keys), op 0 insert, 1 query,
    2 delete."""
    slots = 1 << log2_slots
    cap = int(filter_cap * slots)
    pre = int(prefill * slots)
    ranges = [[(f * pre, (f + 1) * pre)] for f in range(n_filters)]  # inserted stream positions
    live = [pre] * n_filters
    nxt = n_filters * pre
    dead = np.zeros(1 << 20, np.uint8)                                # deleted positions, one bit each
    prefill_batches = [uniform_keys_range(seed + 2, a, b - a) for (a, b), in ranges]
    total_live = pre * n_filters
    goal = int(stop_load * slots * n_filters)
    pick = splitmix64(seed + 10, 0, max_requests) % np.uint64(n_filters)
    opu = uniform01(seed + 11, 0, max_requests)
    szu = uniform01(seed + 12, 0, max_requests)

    def positions(f, u):
        """Map u in [0, 1) to positions in filter f's inserted ranges."""
        lens = np.array([b - a for a, b in ranges[f]], np.int64)
        starts = np.array([a for a, b in ranges[f]], np.int64)
        cum = np.concatenate([[0], np.cumsum(lens)])
        r = np.minimum((u * cum[-1]).astype(np.int64), cum[-1] - 1)
        k = np.searchsorted(cum, r, side="right") - 1
        return starts[k] + (r - cum[k])

    reqs = []
    j = 0
    while total_live < goal and j < max_requests:
        f = int(pick[j])
        u = opu[j]
        op = 0 if u < mix[0] else (1 if u < mix[0] + mix[1] else 2)
        want = max(1, int(2.0 ** (bmin + (bmax - bmin) * szu[j])))
        size = want
        if op == 0 and cap - live[f] <= 0:
            op = 1
        elif op == 0:
            size = min(want, cap - live[f])
        if op == 2 and live[f] == 0:
            op = 1
        elif op == 2:
            size = min(want, live[f])
        if op == 0:
            keys = uniform_keys_range(seed + 2, nxt, size)
            ranges[f].append((nxt, nxt + size))
            nxt += size
            live[f] += size
            total_live += size
        elif op == 1:
            h = size // 2
            pos = positions(f, uniform01(seed + 3, j << 25, h))
            keys = np.concatenate([keys_at(seed + 2, pos), uniform_keys_range(seed + 1000, j << 25, size - h)])
        else:
            while (nxt >> 3) + 1 > dead.size:
                dead = np.concatenate([dead, np.zeros(dead.size, np.uint8)])
            got = np.zeros(0, np.int64)
            attempt = 0
            while got.size < size:
                a_seed = (seed + 4) ^ ((attempt * _ATTEMPT_SALT) & 0xFFFFFFFFFFFFFFFF)
                cand = positions(f, uniform01(a_seed, j << 25, 2 * (size - got.size) + 16))
                alive = ((dead[cand >> 3] >> (cand & 7).astype(np.uint8)) & 1) == 0
                cand = cand[alive]
                if got.size:
                    gs = np.sort(got)
                    at = np.minimum(np.searchsorted(gs, cand), gs.size - 1)
                    cand = cand[gs[at] != cand]
                order = np.argsort(cand, kind="stable")       # first occurrence of each position
                sc = cand[order]
                first = np.ones(sc.size, bool)
                first[1:] = sc[1:] != sc[:-1]
                cand = cand[np.sort(order[first])]
                got = np.concatenate([got, cand[: size - got.size]])
                attempt += 1
            np.bitwise_or.at(dead, got >> 3, (np.uint8(1) << (got & 7).astype(np.uint8)))
            keys = keys_at(seed + 2, got)
            live[f] -= size
            total_live -= size
        reqs.append((f, op, keys))
        j += 1
    return {"n_filters": n_filters, "n_tcf": n_filters // 2, "log2_slots": log2_slots,
            "prefill": prefill_batches, "requests": reqs}


# ---------------------------------------------------------------------------
# Synthetic k-mer counting workload (stand-in for the sequencing reads the
# paper counts k-mers of, Sec. 6: the real dataset is not available here).
# A random genome of `genome_len` bases; reads of `read_len` bases start at
# uniform positions; each base of a read is replaced by a different random base
# with probability `error_rate` (substitution errors); every k-mer of every
# read is packed 2 bits per base (A=0, C=1, G=2, T=3, first base most
# significant) and taken in canonical form, the smaller of the k-mer and its
# reverse complement. Genomic k-mers repeat about coverage times, erroneous
# ones are mostly unique, as in real reads.
# ---------------------------------------------------------------------------

def _bases(seed: int, start: int, n: int) -> np.ndarray:
    """n bases (0..3) from stream `seed`, 32 per 64-bit draw."""
    words = splitmix64(seed, start // 32, (start % 32 + n + 31) // 32)
    b = ((words[:, None] >> (2 * np.arange(32, dtype=np.uint64))[None, :]) & np.uint64(3)).astype(np.uint8)
    return b.reshape(-1)[start % 32: start % 32 + n]


def revcomp_kmer(x: np.ndarray, k: int) -> np.ndarray:
    """Reverse complement of 2-bit packed k-mers (complement: 3 - base)."""
    x = np.asarray(x, dtype=np.uint64)
    out = np.zeros_like(x)
    for j in range(k):
        out = (out << np.uint64(2)) | (np.uint64(3) - ((x >> np.uint64(2 * j)) & np.uint64(3)))
    return out


def kmers_of_reads(reads: np.ndarray, k: int) -> np.ndarray:
    """Canonical k-mers of every read (rows of 2-bit base codes), read by read."""
    n_reads, length = reads.shape
    w = length - k + 1
    fwd = np.zeros((n_reads, w), np.uint64)
    rev = np.zeros((n_reads, w), np.uint64)
    r64 = reads.astype(np.uint64)
    c64 = np.uint64(3) - r64  # complements
    t = np.empty((n_reads, w), np.uint64)
    two = np.uint64(2)
    for j in range(k):
        np.left_shift(fwd, two, out=fwd)
        np.bitwise_or(fwd, r64[:, j:j + w], out=fwd)
        np.left_shift(c64[:, j:j + w], np.uint64(2 * j), out=t)
        np.bitwise_or(rev, t, out=rev)
    np.minimum(fwd, rev, out=fwd)
    return fwd.reshape(-1)


def _genome_kmers(genome: np.ndarray, k: int) -> np.ndarray:
    """k-mer at every position of a base array: the bases packed 32 to a word,
    first base in the top bits, and each k-mer cut from two adjacent words."""
    n = genome.size
    nw = (n + 31) // 32 + 1
    b = np.zeros(nw * 32, np.uint64)
    b[:n] = genome
    words = np.bitwise_or.reduce(b.reshape(nw, 32) << (np.uint64(62) - np.uint64(2) * np.arange(32, dtype=np.uint64)),
                                 axis=1)
    i = np.arange(n - k + 1, dtype=np.int64)
    w = i >> 5
    off = ((i & 31) * 2).astype(np.uint64)
    hi = words[w] << off
    lo = np.where(off > 0, words[w + 1] >> ((np.uint64(64) - off) & np.uint64(63)), np.uint64(0))
    return (hi | lo) >> np.uint64(64 - 2 * k)


_PAIR_MASKS = [(np.uint64(0x3333333333333333), 2), (np.uint64(0x0F0F0F0F0F0F0F0F), 4),
               (np.uint64(0x00FF00FF00FF00FF), 8), (np.uint64(0x0000FFFF0000FFFF), 16)]


def _revcomp_fast(x: np.ndarray, k: int) -> np.ndarray:
    """revcomp_kmer by bit operations: complement every base (xor 3), reverse
    the order of the 32 two-bit groups of the word, shift back to 2k bits."""
    y = np.asarray(x, dtype=np.uint64) ^ np.uint64((1 << (2 * k)) - 1 if k < 32 else 0xFFFFFFFFFFFFFFFF)
    for m, sh in _PAIR_MASKS:
        y = ((y >> np.uint64(sh)) & m) | ((y & m) << np.uint64(sh))
    y = (y >> np.uint64(32)) | (y << np.uint64(32))
    return y >> np.uint64(64 - 2 * k)


def _read_starts(seed: int, r0: int, m: int, read_len: int, genome_len: int) -> np.ndarray:
    return (splitmix64(seed + 1, r0, m) % np.uint64(genome_len - read_len + 1)).astype(np.int64)


def _error_hits(seed: int, r0: int, m: int, read_len: int, error_rate: float) -> np.ndarray:
    u = (splitmix64(seed + 2, r0 * read_len, m * read_len) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return (u < error_rate).reshape(m, read_len)


def _error_shift(seed: int, r0: int, m: int, read_len: int) -> np.ndarray:
    """1..3: how far (mod 4) a substituted base moves from the true one."""
    return (_bases(seed + 3, r0 * read_len, m * read_len).reshape(m, read_len) % 3) + 1


def synthetic_reads(n_reads: int, seed: int = 6, read_len: int = 100, genome_len: int = 1 << 25,
                    error_rate: float = 0.005, r0: int = 0) -> np.ndarray:
    """Reads r0 .. r0 + n_reads - 1 of the k-mer workload as rows of base codes."""
    genome = _bases(seed, 0, genome_len)
    starts = _read_starts(seed, r0, n_reads, read_len, genome_len)
    reads = genome[starts[:, None] + np.arange(read_len)[None, :]]
    hit = _error_hits(seed, r0, n_reads, read_len, error_rate)
    return np.where(hit, (reads + _error_shift(seed, r0, n_reads, read_len)) & 3, reads).astype(np.uint8)


def kmer_workload(n_kmers: int, seed: int = 6, k: int = 28, read_len: int = 100, genome_len: int = 1 << 25,
                  error_rate: float = 0.005, chunk_reads: int = 1 << 18):
    """Canonical k-mers (uint64, 2k bits) of the first ceil(n_kmers / (read_len
    - k + 1)) reads of `synthetic_reads`, in read order, truncated to n_kmers.
    Streams: genome = seed, read starts = seed + 1, error positions = seed + 2,
    substituted bases = seed + 3. Equal to kmers_of_reads(synthetic_reads(..));
    computed faster from the k-mers at every genome position, each sequencing
    error flipping the bits of its base in the up to k k-mers that cover it."""
    assert 1 <= k <= 32 and read_len >= k
    genome = _bases(seed, 0, genome_len)
    G = genome_len - k + 1
    fwd_g = _genome_kmers(genome, k)
    rev_g = _revcomp_fast(fwd_g, k)
    per = read_len - k + 1
    n_reads = (n_kmers + per - 1) // per
    out = np.empty(n_reads * per, np.uint64)
    cols = np.arange(per)
    for r0 in range(0, n_reads, chunk_reads):
        m = min(chunk_reads, n_reads - r0)
        starts = _read_starts(seed, r0, m, read_len, genome_len)
        idx = starts[:, None] + cols[None, :]
        fwd = fwd_g[idx]
        rev = rev_g[idx]
        er, ep = np.nonzero(_error_hits(seed, r0, m, read_len, error_rate))
        if er.size:
            old = genome[starts[er] + ep].astype(np.uint64)
            new = (old + _error_shift(seed, r0, m, read_len)[er, ep].astype(np.uint64)) & np.uint64(3)
            delta = old ^ new
            for o in range(k):  # the error is base o of k-mer ep - o: one k-mer per error, no repeats
                kk = ep - o
                ok = (kk >= 0) & (kk < per)
                if not ok.any():
                    continue
                ri, ki, d = er[ok], kk[ok], delta[ok]
                fwd[ri, ki] ^= d << np.uint64(2 * (k - 1 - o))
                rev[ri, ki] ^= d << np.uint64(2 * o)
        np.minimum(fwd, rev, out=fwd)
        out[r0 * per:(r0 + m) * per] = fwd.reshape(-1)
    return out[:n_kmers]


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """n arrival times (seconds) of a Poisson process of `rate` per second:
    cumulative exponential gaps -ln(1 - u) / rate, u from stream `seed`."""
    u = uniform01(seed, 0, n)
    return np.cumsum(-np.log1p(-u) / rate)
