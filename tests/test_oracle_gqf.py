"""Pins for the oracle GQF (paper Sec. 5): a hand-derived worked example,
brute-force multisets, the independent canonical builder, exact counts when
the fingerprint is injective, the counting-filter over-count guarantee
(Sec. 1 footnote), the false-positive closed form, and the cluster bound of
Sec. 5.2."""
import collections

import numpy as np
import pytest

from paper_2212_09005_gb300.workloads import uniform_keys, zipf_keys
from gqf_golden import load, expected_image, group_arrays


def brute(fps):
    c = collections.Counter(int(x) for x in fps)
    f = np.array(sorted(c), np.uint64)
    n = np.array([c[int(x)] for x in f], np.uint64)
    return c, f, n


def test_worked_example_image(oracle):
    spec = load("gqf_q7_r8_worked.txt")
    G = oracle.GQF(spec["q"], spec["r"])
    fps, cnt = group_arrays(spec)
    assert G.insert_groups(fps, cnt) == len(fps)
    exp = expected_image(spec, G.nslots, G.nblk)
    assert np.array_equal(G.export(), exp)
    assert np.array_equal(oracle.gqf_build(spec["q"], spec["r"], fps, cnt), exp)
    for x, v, c in spec["counts"]:
        assert G.count_fp((x << spec["r"]) | v) == c


@pytest.mark.parametrize("order", ["descending", "shuffled", "split"])
def test_worked_example_history_independent(oracle, order):
    spec = load("gqf_q7_r8_worked.txt")
    fps, cnt = group_arrays(spec)
    exp = expected_image(spec, 256, 4)
    G = oracle.GQF(spec["q"], spec["r"])
    if order == "descending":
        for f, c in zip(fps[::-1], cnt[::-1]):
            assert G.insert_groups([f], [c]) == 1
    elif order == "shuffled":
        perm = np.argsort(uniform_keys(5, len(fps)))
        for i in perm:
            assert G.insert_groups([fps[i]], [cnt[i]]) == 1
    else:
        # counts reached in several increments
        for f, c in zip(fps, cnt):
            c = int(c)
            parts = [1] * min(c, 3) + ([c - 3] if c > 3 else [])
            for p in parts:
                assert G.insert_groups([f], [p]) == 1
    assert np.array_equal(G.export(), exp)


@pytest.mark.parametrize("q,r", [(6, 8), (8, 8), (10, 8), (7, 16), (10, 16)])
def test_brute_force_multiset_batches(oracle, q, r):
    G = oracle.GQF(q, r, seed=q * 31 + r)
    base = uniform_keys(100 + q, 3 * (1 << q))
    live = []
    rng = uniform_keys(200 + q, 64)
    for b in range(6):
        n = int(rng[b] % np.uint64(1 << (q - 2))) + 1
        start = int(rng[b + 10] % np.uint64(len(base) - n))
        batch = base[start:start + n]
        dup = batch[: max(1, n // 4)]
        batch = np.concatenate([batch, dup, dup[:3]])
        st = G.insert(batch)
        assert (st == 0).all()
        live.extend(batch.tolist())
        c, f, n_ = brute(G.fingerprints(np.array(live, np.uint64)))
        gf, gc = G.groups()
        assert np.array_equal(gf, f) and np.array_equal(gc, n_)
        assert np.array_equal(G.export(), oracle.gqf_build(q, r, f, n_))
        probe = np.concatenate([np.array(live[:200], np.uint64), uniform_keys(300 + b, 200)])
        pf = G.fingerprints(probe)
        assert all(int(x) == c.get(int(y), 0) for x, y in zip(G.count(probe), pf))
        if len(live) > (1 << q) * 0.85:
            break


def test_delete_brute_force_and_status(oracle):
    q, r = 9, 8
    G = oracle.GQF(q, r, seed=3)
    keys = uniform_keys(41, 300)
    ins = np.concatenate([keys, keys[:40], keys[:40], keys[:5]])
    assert (G.insert(ins) == 0).all()
    fp = G.fingerprints(ins)
    cnt = collections.Counter(fp.tolist())
    # delete: 3 copies of keys[0..4] (4 live: 3 removed, ok),
    # 5 copies of keys[5..9] (3 live: 2 not found), keys[100..149] once,
    # and 20 never-inserted keys
    absent = uniform_keys(42, 20)
    dele = np.concatenate([np.repeat(keys[:5], 3), np.repeat(keys[5:10], 5), keys[100:150], absent])
    st = G.remove(dele)
    dfp = G.fingerprints(dele)
    # expected status per key: the first min(c, d) occurrences (batch order) succeed
    seen = collections.Counter()
    for i, f in enumerate(dfp.tolist()):
        seen[f] += 1
        exp = 0 if seen[f] <= cnt.get(f, 0) else 2
        assert st[i] == exp, (i, f)
    for f in dfp.tolist():
        cnt[f] = max(0, cnt.get(f, 0) - 1)
    live = {f: c for f, c in cnt.items() if c > 0}
    f = np.array(sorted(live), np.uint64)
    n = np.array([live[int(x)] for x in f], np.uint64)
    gf, gc = G.groups()
    assert np.array_equal(gf, f) and np.array_equal(gc, n)
    assert np.array_equal(G.export(), oracle.gqf_build(q, r, f, n))


def test_delete_everything_leaves_zero_image(oracle):
    G = oracle.GQF(8, 8, seed=9)
    keys = uniform_keys(43, 230)
    ins = np.concatenate([keys, keys[:30]])
    G.insert(ins)
    st = G.remove(ins[::-1])
    assert (st == 0).all()
    assert not G.export().any()


def test_one_quotient_many_remainders_and_big_counts(oracle):
    q, r = 10, 8
    G = oracle.GQF(q, r)
    x = 200
    rems = np.arange(0, 256, 3, dtype=np.uint64)
    counts = np.array([1, 2, 3, 257, 258, 65537, 65538, 1 << 40, 2**64 - 1] * 20, np.uint64)[: len(rems)]
    fps = (np.uint64(x) << np.uint64(r)) | rems
    assert G.insert_groups(fps, counts) == len(fps)
    for f, c in zip(fps.tolist(), counts.tolist()):
        assert G.count_fp(f) == c
    assert np.array_equal(G.export(), oracle.gqf_build(q, r, fps, counts))
    gf, gc = G.groups()
    assert np.array_equal(gf, fps) and np.array_equal(gc, counts)


def test_counter_digit_boundaries_incremental(oracle):
    G = oracle.GQF(6, 8)
    fp = (5 << 8) | 77
    total = 0
    for inc in [1, 1, 1, 254, 1, 1, 65278, 1]:
        total += inc
        assert G.insert_groups([fp], [inc]) == 1
        assert G.count_fp(fp) == total
        assert np.array_equal(G.export(), oracle.gqf_build(6, 8, [fp], [total]))


def test_cluster_into_tail_and_overflow_prefix_rule(oracle):
    q, r = 6, 8  # N = 64, tail = 64, 128 slots
    G = oracle.GQF(q, r)
    # 60 remainders on quotient 63: spills 59 slots into the tail
    fps = (np.uint64(63) << np.uint64(8)) | np.arange(60, dtype=np.uint64)
    assert G.insert_groups(fps, np.ones(60, np.uint64)) == 60
    # groups on quotients 40..59 push that run further right until the tail is full;
    # the accepted prefix must fit and one more group must not
    more = (np.arange(40, 60, dtype=np.uint64) << np.uint64(8)) | np.uint64(1)
    k = G.insert_groups(more, np.ones(20, np.uint64))
    allf = np.sort(np.concatenate([fps, more[:k]]))
    assert oracle.gqf_build(q, r, allf, np.ones(len(allf), np.uint64)) is not None
    if k < 20:
        over = np.sort(np.concatenate([fps, more[: k + 1]]))
        assert oracle.gqf_build(q, r, over, np.ones(len(over), np.uint64)) is None
    assert np.array_equal(G.export(), oracle.gqf_build(q, r, allf, np.ones(len(allf), np.uint64)))


def test_overflow_keeps_longest_sorted_prefix_via_keys(oracle):
    q, r = 6, 8
    G = oracle.GQF(q, r, seed=1)
    keys = uniform_keys(44, 150)  # more than 128 slots
    st = G.insert(keys)
    fp = G.fingerprints(keys)
    ok = st == 0
    assert ok.any() and (~ok).any()
    # accepted keys are exactly those with fingerprint below a cut
    cut = fp[~ok].min()
    assert (fp[ok] < cut).all() and (fp[~ok] >= cut).all()
    c, f, n = brute(fp[ok])
    assert np.array_equal(G.export(), oracle.gqf_build(q, r, f, n))
    c2, f2, n2 = brute(fp[fp <= cut])
    assert oracle.gqf_build(q, r, f2, n2) is None


def test_exact_counts_when_fingerprint_is_injective(oracle):
    """Keys below 2^p fold to themselves and mix_p is a bijection, so counts are
    the true multiplicities of the keys (no hash in the expected values)."""
    q, r = 14, 8
    G = oracle.GQF(q, r, seed=77)
    keys = (uniform_keys(45, 9000) % np.uint64(1 << (q + r)))
    multi = np.concatenate([keys, keys[:3000], keys[:100]])
    assert (G.insert(multi) == 0).all()
    true = collections.Counter(multi.tolist())
    got = G.count(keys)
    assert all(int(g) == true[int(k)] for g, k in zip(got, keys))
    others = uniform_keys(46, 5000) % np.uint64(1 << (q + r))
    others = others[~np.isin(others, keys)]
    assert (G.count(others) == 0).all()


def test_zipf_counts_exact_with_p_36(oracle):
    """Counting config shape: keys < 2^32 <= 2^p give exact per-key counts."""
    G = oracle.GQF(24, 8, seed=3)  # p = 32 = log2 of the key universe
    keys = zipf_keys(3, 200000)
    assert (G.insert(keys) == 0).all()
    u, c = np.unique(keys, return_counts=True)
    pick = np.concatenate([np.arange(50), np.arange(len(u) - 50, len(u))])
    got = G.count(u[pick])
    assert np.array_equal(got, c[pick].astype(np.uint64))


def test_counts_never_under_true(oracle):
    """Sec. 1 footnote: a wrong count is always an over-estimate."""
    q, r = 10, 8  # p = 18 < 64: collisions exist
    G = oracle.GQF(q, r, seed=5)
    keys = uniform_keys(47, 900)
    multi = np.concatenate([keys, keys[:200]])
    G.insert(multi)
    true = collections.Counter(multi.tolist())
    got = G.count(keys)
    assert all(int(g) >= true[int(k)] for g, k in zip(got, keys))
    fp = G.fingerprints(keys)
    byfp = collections.Counter(G.fingerprints(multi).tolist())
    assert all(int(g) == byfp[int(f)] for g, f in zip(got, fp))


def test_fpr_matches_closed_form(oracle):
    """Fresh queries hit a stored fingerprint with probability d / 2^p."""
    q, r = 16, 8
    G = oracle.GQF(q, r, seed=11)
    keys = uniform_keys(48, int(0.9 * (1 << q)))
    G.insert(keys)
    d = len(G.groups()[0])
    neg = uniform_keys(1048, 1 << 20)
    fp = (G.count(neg) > 0).mean()
    eps = d / 2 ** (q + r)
    sigma = np.sqrt(eps * (1 - eps) / neg.size)
    assert abs(fp - eps) <= 4 * sigma, (fp, eps, sigma)


def test_cluster_length_bound(oracle):
    """Sec. 5.2: clusters stay far below the 8192-slot lock region at <= 95% load,
    and below the ln(2^q)/(a - ln a - 1) bound."""
    import math

    q = 16
    G = oracle.GQF(q, 8, seed=12)
    a = 0.95
    G.insert(uniform_keys(49, int(a * (1 << q))))
    mc = G.max_cluster()
    assert mc < 8192
    assert mc < math.log(2 ** q) / (a - math.log(a) - 1)
    assert mc == _clusters_from_image(G.export(), G.nblk, G.nslots)


def test_uniform_config_shape_small(oracle):
    """The 2^20-slot uniform config, scaled to 2^14: one batch to 90% load,
    every inserted key found, counts equal fingerprint multiplicities."""
    q = 14
    G = oracle.GQF(q, 8, seed=1)
    keys = uniform_keys(1, int(0.9 * (1 << q)))
    assert (G.insert(keys) == 0).all()
    assert (G.count(keys) >= 1).all()
    _, f, n = brute(G.fingerprints(keys))
    assert np.array_equal(G.export(), oracle.gqf_build(q, 8, f, n))


@pytest.mark.parametrize("q,r,load", [(10, 8, 0.6), (9, 16, 0.45), (8, 8, 1.3)])
def test_counted_insert_equals_repeated_keys(oracle, q, r, load):
    """Values through the counters: a key with count c is c copies. The table
    equals the one built from the keys repeated c times (at load 1.3 the batch
    overflows and the kept prefix must agree too), each key's status equals
    its copies', and counts are the summed weights for injective keys."""
    n = int(load * (1 << q))
    keys = uniform_keys(1200 + q, n) & np.uint64((1 << (q + r)) - 1)
    keys = np.concatenate([keys, keys[:n // 5]])
    rng = np.random.default_rng(q)
    counts = rng.integers(1, 5, keys.size).astype(np.uint32)
    counts[::37] = rng.integers(250, 70000, counts[::37].size)  # counters of several digits
    A, B = oracle.GQF(q, r, seed=3), oracle.GQF(q, r, seed=3)
    st_a = A.insert_counts(keys, counts)
    rep = np.repeat(keys, counts)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    st_b = B.insert(rep)
    assert np.array_equal(A.export(), B.export())
    assert np.array_equal(st_a, st_b[first])
    if load > 1:
        assert (st_a == 1).any() and (st_a == 0).any()
    else:
        assert (st_a == 0).all()
        want = collections.Counter()
        for k, c in zip(keys.tolist(), counts.tolist()):
            want[k] += c
        u = np.array(sorted(want), np.uint64)
        assert np.array_equal(A.count(u), np.array([want[int(k)] for k in u], np.uint64))


def _clusters_from_image(img, nblk, nslots):
    """Longest stretch of slots in use, read from an image's metadata bits by
    prefix counts, not by walking runs: slot s is in use exactly when more
    occupied quotients lie at or below s than run ends lie below s (the runs
    of quotients <= s that are still open at s cover it; a run never starts
    before its quotient)."""
    meta = img[:nblk * 32].reshape(nblk, 32)
    occ = np.unpackbits(meta[:, 0:8], axis=1, bitorder="little").reshape(-1)[:nslots].astype(np.int64)
    rend = np.unpackbits(meta[:, 8:16], axis=1, bitorder="little").reshape(-1)[:nslots].astype(np.int64)
    used = np.cumsum(occ) > (np.cumsum(rend) - rend)
    best = cur = 0
    for u in used.tolist():
        cur = cur + 1 if u else 0
        best = max(best, cur)
    return best


def test_max_cluster_worked_example(oracle):
    """The hand-derived example's clusters are slots 3..7, 10..14, 60..66 and
    127..133 (the derivation in the fixture), so the longest is 7 slots."""
    spec = load("gqf_q7_r8_worked.txt")
    G = oracle.GQF(spec["q"], spec["r"])
    fps, cnt = group_arrays(spec)
    G.insert_groups(fps, cnt)
    assert G.max_cluster() == 7
    assert _clusters_from_image(G.export(), G.nblk, G.nslots) == 7


@pytest.mark.parametrize("q,r,load", [(10, 8, 0.5), (12, 8, 0.9), (12, 16, 0.95), (14, 8, 0.97)])
def test_max_cluster_equals_prefix_count_scan(oracle, q, r, load):
    """Sec. 5.2 cluster lengths: the oracle's longest cluster equals the
    longest stretch of in-use slots found by prefix counts over the image."""
    G = oracle.GQF(q, r, seed=q + r)
    keys = uniform_keys(4000 + q, int(load * (1 << q)))
    G.insert(np.concatenate([keys, keys[: len(keys) // 7]]))  # some counters too
    mc = G.max_cluster()
    assert mc >= 2
    assert mc == _clusters_from_image(G.export(), G.nblk, G.nslots)
