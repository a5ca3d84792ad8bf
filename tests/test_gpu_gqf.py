"""GPU parity for the GQF (paper Sec. 5): the CUDA library's table image must
equal the oracle's byte for byte, and counts / answers / statuses must equal
the oracle's, on seeded inputs (several tiles, ragged tails, duplicates,
deletes, table overflow) and at the paper-scale configurations."""
import collections

import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, zeros_u64, host, first_diff
from gqf_golden import load, expected_image, group_arrays

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def run_batches(gf, oracle, q, r, seed, batches, deletes=()):
    O = oracle.GQF(q, r, seed=seed)
    G = gf.GQF(q, r, seed=seed, max_batch=max(len(b) for b in list(batches) + list(deletes) + [[0]]))
    for b in batches:
        st_o = O.insert(b)
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        assert np.array_equal(host(st), st_o)
        d = first_diff(G.export(), O.export())
        assert d is None, d
    for b in deletes:
        st_o = O.remove(b)
        st = zeros_u8(len(b))
        G.remove(dev_u64(b), st)
        assert np.array_equal(host(st), st_o)
        d = first_diff(G.export(), O.export())
        assert d is None, d
    return O, G


@pytest.mark.parametrize("q,r", [(8, 8), (11, 8), (13, 8), (10, 16), (14, 16)])
def test_batches_with_duplicates_image_and_counts(gf, oracle, q, r):
    base = W.uniform_keys(500 + q, 1 << q)
    sizes = [1, 7, 300, (1 << q) // 3, (1 << q) // 4]
    batches, at = [], 0
    for s in sizes:
        b = base[at:at + s]
        at += s
        batches.append(np.concatenate([b, b[: s // 3], b[:2]]))
    O, G = run_batches(gf, oracle, q, r, seed=q, batches=batches)
    probe = np.concatenate([base[:at], W.uniform_keys(900 + q, 5000)])
    c = zeros_u64(len(probe))
    G.count(dev_u64(probe), c)
    assert np.array_equal(host(c), O.count(probe))
    f = zeros_u8(len(probe))
    G.query(dev_u64(probe), f)
    assert np.array_equal(host(f), (O.count(probe) > 0).astype(np.uint8))


def test_deletes_status_and_image(gf, oracle):
    q, r = 12, 8
    keys = W.uniform_keys(501, 3000)
    ins = np.concatenate([keys, keys[:500], keys[:500], keys[:7]])
    absent = W.uniform_keys(502, 100)
    dels = [
        np.concatenate([np.repeat(keys[:20], 4), keys[1000:1500], absent]),
        keys[::3],
        ins,  # everything, including copies already gone
    ]
    O, G = run_batches(gf, oracle, q, r, seed=5, batches=[ins], deletes=dels)
    assert not G.export().any()


def test_worked_example_from_keys(gf, oracle):
    """The hand-derived golden table, reached through keys whose fingerprints
    are the example's groups (keys = inverse hash of each fingerprint)."""
    spec = load("gqf_q7_r8_worked.txt")
    q, r = spec["q"], spec["r"]
    p = q + r
    fps, cnt = group_arrays(spec)
    keys = []
    for f, c in zip(fps.tolist(), cnt.tolist()):
        k = oracle.unmix_p(f, p)  # seed 0: fingerprint = mix_p(key) for key < 2^p
        keys += [k] * min(c, 5000)
    # counts above 5000 are reached with a second, repeated batch
    G = gf.GQF(q, r, seed=0, max_batch=200000)
    G.insert(dev_u64(np.array(keys, np.uint64)))
    rest = []
    for f, c in zip(fps.tolist(), cnt.tolist()):
        if c > 5000:
            rest += [oracle.unmix_p(f, p)] * (c - 5000)
    if rest:
        G.insert(dev_u64(np.array(rest, np.uint64)))
    exp = expected_image(spec, 256, 4)
    d = first_diff(G.export(), exp)
    assert d is None, d


def test_overflow_longest_prefix(gf, oracle):
    """More keys than slots: the longest sorted prefix of the groups is kept,
    the other keys get FULL, exactly as in the oracle."""
    q, r = 7, 8  # 128 + 128 slots
    keys = W.uniform_keys(503, 300)
    O = oracle.GQF(q, r, seed=1)
    G = gf.GQF(q, r, seed=1, max_batch=300)
    failed = 0
    for b in (keys[:100], keys[100:]):
        st_o = O.insert(b)
        failed += int((st_o == gf.KEY_FULL).sum())
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        assert np.array_equal(host(st), st_o)
        d = first_diff(G.export(), O.export())
        assert d is None, d
    assert failed > 0
    s_ = G.stats()
    assert s_["status_word"] & gf.STATUS_FULL
    assert s_["failed_keys"] == failed


def test_empty_and_single(gf, oracle):
    G = gf.GQF(6, 8, seed=0, max_batch=16)
    G.insert(dev_u64(np.zeros(0, np.uint64)))
    assert not G.export().any()
    O, G2 = run_batches(gf, oracle, 6, 8, seed=2, batches=[np.array([12345], np.uint64)])
    c = zeros_u64(1)
    G2.count(dev_u64(np.array([12345], np.uint64)), c)
    assert host(c)[0] == 1


def test_zipf_small_exact_counts(gf, oracle):
    q = 18
    keys = W.zipf_keys(3, 300000, 1.0, 1 << 20)  # universe 2^20 <= 2^p; ~90K distinct
    O, G = run_batches(gf, oracle, q, 8, seed=3, batches=[keys[:200000], keys[200000:]])
    assert G.stats()["failed_keys"] == 0
    u, c = np.unique(keys, return_counts=True)
    got = zeros_u64(len(u))
    G.count(dev_u64(u), got)
    assert np.array_equal(host(got), c.astype(np.uint64))


def test_uniform_config_2_20(gf, oracle):
    """2^20 slots, 8-bit remainders: one batch of floor(0.9 * 2^20) keys, then
    queries of those keys and 2^20 fresh keys; image, answers and FPR."""
    w = W.gqf_uniform_workload(20, seed=1)
    O, G = run_batches(gf, oracle, 20, 8, seed=1, batches=[w["insert"]])
    probe = np.concatenate([w["insert"], w["negatives"]])
    f = zeros_u8(len(probe))
    G.query(dev_u64(probe), f)
    got = host(f)
    assert got[: len(w["insert"])].all()
    exp = (O.count(probe) > 0).astype(np.uint8)
    assert np.array_equal(got, exp)
    d = len(O.groups()[0])
    eps = d / 2 ** 28
    fpr = got[len(w["insert"]):].mean()
    assert abs(fpr - eps) <= 4 * np.sqrt(eps * (1 - eps) / len(w["negatives"]))


@pytest.mark.slow
def test_counting_config_2_28_zipf(gf, oracle):
    """2^28 slots, 2.4e8 Zipf(1.0) keys over 2^32 in one batch: every sampled
    count equals the key's true multiplicity (fingerprints are injective, p = 36),
    and the whole table image equals the canonical builder's."""
    import torch

    w = W.gqf_zipf_workload()
    keys = w["insert"]
    G = gf.GQF(28, 8, seed=3, max_batch=len(keys))
    st = zeros_u8(len(keys))
    G.insert(dev_u64(keys), st)
    assert not host(st).any()
    u, c = np.unique(keys, return_counts=True)
    qk = w["query"]
    got = zeros_u64(len(qk))
    G.count(dev_u64(qk), got)
    exp = c[np.searchsorted(u, qk)].astype(np.uint64)
    assert np.array_equal(host(got), exp)
    O = oracle.GQF(28, 8, seed=3)
    fu = O.fingerprints(u)
    order = np.argsort(fu)
    img = oracle.gqf_build(28, 8, fu[order], c[order].astype(np.uint64))
    d = first_diff(G.export(), img)
    assert d is None, d
    del G
    torch.cuda.empty_cache()
    # the same batch without statuses (no sorted indices)
    G2 = gf.GQF(28, 8, seed=3, max_batch=len(keys))
    G2.insert(dev_u64(keys))
    d = first_diff(G2.export(), img)
    assert d is None, d
    del G2
    torch.cuda.empty_cache()


def _no_status_rounds(gf, oracle, q, r, seed, rounds):
    """Inserts and removes without per-key statuses (the benchmark's calls:
    no sorted indices travel with the fingerprints); the image must equal the
    oracle's after every call."""
    O = oracle.GQF(q, r, seed=seed)
    G = gf.GQF(q, r, seed=seed, max_batch=max(len(b) for _, b in rounds))
    for op, b in rounds:
        if op == "ins":
            O.insert(b)
            G.insert(dev_u64(b))
        else:
            O.remove(b)
            G.remove(dev_u64(b))
        d = first_diff(G.export(), O.export())
        assert d is None, (op, len(b), d)
    return O, G


def test_no_status_zipf_batches_match_oracle(gf, oracle):
    """Skewed batches of about 2^20 keys without statuses: heavy keys repeat
    thousands of times inside one sort tile and across tiles; a ragged length,
    then a remove of a skewed batch."""
    q = 22
    keys = W.zipf_keys(31, (1 << 20) + 77, 1.0, 1 << 24)
    more = W.zipf_keys(32, (1 << 20) + 4096, 1.2, 1 << 24)
    dele = np.concatenate([keys[: 1 << 19], more[: (1 << 19) + 5]])
    O, G = _no_status_rounds(gf, oracle, q, 8, 31, [("ins", keys), ("ins", more), ("rem", dele)])
    u, c = np.unique(np.concatenate([keys, more]), return_counts=True)
    probe = u[::97]
    got = zeros_u64(len(probe))
    G.count(dev_u64(probe), got)
    assert np.array_equal(host(got), O.count(probe))


def test_no_status_extremes_match_oracle(gf, oracle):
    """Exactly 2^20 keys of one value (one group of 2^20 copies), 2^20
    distinct keys, and 16-bit remainders."""
    same = np.full(1 << 20, 12345, np.uint64)
    distinct = W.uniform_keys(33, 1 << 20)
    _no_status_rounds(gf, oracle, 22, 8, 7, [("ins", same), ("ins", distinct), ("rem", same[: (1 << 20) - 1])])
    _no_status_rounds(gf, oracle, 21, 16, 8, [("ins", W.zipf_keys(34, (1 << 20) + 1, 1.0, 1 << 22))])


def test_kmer_counting_matches_oracle(gf, oracle):
    """Canonical 28-mers of synthetic reads (repeats near the coverage, unique
    error k-mers) counted in one batch and in two: table image equal to the
    oracle's, and every k-mer's count equal to the oracle's and at least its
    true multiplicity (56-bit k-mers, 26-bit fingerprints)."""
    q, r = 18, 8
    kmers = W.kmer_workload(150000, seed=21, genome_len=1 << 14)
    _no_status_rounds(gf, oracle, q, r, 21, [("ins", kmers)])
    O, G = _no_status_rounds(gf, oracle, q, r, 21, [("ins", kmers[:70001]), ("ins", kmers[70001:])])
    u, c = np.unique(kmers, return_counts=True)
    got = zeros_u64(len(u))
    G.count(dev_u64(u), got)
    got = host(got)
    assert np.array_equal(got, O.count(u))
    assert (got >= c.astype(np.uint64)).all()


def test_inplace_delete_matches_oracle(gf, oracle):
    """Deletes of a small fraction of the table take the in-place cluster path
    (even-odd regions); image and statuses must equal the oracle's."""
    ins = W.uniform_keys(1, int(0.4 * (1 << 20)))  # 40% load: short clusters
    dele1 = np.concatenate([ins[::80], ins[:1000:20], W.uniform_keys(77, 3000)])  # repeats, absent keys
    dele2 = np.concatenate([ins[1::37], ins[1::37]])
    gf.trace_reset()
    gf.trace_enable(True)
    try:
        run_batches(gf, oracle, 20, 8, seed=1, batches=[ins], deletes=[dele1, dele2])
        assert "gqf_delete_phase" in gf.trace_summary(), "the deletes should have been applied in place"
    finally:
        gf.trace_enable(False)


def test_deletes_at_high_load(gf, oracle):
    """At 90% load the clusters are long; whichever path the library takes,
    image and statuses must equal the oracle's."""
    w = W.gqf_uniform_workload(20, seed=1)
    ins = w["insert"]
    dele1 = np.concatenate([ins[::80], ins[:1000:20], W.uniform_keys(77, 3000)])
    dele2 = np.concatenate([ins[1::37], ins[1::37]])
    run_batches(gf, oracle, 20, 8, seed=1, batches=[ins], deletes=[dele1, dele2])


def test_inplace_delete_small_tables_and_counters(gf, oracle):
    q = 11
    keys = W.uniform_keys(78, 1500)
    ins = np.concatenate([keys, np.repeat(keys[:30], 300), np.repeat(keys[30:40], 3)])  # multi-digit counters
    dele = [np.concatenate([np.repeat(keys[:30], 290), keys[30:35]]), np.repeat(keys[:10], 20), keys[100:130]]
    run_batches(gf, oracle, q, 8, seed=4, batches=[ins], deletes=dele)


def _inplace_used(gf):
    return "gqf_insert_phase" in gf.trace_summary()


@pytest.mark.parametrize("q,r,load", [(12, 8, 0.3), (14, 8, 0.6), (13, 16, 0.5), (12, 8, 0.85), (16, 8, 0.7)])
def test_inplace_insert_matches_oracle(gf, oracle, q, r, load):
    """Small batches into a filled table go in place over even-odd regions (the
    paper's Sec. 5.3 scheme); the image must stay byte-identical to the oracle's
    after every batch, with new fingerprints, repeats of stored ones (counters
    growing past one and two digits) and new quotients at every load."""
    n_fill = int(load * (1 << q))
    base = W.uniform_keys(1700 + q, n_fill)
    nf, na = (1 << q) // 80, (1 << q) // 640  # a few groups per delete region of 256 quotients
    extra = W.uniform_keys(1800 + q, 6 * nf)
    batches = [base]  # the merge fills the table
    for j in range(6):
        fresh = extra[j * nf:(j + 1) * nf]
        again = base[j * na:(j + 1) * na]
        hot = np.full(300 * (j + 1), base[7], dtype=np.uint64)  # one counter keeps growing
        batches.append(np.concatenate([fresh, again, hot, fresh[:10]]))
    O = oracle.GQF(q, r, seed=q)
    G = gf.GQF(q, r, seed=q, max_batch=max(len(b) for b in batches))
    gf.trace_reset()
    gf.trace_enable(True)
    try:
        for k, b in enumerate(batches):
            st_o = O.insert(b)
            st = zeros_u8(len(b))
            G.insert(dev_u64(b), st)
            assert np.array_equal(host(st), st_o), k
            d = first_diff(G.export(), O.export())
            assert d is None, (k, d)
        used = _inplace_used(gf)
    finally:
        gf.trace_enable(False)
    if load <= 0.7:
        assert used, "small batches should have been inserted in place"
    probe = np.concatenate([base[:3000], extra, W.uniform_keys(1900 + q, 3000)])
    c = zeros_u64(len(probe))
    G.count(dev_u64(probe), c)
    assert np.array_equal(host(c), O.count(probe))


def test_inplace_insert_and_delete_alternating(gf, oracle):
    """In-place inserts and deletes, alternating on one table, keep it equal to
    the oracle's."""
    q, r = 13, 8
    keys = W.uniform_keys(2100, 6000)
    O = oracle.GQF(q, r, seed=5)
    G = gf.GQF(q, r, seed=5, max_batch=6000)
    O.insert(keys[:4000])
    G.insert(dev_u64(keys[:4000]))
    for j in range(8):
        ins = np.concatenate([keys[4000 + 200 * j:4000 + 200 * (j + 1)], keys[j * 30:(j + 1) * 30]])
        dl = keys[1000 + 150 * j:1000 + 150 * (j + 1)]
        for op, b in (("insert", ins), ("remove", dl)):
            st_o = getattr(O, op)(b)
            st = zeros_u8(len(b))
            getattr(G, op)(dev_u64(b), st)
            assert np.array_equal(host(st), st_o), (j, op)
            assert first_diff(G.export(), O.export()) is None, (j, op)


def test_enumerate_equals_oracle_groups(gf, oracle):
    """The groups of the table in fingerprint order, with their counts, equal
    the oracle's, for 8- and 16-bit remainders, after inserts and deletes;
    an empty filter has none; a smaller cap writes a prefix."""
    import torch

    for q, r in ((16, 8), (15, 16)):
        keys = W.zipf_keys(91 + r, int(0.5 * (1 << q)), 1.0, 1 << 22)
        O = oracle.GQF(q, r, seed=31)
        G = gf.GQF(q, r, seed=31, max_batch=len(keys))
        f0, c0 = G.enumerate()
        assert f0.numel() == 0 and c0.numel() == 0
        for op, b in (("ins", keys), ("rem", keys[::4])):
            (O.insert if op == "ins" else O.remove)(b)
            (G.insert if op == "ins" else G.remove)(dev_u64(b))
            f, c = G.enumerate()
            of, oc = O.groups()
            assert np.array_equal(host(f), of) and np.array_equal(host(c), oc)
        part = torch.empty(100, dtype=torch.int64, device="cuda")
        partc = torch.empty(100, dtype=torch.int64, device="cuda")
        import ctypes
        m = ctypes.c_uint64()
        assert gf.lib().filter_gqf_enumerate(G._h, ctypes.c_void_p(part.data_ptr()), ctypes.c_void_p(partc.data_ptr()),
                                             100, ctypes.byref(m), None) == 0
        assert m.value == len(of)
        assert np.array_equal(host(part), of[:100]) and np.array_equal(host(partc), oc[:100])


def test_keys_of_recovers_keys_and_resizes(gf, oracle):
    """Keys below 2^p come back exactly from the enumerated fingerprints;
    re-inserting them with their counts into a filter twice as large gives
    the same counts there (a resize)."""
    import torch

    q, r = 14, 8
    keys = W.zipf_keys(93, 6000, 1.0, 1 << 20)  # keys < 2^20 <= 2^(q + r)
    G = gf.GQF(q, r, seed=37, max_batch=len(keys))
    G.insert(dev_u64(keys))
    f, c = G.enumerate()
    back = torch.empty_like(f)
    G.keys_of(f, back)
    u, uc = np.unique(keys, return_counts=True)
    got_keys, got_counts = host(back), host(c)
    order = np.argsort(got_keys)
    assert np.array_equal(got_keys[order], u) and np.array_equal(got_counts[order], uc.astype(np.uint64))
    big = gf.GQF(q + 1, r, seed=41, max_batch=len(keys))
    big.insert(dev_u64(np.repeat(got_keys, got_counts.astype(np.int64))))
    cnt = zeros_u64(len(u))
    big.count(dev_u64(u), cnt)
    assert np.array_equal(host(cnt), uc.astype(np.uint64))
