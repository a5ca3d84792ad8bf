"""GPU parity for the TCF (paper Sec. 4). Bulk mode: the table image (sorted
blocks and backing buckets) equals the oracle's byte for byte after every
batch, and query answers and statuses equal the oracle's. Point mode (Alg. 1):
placement may differ, but answers equal fingerprint membership, which the
oracle computes by brute force."""
import collections

import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, host, first_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def bulk_run(gf, oracle, log2_slots, f, seed, batches, deletes=(), check_each=True):
    O = oracle.TCF(log2_slots, f, seed=seed)
    mb = max(len(b) for b in list(batches) + list(deletes))
    G = gf.TCF(log2_slots, f, gf.MODE_BULK, seed=seed, max_batch=mb)
    for k, b in enumerate(batches):
        st_o = O.insert(b)
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        if check_each or k == len(batches) - 1:
            assert np.array_equal(host(st), st_o)
            d = first_diff(G.export(), O.export())
            assert d is None, (k, d)
    for b in deletes:
        st_o = O.remove(b)
        st = zeros_u8(len(b))
        G.remove(dev_u64(b), st)
        assert np.array_equal(host(st), st_o)
        d = first_diff(G.export(), O.export())
        assert d is None, d
    return O, G


@pytest.mark.parametrize("log2_slots,f", [(10, 16), (14, 16), (17, 16), (12, 8), (15, 8)])
def test_bulk_image_and_answers(gf, oracle, log2_slots, f):
    n = int(0.75 * (1 << log2_slots))  # plus 20% repeated keys: 90% load
    keys = W.uniform_keys(600 + log2_slots, n)
    cuts = [0, 1, 5, n // 7, n // 3, n // 2, n]
    batches = [np.concatenate([keys[a:b], keys[a:a + (b - a) // 5]]) for a, b in zip(cuts, cuts[1:]) if b > a]
    O, G = bulk_run(gf, oracle, log2_slots, f, seed=log2_slots, batches=batches)
    probe = np.concatenate([keys, W.uniform_keys(700 + log2_slots, 50000)])
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))
    # keys rejected as FULL (large batches overflow the backing table) are the
    # only inserted keys that may be missing
    assert host(found)[:n].sum() >= n - G.stats()["failed_keys"]


def test_bulk_small_batches_reach_90_percent(gf, oracle):
    """Batches of 1/16 of the table (the 2^26-slot configuration's ratio) fill
    to 90% with no rejected key, and every inserted key is found."""
    log2_slots = 16
    n = int(0.9 * (1 << log2_slots))
    keys = W.uniform_keys(610, n)
    B = (1 << log2_slots) // 16
    O, G = bulk_run(gf, oracle, log2_slots, 16, seed=6, batches=[keys[i:i + B] for i in range(0, n, B)])
    assert G.stats()["failed_keys"] == 0
    found = zeros_u8(n)
    G.query(dev_u64(keys), found)
    assert host(found).all()


def test_bulk_overfill_backing_and_full(gf, oracle):
    keys = W.uniform_keys(601, 400)
    O, G = bulk_run(gf, oracle, 7, 16, seed=3, batches=[keys[:100], keys[100:250], keys[250:]])
    s = G.stats()
    assert s["backing_used"] == O.backing_count()
    assert s["status_word"] & gf.STATUS_FULL


def test_bulk_deletes(gf, oracle):
    log2_slots = 14
    keys = W.uniform_keys(602, int(0.9 * (1 << log2_slots)))
    ins = [keys[i:i + 4000] for i in range(0, len(keys), 4000)]
    absent = W.uniform_keys(603, 300)
    dels = [keys[::2], np.concatenate([keys[1:2000:2], keys[1:200:2], absent]), keys]
    O, G = bulk_run(gf, oracle, log2_slots, 16, seed=9, batches=ins, deletes=dels)
    probe = np.concatenate([keys, absent])
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))


def test_bulk_one_block_hot_batch(gf, oracle):
    """A batch whose keys all share one primary block: one long segment."""
    O = oracle.TCF(12, 16, seed=4)
    cand = W.uniform_keys(604, 400000)
    b1, _, _ = O.keyinfo(cand)
    hot = cand[b1 == b1[0]][:60]
    batch = np.concatenate([hot, hot[:10]])
    O2, G = bulk_run(gf, oracle, 12, 16, seed=4, batches=[batch], deletes=[batch[::-1]])


def point_membership(O, inserted_ok, probe):
    live = collections.Counter(O.fingerprints(inserted_ok).tolist())
    return np.array([live.get(int(x), 0) > 0 for x in O.fingerprints(probe)], np.uint8)


@pytest.mark.parametrize("log2_slots,f", [(12, 16), (16, 16), (14, 8)])
def test_point_mode_answers_equal_membership(gf, oracle, log2_slots, f):
    O = oracle.TCF(log2_slots, f, seed=11)  # hash only
    G = gf.TCF(log2_slots, f, gf.MODE_POINT, seed=11, max_batch=1 << 20)
    n = int(0.9 * (1 << log2_slots))
    keys = W.uniform_keys(605 + log2_slots, n)
    ok = []
    for i in range(0, n, 5000):
        b = keys[i:i + 5000]
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        s = host(st)
        ok.append(b[s == 0])
    ok = np.concatenate(ok)
    assert len(ok) >= 0.99 * n  # 90% load fits (the backing table takes most overflow)
    probe = np.concatenate([keys, W.uniform_keys(706, 40000)])
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), point_membership(O, ok, probe))
    # delete half of the stored keys: no false negatives for the rest
    gone, kept = ok[::2], ok[1::2]
    st = zeros_u8(len(gone))
    G.remove(dev_u64(gone), st)
    assert not host(st).any()
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), point_membership(O, kept, probe))


def test_point_mode_remove_absent(gf, oracle):
    G = gf.TCF(10, 16, gf.MODE_POINT, seed=1, max_batch=1000)
    keys = W.uniform_keys(607, 500)
    G.insert(dev_u64(keys))
    absent = W.uniform_keys(608, 200)
    O = oracle.TCF(10, 16, seed=1)
    live = collections.Counter(O.fingerprints(keys).tolist())
    exp = np.array([0 if live.get(int(x), 0) > 0 else 2 for x in O.fingerprints(absent)], np.uint8)
    st = zeros_u8(len(absent))
    G.remove(dev_u64(absent), st)
    assert np.array_equal(host(st), exp)


@pytest.mark.slow
def test_bulk_config_2_26(gf, oracle):
    """2^26 slots, 16-bit tags: 15 batches of 2^22 keys to 90% load, 2^24
    positive and 2^24 negative queries, delete a random half, query again.
    Image, statuses and answers equal the oracle's."""
    w = W.tcf_workload()
    ins = w["insert"]
    batches = [ins[i:i + w["batch"]] for i in range(0, len(ins), w["batch"])]
    dels = ins[w["del_idx"]]
    O, G = bulk_run(gf, oracle, 26, 16, seed=2, batches=batches, check_each=False)
    pos = ins[w["pos_idx"]]
    probe = np.concatenate([pos, w["negatives"]])
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))
    for i in range(0, len(dels), w["batch"]):
        b = dels[i:i + w["batch"]]
        st_o = O.remove(b)
        st = zeros_u8(len(b))
        G.remove(dev_u64(b), st)
        assert np.array_equal(host(st), st_o)
    d = first_diff(G.export(), O.export())
    assert d is None, d
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))


def test_worked_example_from_keys(gf, oracle):
    """The hand-derived worked example of the placement rules (tests/golden/
    tcf_q6_f16_worked.txt) through the C ABI: 4 blocks of 16, the shortcut
    limit, the tie to b1, the other block, the backing table, and deletes
    from b1, b2 and the backing table; bytes and statuses as derived."""
    from test_oracle_tcf_golden import expect_rows, load

    spec = load("tcf_q6_f16_worked.txt")
    G = gf.TCF(6, 16, gf.MODE_BULK, seed=0, max_batch=64)
    nb, nbk = 4, 8

    def image():
        img = G.export()
        return img[:nb * 32].view(np.uint16).reshape(nb, 16), img[nb * 32:].view(np.uint64).reshape(nbk, 8)

    st = zeros_u8(len(spec["batch1"]))
    G.insert(dev_u64(np.array(spec["batch1"], np.uint64)), st)
    assert (host(st) == 0).all()
    blocks, buckets = image()
    assert np.array_equal(blocks, expect_rows(spec["block1"], nb, 16, np.uint16)) and not buckets.any()
    st = zeros_u8(3)
    G.insert(dev_u64(np.array(spec["batch2"], np.uint64)), st)
    assert (host(st) == 0).all()
    blocks, buckets = image()
    assert np.array_equal(buckets, expect_rows(spec["bucket2"], nbk, 8, np.uint64))
    assert G.stats()["backing_used"] == 3
    st = zeros_u8(len(spec["delete"]))
    G.remove(dev_u64(np.array(spec["delete"], np.uint64)), st)
    assert host(st).tolist() == spec["delete_status"]
    blocks, buckets = image()
    assert np.array_equal(blocks, expect_rows(spec["block3"], nb, 16, np.uint16))
    assert np.array_equal(buckets, expect_rows(spec["bucket3"], nbk, 8, np.uint64))
