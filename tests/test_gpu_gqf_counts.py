"""GPU parity for the GQF counted insert (values through the counters): a key
with count c adds c to its fingerprint's count in one pass. The table image
equals the oracle's byte for byte after every batch, on both insert paths
(in place for batches of at most one group per 32 slots, the merge for larger
ones) and when the batch overflows; statuses and counts equal the oracle's.
Invalid counts leave the table unchanged."""
import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, zeros_u64, host, first_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def dev_u32(a):
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def counts_for(seed, n, big_every=41):
    rng = np.random.default_rng(seed)
    c = rng.integers(1, 6, n).astype(np.uint32)
    c[::big_every] = rng.integers(200, 300000, c[::big_every].size)  # multi-digit counters
    return c


@pytest.mark.parametrize("q,r,with_status", [(12, 8, True), (14, 8, True), (13, 16, True), (12, 8, False),
                                             (13, 16, False)])
def test_counted_batches_both_paths(gf, oracle, q, r, with_status):
    """Without statuses the counts ride through the sort; with them the
    sorted batch indices pick each key's count."""
    N = 1 << q
    keys = W.zipf_keys(1300 + q, int(0.5 * N), 1.0, 1 << 20)
    # a large batch (merge), then small ones (in place: <= N/32 groups), then large again
    cuts = [0, int(0.3 * N), int(0.3 * N) + N // 64, int(0.3 * N) + N // 40, len(keys)]
    O = oracle.GQF(q, r, seed=q)
    G = gf.GQF(q, r, seed=q, max_batch=len(keys))
    for k, (a, b) in enumerate(zip(cuts, cuts[1:])):
        ks = keys[a:b]
        cs = counts_for(k + q, len(ks))
        st_o = O.insert_counts(ks, cs)
        st = zeros_u8(len(ks)) if with_status else None
        G.insert_counts(dev_u64(ks), dev_u32(cs), st)
        if with_status:
            assert np.array_equal(host(st), st_o), k
        d = first_diff(G.export(), O.export())
        assert d is None, (k, d)
    probe = np.concatenate([keys[:5000], W.uniform_keys(1400 + q, 5000)])
    got = zeros_u64(len(probe))
    G.count(dev_u64(probe), got)
    assert np.array_equal(host(got), O.count(probe))
    # plain inserts and deletes mix with counted ones
    st_o = O.remove(keys[:300])
    st = zeros_u8(300)
    G.remove(dev_u64(keys[:300]), st)
    assert np.array_equal(host(st), st_o)
    assert first_diff(G.export(), O.export()) is None


def test_counted_overflow_keeps_the_prefix(gf, oracle):
    q, r = 8, 8
    keys = W.uniform_keys(1310, 400)
    cs = counts_for(1311, len(keys), big_every=7)
    O = oracle.GQF(q, r, seed=2)
    G = gf.GQF(q, r, seed=2, max_batch=len(keys))
    st_o = O.insert_counts(keys, cs)
    assert (st_o == 1).any() and (st_o == 0).any()
    st = zeros_u8(len(keys))
    G.insert_counts(dev_u64(keys), dev_u32(cs), st)
    assert np.array_equal(host(st), st_o)
    assert first_diff(G.export(), O.export()) is None
    assert G.stats()["failed_keys"] == int((st_o == 1).sum())


def test_invalid_counts_leave_the_table(gf, oracle):
    keys = W.uniform_keys(1320, 1000)
    G = gf.GQF(12, 8, seed=1, max_batch=len(keys))
    G.insert(dev_u64(keys[:500]))
    before = G.export()
    cs = np.ones(len(keys), np.uint32)
    cs[777] = 0
    with pytest.raises(gf.FilterError):
        G.insert_counts(dev_u64(keys), dev_u32(cs))
    cs = np.full(len(keys), 1 << 23, np.uint32)  # 1000 x 2^23 > 2^32
    with pytest.raises(gf.FilterError):
        G.insert_counts(dev_u64(keys), dev_u32(cs))
    assert np.array_equal(G.export(), before)
    T = gf.TCF(12, 16, gf.MODE_BULK, max_batch=16)
    with pytest.raises(gf.FilterError):
        T.insert_counts(dev_u64(keys[:10]), dev_u32(np.ones(10, np.uint32)))
    # one key with the largest count a batch may carry
    G.insert_counts(dev_u64(keys[:1]), dev_u32(np.array([(1 << 32) - 1], np.uint32)))
    O = oracle.GQF(12, 8, seed=1)
    O.insert(keys[:500])
    O.insert_counts(keys[:1], np.array([(1 << 32) - 1], np.uint32))
    assert first_diff(G.export(), O.export()) is None
