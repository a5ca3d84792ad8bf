"""GPU parity for the GQF point updates of the C ABI (paper Sec. 5.2, the
point insertion API: one thread per key, locks on two consecutive regions of
8192 quotients). A GQF's table is a function of its fingerprint multiset, so
after point inserts, in whatever order the threads ran, the image equals the
oracle's after a bulk insert of the same keys; after point removes, the
per-fingerprint statuses and the image equal the oracle's."""
import collections

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


def keys_at_load(seed, q):
    n = int(0.68 * (1 << q))  # with the repeats (3 slots each): 85 % of the home slots
    base = W.uniform_keys(seed, n * 3 // 4)
    keys = np.concatenate([base, base[: n // 4]])
    return base, keys[W.sample_without_replacement(seed + 1, keys.size, keys.size)]


@pytest.mark.parametrize("q,r", [(18, 8), (16, 16), (12, 8)])
def test_point_updates_equal_the_oracle(gf, oracle, q, r):
    base, keys = keys_at_load(6100 + q, q)
    G = gf.GQF(q, r, seed=q * r, max_batch=keys.size)
    st = zeros_u8(keys.size)
    G.point_update(dev_u64(keys), status=st)
    assert not host(st).any(), np.unique(host(st), return_counts=True)
    O = oracle.GQF(q, r, seed=q * r)
    O.insert(keys)
    assert first_diff(G.export(), O.export()) is None
    probe = np.concatenate([base[::7], W.uniform_keys(6200 + q, 2000)])
    c = zeros_u64(probe.size)
    G.count(dev_u64(probe), c)
    assert np.array_equal(host(c), O.count(probe))
    rem = np.concatenate([base[::2], base[: keys.size // 16], W.uniform_keys(6300 + q, 400)])
    st = zeros_u8(rem.size)
    G.point_update(dev_u64(rem), remove=True, status=st)
    fp = O.fingerprints(rem)
    want = O.remove(rem)
    assert collections.Counter(zip(fp.tolist(), host(st).tolist())) == collections.Counter(zip(fp.tolist(), want.tolist()))
    assert first_diff(G.export(), O.export()) is None
    assert G.stats()["status_word"] == 0


def test_point_and_bulk_calls_mix(gf, oracle):
    """Bulk insert, point inserts, bulk remove, point removes on one filter:
    every stage leaves the oracle's table."""
    q, r = 16, 8
    a = W.uniform_keys(6400, 20000)
    b = W.uniform_keys(6401, 15000)
    G = gf.GQF(q, r, seed=5, max_batch=40000)
    O = oracle.GQF(q, r, seed=5)
    G.insert(dev_u64(a)); O.insert(a)
    G.point_update(dev_u64(b)); O.insert(b)
    assert first_diff(G.export(), O.export()) is None
    G.remove(dev_u64(a[::3])); O.remove(a[::3])
    G.point_update(dev_u64(b[::2]), remove=True); O.remove(b[::2])
    assert first_diff(G.export(), O.export()) is None
    G.insert(dev_u64(b[:100])); O.insert(b[:100])  # a bulk call after point updates
    assert first_diff(G.export(), O.export()) is None


def test_point_updates_in_a_cuda_graph(gf, oracle):
    import torch

    q, r = 14, 8
    keys = W.uniform_keys(6500, 9000)
    G = gf.GQF(q, r, seed=7, max_batch=keys.size)
    dk = dev_u64(keys)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        G.clear()
        G.point_update(dk)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        G.clear()
        G.point_update(dk)
    O = oracle.GQF(q, r, seed=7)
    O.insert(keys)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert first_diff(G.export(), O.export()) is None
    del graph


def test_point_update_refused_for_a_tcf(gf):
    T = gf.TCF(12, 16, gf.MODE_POINT, seed=1)
    with pytest.raises(gf.FilterError):
        T.point_update(dev_u64(W.uniform_keys(1, 10)))
