"""The allocation-free GQF insert (filter_gqf_insert_noalloc), for callers that
must not call cudaMalloc: its table images must equal those of the regular
filter_insert, call after call, through the C ABI."""
import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q,r", [(12, 8), (16, 16)])
def test_noalloc_insert_matches_filter_insert(q, r):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    seed = 7
    G = gf.GQF(q, r, seed=seed, max_batch=gf.NOALLOC_MAX_KEYS)
    size = G.export().size
    a = torch.zeros(size, dtype=torch.uint8, device="cuda")  # empty table image
    b = torch.zeros(size, dtype=torch.uint8, device="cuda")
    keys = W.uniform_keys(900 + q, 3 * (1 << q) // 5)
    batches = [np.concatenate([keys[: len(keys) // 2], keys[:100]]), keys[len(keys) // 2:]]
    for k, batch in enumerate(batches):  # two calls in a row, each from the previous image
        st_ref = zeros_u8(len(batch))
        G.insert(dev_u64(batch), st_ref)
        st = zeros_u8(len(batch))
        gf.gqf_insert_noalloc(q, r, seed, a, b, dev_u64(batch), st)
        assert np.array_equal(host(b), G.export()), f"image differs after call {k}"
        assert np.array_equal(host(st), host(st_ref))
        a, b = b, a


def test_noalloc_rejects_oversize_arguments():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    a = torch.zeros(64, dtype=torch.uint8, device="cuda")
    big = torch.zeros(gf.NOALLOC_MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(gf.FilterError):
        gf.gqf_insert_noalloc(12, 8, 0, a, a.clone(), big)
    with pytest.raises(gf.FilterError):
        gf.gqf_insert_noalloc(gf.NOALLOC_MAX_Q + 1, 8, 0, a, a.clone(), big[:10])


def _pair(q, r, seed):
    import torch

    import paper_2212_09005_gb300 as gf

    G = gf.GQF(q, r, seed=seed, max_batch=gf.NOALLOC_MAX_KEYS)
    size = G.export().size
    return G, torch.zeros(size, dtype=torch.uint8, device="cuda"), torch.zeros(size, dtype=torch.uint8, device="cuda")


def test_noalloc_at_its_limits():
    """q = 20 with the largest batch (the sizes that fill most of the static
    scratch), then an empty batch, which copies the image unchanged."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    q, r, seed = gf.NOALLOC_MAX_Q, 8, 31
    G, a, b = _pair(q, r, seed)
    keys = W.uniform_keys(931, gf.NOALLOC_MAX_KEYS)
    st_ref, st = zeros_u8(len(keys)), zeros_u8(len(keys))
    G.insert(dev_u64(keys), st_ref)
    gf.gqf_insert_noalloc(q, r, seed, a, b, dev_u64(keys), st)
    assert np.array_equal(host(b), G.export())
    assert np.array_equal(host(st), host(st_ref))
    a.fill_(0xAB)
    gf.gqf_insert_noalloc(q, r, seed, b, a, dev_u64(np.zeros(0, np.uint64)))
    assert np.array_equal(host(a), G.export())


def test_noalloc_overflow_keeps_prefix_and_leaves_input_unchanged():
    """A batch that does not fit: the longest prefix of its sorted groups is
    kept, as filter_insert keeps it, statuses agree, and the input image is
    byte for byte what it was (it is only read)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    q, r, seed = 10, 8, 32
    G, a, b = _pair(q, r, seed)
    first = W.uniform_keys(932, 900)
    G.insert(dev_u64(first))
    gf.gqf_insert_noalloc(q, r, seed, a, b, dev_u64(first))
    assert np.array_equal(host(b), G.export())
    before = host(b).copy()
    over = W.uniform_keys(933, 4000)  # 2048 slots in all: does not fit
    st_ref, st = zeros_u8(len(over)), zeros_u8(len(over))
    G.insert(dev_u64(over), st_ref)
    gf.gqf_insert_noalloc(q, r, seed, b, a, dev_u64(over), st)
    assert (host(st_ref) == gf.KEY_FULL).any() and (host(st_ref) == gf.KEY_OK).any()
    assert np.array_equal(host(a), G.export())
    assert np.array_equal(host(st), host(st_ref))
    assert np.array_equal(host(b), before), "the input image was written"
