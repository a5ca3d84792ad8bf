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
