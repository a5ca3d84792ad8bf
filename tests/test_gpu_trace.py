"""GPU tests of the kernel trace's work units: the launches whose work is only
known on the device (sparse TCF phases, the GQF merge) count it there, and the
counts equal what the oracle says the call did."""
import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def traced(gf, fn):
    import torch

    torch.cuda.synchronize()
    gf.trace_reset()
    gf.trace_enable(True)
    try:
        fn()
        torch.cuda.synchronize()
        return gf.trace_summary()
    finally:
        gf.trace_enable(False)


def test_tcf_phase_units_match_the_oracle(gf, oracle):
    """Dense phase A: one unit per block with candidates = the distinct b1 of
    the batch. Sparse phases: one histogram unit per candidate, i.e. per key
    that reached phase B, C or D (phase codes from the oracle's trace)."""
    q = 14
    pre = W.uniform_keys(71, int(0.7 * (1 << q)))
    batch = W.uniform_keys(72, int(0.2 * (1 << q)))
    O = oracle.TCF(q, 16, seed=9)
    T = gf.TCF(q, 16, gf.MODE_BULK, seed=9, max_batch=len(pre))
    O.insert(pre)
    T.insert(dev_u64(pre))
    b1, _, _ = O.keyinfo(batch)
    st_o, ph, _ = O.insert(batch, trace=True)
    st = zeros_u8(len(batch))
    tr = traced(gf, lambda: T.insert(dev_u64(batch), st))
    assert tr["tcf_group_hist"]["units"] == len(batch)
    assert tr["tcf_block_insert"]["units"] == len(np.unique(b1))
    reached = int((ph >= 1).sum() + (ph >= 2).sum() + (ph >= 3).sum())
    assert reached > 0, "the batch should spill past phase A at this load"
    assert tr["tcf_group_hist_sparse"]["units"] == reached
    assert tr["tcf_group_scatter_sparse"]["units"] == reached
    assert np.array_equal(T.export(), O.export())


def test_gqf_merge_counts_its_algorithmic_bytes(gf, oracle):
    """Merge units are bytes: (r / 4 + 1) per slot for the old table read and
    the new one written, plus 12 per group of the batch."""
    q, r = 14, 8
    keys = W.zipf_keys(73, 6000, 1.0, 1 << 16)
    O = oracle.GQF(q, r, seed=4)
    G = gf.GQF(q, r, seed=4, max_batch=len(keys))
    tr = traced(gf, lambda: G.insert(dev_u64(keys)))
    O.insert(keys)
    groups = len(O.groups()[0])
    nslots = G.stats()["nslots"]
    assert tr["gqf_merge_kernel"]["launches"] == 1
    assert tr["gqf_merge_kernel"]["units"] == nslots * (r // 4 + 1) + 12 * groups
