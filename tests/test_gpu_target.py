"""Parity at the target size: 2^28 slots at 90 % load, both filters.

TCF: 2^28 slots, 16-bit tags, bulk mode; floor(0.9 * 2^28) = 241,591,910
uniform keys in 2^24-key batches; 2^24 positive and 2^24 negative queries;
a random half deleted in 2^24-key batches; the probes queried again. The
image after the inserts and after the deletes, every status and every
answer equal the incremental oracle's (run batch by batch in a spawned
process, compared through per-MiB digests of the images).

GQF: 2^28 home slots, 8-bit remainders; the same number of uniform keys in
one batch (90 % load); counts of 2^24 inserted and 2^24 fresh keys; 2^24
distinct inserted keys deleted; counts again. Images equal the oracle's
canonical builder on the brute-force fingerprint multiset before and after
the delete, and every count equals the fingerprint's multiplicity."""
import numpy as np
import pytest

import target_oracle as TO
from gpu_util import dev_u64, zeros_u8, zeros_u64, host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    TO.start()
    return gf


def test_tcf_2_28_slots_90_percent(gf):
    import torch

    ins, probe, dels = TO.tcf_inputs()
    B = TO.TCF_BATCH
    T = gf.TCF(TO.TCF_LOG2, 16, gf.MODE_BULK, seed=TO.TCF_SEED, max_batch=B)
    d_ins = dev_u64(ins)
    st = zeros_u8(len(ins))
    for i in range(0, len(ins), B):
        T.insert(d_ins[i:i + B], st[i:i + B])
    st_ins = host(st)
    img_ins = TO.digests(T.export())
    d_probe = dev_u64(probe)
    q1 = zeros_u8(len(probe))
    T.query(d_probe, q1)
    backing = T.stats()["backing_used"]
    d_del = dev_u64(dels)
    sd = zeros_u8(len(dels))
    for i in range(0, len(dels), B):
        T.remove(d_del[i:i + B], sd[i:i + B])
    st_del = host(sd)
    img_del = TO.digests(T.export())
    q2 = zeros_u8(len(probe))
    T.query(d_probe, q2)
    q1, q2 = host(q1), host(q2)
    del T, d_ins, d_del, d_probe
    torch.cuda.empty_cache()

    exp = TO.result("tcf")
    assert int(np.count_nonzero(st_ins)) == exp["ins_failed"]
    assert TO.digests(st_ins) == exp["ins_status_digest"]
    d = TO.first_chunk_diff(img_ins, exp["img_ins"])
    assert d is None, f"image after the inserts: {d}"
    assert backing == exp["backing"]
    assert np.array_equal(q1, exp["q1"])
    assert q1[: len(probe) // 2].all()  # no false negatives
    assert TO.digests(st_del) == exp["del_status_digest"]
    d = TO.first_chunk_diff(img_del, exp["img_del"])
    assert d is None, f"image after the deletes: {d}"
    assert np.array_equal(q2, exp["q2"])


def test_gqf_2_28_slots_90_percent(gf):
    import torch

    ins, probe, dels = TO.gqf_inputs()
    G = gf.GQF(TO.GQF_Q, 8, seed=TO.GQF_SEED, max_batch=len(ins))
    st = zeros_u8(len(ins))
    G.insert(dev_u64(ins), st)
    st_ins = host(st)
    img_ins = TO.digests(G.export())
    d_probe = dev_u64(probe)
    c1 = zeros_u64(len(probe))
    G.count(d_probe, c1)
    sd = zeros_u8(len(dels))
    G.remove(dev_u64(dels), sd)
    st_del = host(sd)
    img_del = TO.digests(G.export())
    c2 = zeros_u64(len(probe))
    G.count(d_probe, c2)
    c1, c2 = host(c1), host(c2)
    del G, d_probe, st
    torch.cuda.empty_cache()

    exp = TO.result("gqf")
    assert not st_ins.any(), "an insert at 90 % load reported FULL"
    d = TO.first_chunk_diff(img_ins, exp["img_ins"])
    assert d is None, f"image after the insert: {d}"
    assert np.array_equal(c1, exp["c1"])
    assert not st_del.any(), "a delete of an inserted key reported NOT_FOUND"
    d = TO.first_chunk_diff(img_del, exp["img_del"])
    assert d is None, f"image after the delete: {d}"
    assert np.array_equal(c2, exp["c2"])
