"""GPU parity for the TCF block geometries other than one 32-byte sector
(paper Sec. 4.1 block sizes up to and past a cache line, Sec. 4.2 128-slot
bulk blocks, Sec. 4 12-bit tags): the packed-block kernels leave the oracle's
table image byte for byte after every insert and remove batch, with the
oracle's statuses, and answer queries as the oracle does. The filter of
2^log2_slots slots has nb = the largest power of two with nb * B <=
2^log2_slots blocks, which is the oracle's geometry with log2_blocks."""
import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, host, first_diff

pytestmark = pytest.mark.gpu

GEOMS = [(16, 8), (16, 32), (16, 64), (16, 128), (12, 21), (8, 64)]


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def log2_blocks(log2_slots, B):
    lb = 0
    while (1 << lb) < B:
        lb += 1
    return log2_slots - lb


def run(gf, oracle, lg, f, B, seed, load=0.9, batches=5):
    nb_log = log2_blocks(lg, B)
    O = oracle.TCF(0, f, seed=seed, block_slots=B, log2_blocks=nb_log)
    nslots = (1 << nb_log) * B
    n = int(load * nslots)
    keys = W.uniform_keys(seed, n)
    cuts = np.linspace(0, n, batches + 1).astype(int)
    ins = [np.concatenate([keys[a:b], keys[a:a + (b - a) // 6]]) for a, b in zip(cuts, cuts[1:])]  # duplicates
    dels = [keys[: n // 3], np.concatenate([keys[n // 3: n // 2], W.uniform_keys(seed + 1, 500)])]
    G = gf.TCF(lg, f, gf.MODE_BULK, seed=seed, max_batch=max(map(len, ins + dels)), block_slots=B)
    assert G.stats()["nslots"] == nslots
    for k, b in enumerate(ins):
        want = O.insert(b)
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        assert np.array_equal(host(st), want), ("insert", k)
        d = first_diff(G.export(), O.export())
        assert d is None, ("insert", k, d)
    probe = np.concatenate([keys[::3], W.uniform_keys(seed + 2, 20000)])
    found = zeros_u8(len(probe))
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))
    for k, b in enumerate(dels):
        want = O.remove(b)
        st = zeros_u8(len(b))
        G.remove(dev_u64(b), st)
        assert np.array_equal(host(st), want), ("remove", k)
        d = first_diff(G.export(), O.export())
        assert d is None, ("remove", k, d)
    G.query(dev_u64(probe), found)
    assert np.array_equal(host(found), O.query(probe))
    return O, G


@pytest.mark.parametrize("f,B", GEOMS)
def test_packed_geometry_image_and_answers(gf, oracle, f, B):
    run(gf, oracle, 16, f, B, seed=40 + f + B)


@pytest.mark.parametrize("f,B", [(16, 128), (12, 21)])
def test_packed_geometry_overfull_uses_backing_and_reports_full(gf, oracle, f, B):
    """Past 100 % load the backing buckets fill and the rest is FULL, as in
    the oracle (the statuses and images are compared inside run)."""
    O, G = run(gf, oracle, 12, f, B, seed=77 + B, load=1.08, batches=3)
    assert O.backing_count() > 0


@pytest.mark.parametrize("f,B", [(16, 64), (12, 21)])
def test_packed_geometry_several_tiles_large(gf, oracle, f, B):
    """2^22 slots: many CTAs per phase, sparse and dense phases alike."""
    run(gf, oracle, 22, f, B, seed=91 + B, batches=4)


def test_packed_geometry_empty_and_tiny_batches(gf, oracle):
    f, B = 16, 128
    lg = 10
    O = oracle.TCF(0, f, seed=5, block_slots=B, log2_blocks=log2_blocks(lg, B))
    G = gf.TCF(lg, f, gf.MODE_BULK, seed=5, max_batch=64, block_slots=B)
    empty = dev_u64(np.zeros(0, dtype=np.uint64))
    G.insert(empty)
    G.remove(empty)
    for b in (W.uniform_keys(6, 1), W.uniform_keys(7, 3), W.uniform_keys(6, 1)):
        want = O.insert(b)
        st = zeros_u8(len(b))
        G.insert(dev_u64(b), st)
        assert np.array_equal(host(st), want)
    assert first_diff(G.export(), O.export()) is None


def test_packed_geometry_refuses_unsupported_calls(gf):
    G = gf.TCF(14, 16, gf.MODE_BULK, seed=1, block_slots=64)
    with pytest.raises(gf.FilterError):
        G.device_view()
