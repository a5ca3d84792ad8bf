"""GPU checks of the serving loop: a stream of batches for many filters, run
concurrently on several worker streams, gives every batch exactly the results
of the same per-filter sequence run alone, and the served filters end up
byte-identical to the oracle's."""
import time

import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, first_diff

pytestmark = pytest.mark.gpu

OPS = {0: 0, 1: 1, 2: 2}  # workload op -> FILTER_OP_INSERT / QUERY / REMOVE


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def make_filters(gf, w, lg):
    nt = w["n_tcf"]
    mb = max(max(len(b) for b in w["prefill"]), max(len(k) for _, _, k in w["requests"]))
    fs = []
    for i in range(w["n_filters"]):
        f = gf.TCF(lg, 16, gf.MODE_BULK, seed=100 + i, max_batch=mb) if i < nt else gf.GQF(lg, 8, seed=100 + i,
                                                                                         max_batch=mb)
        f.insert(dev_u64(w["prefill"][i]))
        fs.append(f)
    return fs, mb


def run_alone(gf, fs, reqs):
    import torch

    out = []
    for f, op, keys in reqs:
        d = dev_u64(keys)
        r = torch.zeros(len(keys), dtype=torch.uint8, device="cuda")
        if op == 0:
            fs[f].insert(d, r)
        elif op == 1:
            fs[f].query(d, r)
        else:
            fs[f].remove(d, r)
        out.append(r.cpu().numpy())
    return out


@pytest.mark.parametrize("workers", [1, 3])
def test_served_batches_equal_alone(gf, oracle, workers):
    lg = 14
    w = W.serving_workload(n_filters=8, log2_slots=lg, bmin=6, bmax=12)
    reqs = w["requests"]
    fs, mb = make_filters(gf, w, lg)
    S = gf.FilterServer(fs, workers=workers, max_keys=mb)
    tickets = [S.submit(f, OPS[op], keys) for f, op, keys in reqs]
    served = [S.wait(t) for t in tickets]
    S.close()
    ref_fs, _ = make_filters(gf, w, lg)
    alone = run_alone(gf, ref_fs, reqs)
    for j, ((out, lat), ref) in enumerate(zip(served, alone)):
        assert np.array_equal(out, ref), j
        assert lat > 0
    for a, b in zip(fs, ref_fs):
        assert first_diff(a.export(), b.export()) is None
    # two of the served filters against the oracle
    for i in (0, w["n_tcf"]):
        O = oracle.TCF(lg, 16, seed=100 + i) if i < w["n_tcf"] else oracle.GQF(lg, 8, seed=100 + i)
        O.insert(w["prefill"][i])
        for f, op, keys in reqs:
            if f == i and op != 1:  # queries leave the table as it is
                (O.insert if op == 0 else O.remove)(keys)
        assert first_diff(fs[i].export(), O.export()) is None, i


def test_server_paced_arrivals(gf):
    """Requests submitted at Poisson arrival times; latencies are positive and
    results still equal the per-filter sequence run alone."""
    lg = 13
    w = W.serving_workload(n_filters=4, log2_slots=lg, bmin=6, bmax=11, seed=9)
    reqs = w["requests"][:60]
    fs, mb = make_filters(gf, w, lg)
    S = gf.FilterServer(fs, workers=2, max_keys=mb)
    arr = W.poisson_arrivals(29, len(reqs), rate=2000.0)
    t0 = time.perf_counter()
    tickets = []
    for (f, op, keys), a in zip(reqs, arr):
        while time.perf_counter() - t0 < a:
            pass
        tickets.append(S.submit(f, OPS[op], keys))
    served = [S.wait(t) for t in tickets]
    S.close()
    ref_fs, _ = make_filters(gf, w, lg)
    alone = run_alone(gf, ref_fs, reqs)
    for (out, lat), ref in zip(served, alone):
        assert np.array_equal(out, ref)
        assert 0 < lat < 60


def test_server_rejects_oversized_batch(gf):
    w = W.serving_workload(n_filters=2, log2_slots=10, bmin=4, bmax=6)
    fs, mb = make_filters(gf, w, 10)
    S = gf.FilterServer(fs, workers=1, max_keys=64)
    with pytest.raises(gf.FilterError):
        S.submit(0, 0, np.arange(65, dtype=np.uint64))
    with pytest.raises(gf.FilterError):
        S.submit(5, 0, np.arange(4, dtype=np.uint64))  # no such filter
    S.close()


def test_merged_requests_equal_alone(gf):
    """Continuous batching merges the queries, counts and GQF removes queued
    behind each other on one filter into one device batch; every request's
    results still equal the same per-filter sequence run alone, and the
    filters end byte-identical."""
    import torch

    lg = 12
    keys = W.uniform_keys(77, 6000)

    def filters():
        fs = [gf.TCF(lg, 16, gf.MODE_BULK, seed=300 + i, max_batch=4096) for i in range(2)] + \
             [gf.GQF(lg, 8, seed=300 + i, max_batch=4096) for i in range(2, 4)]
        for i, f in enumerate(fs):
            f.insert(dev_u64(keys[i * 1000:(i + 1) * 1000]))
            if i >= 2:  # some repeated copies in the GQFs, so that removes can leave counts behind
                f.insert(dev_u64(keys[i * 1000:i * 1000 + 300]))
        return fs

    rng = np.random.default_rng(5)
    reqs = []
    for r in range(120):
        f = int(rng.integers(4))
        kind = rng.choice(["q", "q", "q", "r", "c", "i"])
        pool = keys[f * 1000:(f + 1) * 1000]
        k = np.concatenate([pool[rng.integers(0, 1000, 40)], W.uniform_keys(900 + r, 10)])
        if kind == "i":
            reqs.append((f, gf.OP_INSERT, W.uniform_keys(2000 + r, 30)))
        elif kind == "r" and f >= 2:
            reqs.append((f, gf.OP_REMOVE, pool[rng.integers(0, 1000, 25)]))
        elif kind == "c" and f >= 2:
            reqs.append((f, gf.OP_COUNT, k))
        else:
            reqs.append((f, gf.OP_QUERY, k))
    fs = filters()
    S = gf.FilterServer(fs, workers=1, max_keys=4096)
    tickets = [S.submit(f, op, k) for f, op, k in reqs]
    served = [S.wait(t)[0] for t in tickets]
    st = S.stats()
    S.close()
    assert st["requests"] == len(reqs) and st["merged_requests"] > 0 and st["batches"] < len(reqs)
    ref = filters()
    for j, (f, op, k) in enumerate(reqs):
        d = dev_u64(k)
        if op == gf.OP_COUNT:
            out = torch.zeros(len(k), dtype=torch.int64, device="cuda")
            ref[f].count(d, out)
            want = out.cpu().numpy().view(np.uint64)
        else:
            out = torch.zeros(len(k), dtype=torch.uint8, device="cuda")
            {gf.OP_INSERT: ref[f].insert, gf.OP_QUERY: ref[f].query, gf.OP_REMOVE: ref[f].remove}[op](d, out)
            want = out.cpu().numpy()
        assert np.array_equal(served[j], want), (j, op)
    for a, b in zip(fs, ref):
        assert first_diff(a.export(), b.export()) is None
