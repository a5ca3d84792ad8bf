"""GPU checks of the batched work list (filter_batch_run): a list of
(group, member, operation, keys) items over a TCF group and a GQF group gives
each member exactly what a standalone filter gives for its keys (a member's
items of one class concatenated in list order, inserts before removes before
queries and counts); a sequence of runs captured in one CUDA graph replays to
the same results; a GQF member whose insert does not fit keeps its table and
reports FULL for its keys."""
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


LOGS_T = [10, 11, 12, 10, 11, 12]
LOGS_G = [10, 12, 11, 10, 12, 11]


def groups(gf, max_total=1 << 16):
    T = gf.FilterGroup(gf.FILTER_TCF, LOGS_T, 16, [11 + m for m in range(6)], max_total=max_total)
    G = gf.FilterGroup(gf.FILTER_GQF, LOGS_G, 8, [21 + m for m in range(6)], max_total=max_total)
    return T, G


def member_keys(seed, lg, load):
    n = int(load * (1 << lg))
    k = W.uniform_keys(seed, n)
    return k[: n // 3], k[n // 3:]  # two insert items per member


def test_batch_run_equals_standalone_filters(gf, oracle):
    T, G = groups(gf)
    B = gf.FilterBatch(T, G, max_keys=1 << 16, max_items=256)
    items, keep, ref = [], [], {}
    for g, logs, kind in ((gf.BATCH_TCF, LOGS_T, "t"), (gf.BATCH_GQF, LOGS_G, "g")):
        for m, lg in enumerate(logs):
            a, b = member_keys(700 + 10 * g + m, lg, 0.8)
            st_a, st_b = zeros_u8(len(a)), zeros_u8(len(b))
            da, db = dev_u64(a), dev_u64(b)
            # list order interleaves the members; a member's two inserts stay in order
            items.append((g, m, gf.OP_INSERT, da, st_a))
            keep.append((g, m, a, b, da, db, st_a, st_b))
    for g, m, a, b, da, db, st_a, st_b in keep:
        items.append((g, m, gf.OP_INSERT, db, st_b))
    probes = {}
    for g, m, a, b, *_ in keep:
        p = np.concatenate([a[::3], b[::5], W.uniform_keys(900 + 10 * g + m, 300)])
        dp = dev_u64(p)
        fq = zeros_u8(len(p))
        items.append((g, m, gf.OP_QUERY, dp, fq))
        cq = None
        if g == gf.BATCH_GQF:
            cq = zeros_u64(len(p))
            items.append((g, m, gf.OP_COUNT, dp, cq))
        probes[(g, m)] = (p, dp, fq, cq)
    B.run(items)
    for g, m, a, b, da, db, st_a, st_b in keep:
        lg = (LOGS_T if g == gf.BATCH_TCF else LOGS_G)[m]
        seed = (11 if g == gf.BATCH_TCF else 21) + m
        O = oracle.TCF(lg, 16, seed=seed) if g == gf.BATCH_TCF else oracle.GQF(lg, 8, seed=seed)
        st = O.insert(np.concatenate([a, b]))
        got_img = (T if g == gf.BATCH_TCF else G).export(m)
        d = first_diff(got_img, O.export())
        assert d is None, (g, m, d)
        assert np.array_equal(np.concatenate([host(st_a), host(st_b)]), st), (g, m)
        p, dp, fq, cq = probes[(g, m)]
        if g == gf.BATCH_TCF:
            assert np.array_equal(host(fq), O.query(p))
        else:
            c = O.count(p)
            assert np.array_equal(host(cq), c)
            assert np.array_equal(host(fq), (c > 0).astype(np.uint8))
    # removes: one item per member, statuses and images against the oracle
    items, rem = [], []
    for g, m, a, b, *_ in keep:
        r = np.concatenate([a[::2], W.uniform_keys(950 + 10 * g + m, 40)])
        sr = zeros_u8(len(r))
        items.append((g, m, gf.OP_REMOVE, dev_u64(r), sr))
        rem.append((g, m, a, b, r, sr))
    B.run(items)
    for g, m, a, b, r, sr in rem:
        lg = (LOGS_T if g == gf.BATCH_TCF else LOGS_G)[m]
        seed = (11 if g == gf.BATCH_TCF else 21) + m
        O = oracle.TCF(lg, 16, seed=seed) if g == gf.BATCH_TCF else oracle.GQF(lg, 8, seed=seed)
        O.insert(np.concatenate([a, b]))
        st = O.remove(r)
        d = first_diff((T if g == gf.BATCH_TCF else G).export(m), O.export())
        assert d is None, (g, m, d)
        assert np.array_equal(host(sr), st), (g, m)
    B.close()


def test_batch_runs_captured_in_a_cuda_graph(gf):
    """Clear both groups, insert, query: captured once, replayed twice, the
    answers and the tables equal those of the same calls run directly."""
    import torch

    T, G = groups(gf)
    B = gf.FilterBatch(T, G, max_keys=1 << 16, max_items=64)
    ins, qry = [], []
    outs = []
    for g, logs in ((gf.BATCH_TCF, LOGS_T), (gf.BATCH_GQF, LOGS_G)):
        for m, lg in enumerate(logs):
            a, b = member_keys(1700 + 10 * g + m, lg, 0.85)
            k = dev_u64(np.concatenate([a, b]))
            p = dev_u64(np.concatenate([a[::4], W.uniform_keys(1900 + 10 * g + m, 200)]))
            f = torch.zeros(p.numel(), dtype=torch.uint8, device="cuda")
            ins.append((g, m, gf.OP_INSERT, k, None))
            qry.append((g, m, gf.OP_QUERY, p, f))
            outs.append(f)

    def step():
        T.clear()
        G.clear()
        B.run(ins)
        B.run(qry)

    step()
    torch.cuda.synchronize()
    want = [o.clone() for o in outs]
    imgs = [T.export(m) for m in range(6)] + [G.export(m) for m in range(6)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        for o in outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for o, w in zip(outs, want):
            assert torch.equal(o, w)
        got = [T.export(m) for m in range(6)] + [G.export(m) for m in range(6)]
        for x, y in zip(got, imgs):
            assert first_diff(x, y) is None
    del graph
    B.close()


def test_many_calls_without_synchronising(gf, oracle):
    """Forty calls enqueued back to back (the host builds each call's
    descriptors while the earlier calls are still queued), each inserting one
    chunk into a changing subset of members, then a graph of a query call
    replayed between direct calls: every member's table equals the oracle's
    after the same batches."""
    import torch

    T, G = groups(gf)
    B = gf.FilterBatch(T, G, max_keys=1 << 16, max_items=64)
    calls = 40
    chunks = {}
    for g, logs in ((gf.BATCH_TCF, LOGS_T), (gf.BATCH_GQF, LOGS_G)):
        for m, lg in enumerate(logs):
            k = W.uniform_keys(2300 + 10 * g + m, int(0.8 * (1 << lg)))
            chunks[(g, m)] = np.array_split(k, calls)
    plan = []  # per call, the (g, m) that take their next chunk
    for j in range(calls):
        plan.append([(g, m) for (g, m) in chunks if (j + 3 * m + g) % 4 != 0 or j == calls - 1])
    taken = {gm: [] for gm in chunks}
    keep = []
    for j, who in enumerate(plan):
        items = []
        for g, m in reversed(who) if j % 2 else who:
            c = chunks[(g, m)][len(taken[(g, m)])]
            d = dev_u64(c)
            keep.append(d)
            taken[(g, m)].append(c)
            items.append((g, m, gf.OP_INSERT, d, None))
        B.run(items)
    probe = {gm: dev_u64(np.concatenate(chunks[gm][:5] + [W.uniform_keys(2500 + gm[0] * 10 + gm[1], 100)]))
             for gm in chunks}
    found = {gm: torch.zeros(probe[gm].numel(), dtype=torch.uint8, device="cuda") for gm in chunks}
    qitems = [(g, m, gf.OP_QUERY, probe[(g, m)], found[(g, m)]) for (g, m) in chunks]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.run(qitems)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.run(qitems)
    for o in found.values():
        o.zero_()
    B.run([(gf.BATCH_TCF, 0, gf.OP_QUERY, probe[(0, 0)], found[(0, 0)])])  # a direct call in between
    graph.replay()
    torch.cuda.synchronize()
    for (g, m), cs in taken.items():
        lg = (LOGS_T if g == gf.BATCH_TCF else LOGS_G)[m]
        seed = (11 if g == gf.BATCH_TCF else 21) + m
        O = oracle.TCF(lg, 16, seed=seed) if g == gf.BATCH_TCF else oracle.GQF(lg, 8, seed=seed)
        for c in cs:
            O.insert(c)
        d = first_diff((T if g == gf.BATCH_TCF else G).export(m), O.export())
        assert d is None, (g, m, d)
        p = host(probe[(g, m)])
        want = O.query(p) if g == gf.BATCH_TCF else (O.count(p) > 0).astype(np.uint8)
        assert np.array_equal(host(found[(g, m)]), want), (g, m)
    del graph
    B.close()


def test_gqf_member_that_does_not_fit_keeps_its_table(gf, oracle):
    T, G = groups(gf)
    B = gf.FilterBatch(None, G, max_keys=1 << 16, max_items=16)
    small = W.uniform_keys(2100, 500)
    B.run([(gf.BATCH_GQF, 0, gf.OP_INSERT, dev_u64(small), None)])
    before = G.export(0)
    too_many = W.uniform_keys(2101, 4 << LOGS_G[0])  # four times the home slots
    st = zeros_u8(len(too_many))
    other = W.uniform_keys(2102, 1000)
    st2 = zeros_u8(len(other))
    B.run([(gf.BATCH_GQF, 0, gf.OP_INSERT, dev_u64(too_many), st),
           (gf.BATCH_GQF, 1, gf.OP_INSERT, dev_u64(other), st2)])
    assert first_diff(G.export(0), before) is None
    assert (host(st) == gf.KEY_FULL).all()
    assert not host(st2).any()
    O = oracle.GQF(LOGS_G[1], 8, seed=22)
    O.insert(other)
    assert first_diff(G.export(1), O.export()) is None
    assert G.stats(0)["failed_keys"] == len(too_many)
    B.close()
