"""GPU parity for filter groups: many filters driven by one set of launches per
call. Every member must end up byte-identical to a standalone oracle filter
of its configuration that received the same keys in the same order, and its
per-key answers must equal that oracle's."""
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


def call_arrays(keys, spans):
    """Keys of one group call: member i gets keys[spans[i, 0]:spans[i, 1]]."""
    spans = np.asarray(spans, dtype=np.int64)
    lens = spans[:, 1] - spans[:, 0]
    off = np.zeros(len(spans) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    parts = [keys[s:e] for s, e in spans]
    k = np.concatenate(parts) if parts else np.zeros(0, np.uint64)
    return off, k.astype(np.uint64)


def dev_off(off):
    import torch

    return torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()


def check_images(G, oracles, members=None):
    for m in (range(len(oracles)) if members is None else members):
        d = first_diff(G.export(m), oracles[m].export())
        assert d is None, (m, d)


def run_tcf_group(gf, oracle, logs, seeds, keys, off, rounds, f=16, check_rounds=True, max_total=0):
    n = len(logs)
    chunks = W.round_chunks(off, rounds)
    mt = max(int((chunks[j, :, 1] - chunks[j, :, 0]).sum()) for j in range(rounds))
    G = gf.FilterGroup(gf.FILTER_TCF, logs, f, seeds, max_total=max(1, mt, max_total))
    O = [oracle.TCF(int(logs[m]), f, seed=int(seeds[m])) for m in range(n)]
    for j in range(rounds):
        o, k = call_arrays(keys, chunks[j])
        st = zeros_u8(len(k))
        G.insert(dev_off(o), dev_u64(k), st)
        st = host(st)
        for m in range(n):
            st_o = O[m].insert(k[o[m]:o[m + 1]])
            assert np.array_equal(st[o[m]:o[m + 1]], st_o), (j, m)
        if check_rounds or j == rounds - 1:
            check_images(G, O)
    return G, O


@pytest.mark.parametrize("f", [16, 8])
def test_tcf_group_insert_query_remove(gf, oracle, f):
    w = W.batched_workload(n_filters=40, seed=41, emin=10, emax=13, tcf_rounds=3)
    logs = w["log2_slots"] + (1 if f == 8 else 0)  # 8-bit tags: 32-slot blocks
    seeds = w["hash_seeds"]
    keys, off = w["insert"], w["offsets"]
    G, O = run_tcf_group(gf, oracle, logs, seeds, keys, off, rounds=3, f=f, max_total=len(keys))
    n = len(logs)
    # queries: each member's own keys, then as many fresh keys
    qo, qk = [0], []
    for m in range(n):
        qk += [keys[off[m]:off[m + 1]], w["negatives"][off[m]:off[m + 1]]]
        qo.append(qo[-1] + 2 * int(off[m + 1] - off[m]))
    qo = np.array(qo, np.int64)
    qk = np.concatenate(qk)
    found = zeros_u8(len(qk))
    G.query(dev_off(qo), dev_u64(qk), found)
    found = host(found)
    for m in range(n):
        assert np.array_equal(found[qo[m]:qo[m + 1]], O[m].query(qk[qo[m]:qo[m + 1]])), m
    # remove every other key of every member, then compare images and re-query
    rk, ro = [], [0]
    for m in range(n):
        part = keys[off[m]:off[m + 1]][::2]
        rk.append(part)
        ro.append(ro[-1] + len(part))
    rk = np.concatenate(rk)
    ro = np.array(ro, np.int64)
    st = zeros_u8(len(rk))
    G.remove(dev_off(ro), dev_u64(rk), st)
    st = host(st)
    for m in range(n):
        assert np.array_equal(st[ro[m]:ro[m + 1]], O[m].remove(rk[ro[m]:ro[m + 1]])), m
    check_images(G, O)
    found = zeros_u8(len(qk))
    G.query(dev_off(qo), dev_u64(qk), found)
    found = host(found)
    for m in range(n):
        assert np.array_equal(found[qo[m]:qo[m + 1]], O[m].query(qk[qo[m]:qo[m + 1]])), m


def test_tcf_group_duplicates_empty_members_and_full(gf, oracle):
    """Repeated keys inside a member, members with no keys in a call, and
    members loaded past their capacity (keys rejected as FULL exactly where
    the oracle rejects them)."""
    logs = np.array([10, 11, 10, 12, 10, 10], np.int64)
    seeds = np.arange(6, dtype=np.uint64) * 77 + 5
    want = [0, 1900, 1200, 0, 1150, 40]  # member 2 and 4 past 100% of 1024 slots
    parts, off = [], [0]
    for m, c in enumerate(want):
        base = W.uniform_keys(900 + m, max(1, c))[:c]
        if c:
            base = np.concatenate([base[: c - c // 4], base[: c // 4]])  # a quarter repeated
        parts.append(base)
        off.append(off[-1] + len(base))
    keys = np.concatenate(parts).astype(np.uint64)
    off = np.array(off, np.int64)
    G, O = run_tcf_group(gf, oracle, logs, seeds, keys, off, rounds=2)
    st = [G.stats(m) for m in range(len(logs))]
    assert st[0]["failed_keys"] == st[-1]["failed_keys"]  # shared counters in a TCF group
    assert st[0]["failed_keys"] > 0


def test_gqf_group_insert_count_remove(gf, oracle):
    w = W.batched_workload(n_filters=40, seed=42, emin=10, emax=13)
    logs, seeds = w["log2_slots"], w["hash_seeds"]
    keys, off = w["insert"], w["offsets"]
    n = len(logs)
    # repeats: every member's first fifth again, so counts above 1 appear
    parts, o2 = [], [0]
    for m in range(n):
        k = keys[off[m]:off[m + 1]]
        k = np.concatenate([k, k[: len(k) // 5], k[:3], k[:3]])
        parts.append(k)
        o2.append(o2[-1] + len(k))
    ik = np.concatenate(parts)
    io = np.array(o2, np.int64)
    G = gf.FilterGroup(gf.FILTER_GQF, logs, 8, seeds, max_total=len(ik))
    O = [oracle.GQF(int(logs[m]), 8, seed=int(seeds[m])) for m in range(n)]
    st = zeros_u8(len(ik))
    G.insert(dev_off(io), dev_u64(ik), st)
    st = host(st)
    for m in range(n):
        assert np.array_equal(st[io[m]:io[m + 1]], O[m].insert(ik[io[m]:io[m + 1]])), m
    check_images(G, O)
    # counts of own keys and fresh keys
    qk, qo = [], [0]
    for m in range(n):
        q = np.concatenate([keys[off[m]:off[m + 1]], w["negatives"][off[m]:off[m + 1]]])
        qk.append(q)
        qo.append(qo[-1] + len(q))
    qk = np.concatenate(qk)
    qo = np.array(qo, np.int64)
    cnt = zeros_u64(len(qk))
    G.count(dev_off(qo), dev_u64(qk), cnt)
    cnt = host(cnt)
    found = zeros_u8(len(qk))
    G.query(dev_off(qo), dev_u64(qk), found)
    found = host(found)
    for m in range(n):
        c_o = O[m].count(qk[qo[m]:qo[m + 1]])
        assert np.array_equal(cnt[qo[m]:qo[m + 1]], c_o), m
        assert np.array_equal(found[qo[m]:qo[m + 1]], (c_o > 0).astype(np.uint8)), m
    # remove: a third of each member's keys, some of them twice, plus absent keys
    rk, ro = [], [0]
    for m in range(n):
        k = keys[off[m]:off[m + 1]]
        r = np.concatenate([k[::3], k[:2], w["negatives"][off[m]:off[m] + 5]])
        rk.append(r)
        ro.append(ro[-1] + len(r))
    rk = np.concatenate(rk)
    ro = np.array(ro, np.int64)
    st = zeros_u8(len(rk))
    G.remove(dev_off(ro), dev_u64(rk), st)
    st = host(st)
    for m in range(n):
        assert np.array_equal(st[ro[m]:ro[m + 1]], O[m].remove(rk[ro[m]:ro[m + 1]])), m
    check_images(G, O)


def test_gqf_group_overflowing_member(gf, oracle):
    """A member given far more keys than it can hold keeps the longest prefix
    of its sorted groups that fits, as a standalone filter does; the other
    members are unaffected."""
    logs = np.array([10, 8, 11, 8], np.int64)
    seeds = np.array([3, 4, 5, 6], np.uint64)
    want = [900, 2000, 1500, 100]
    parts, off = [], [0]
    for m, c in enumerate(want):
        parts.append(W.uniform_keys(1300 + m, c))
        off.append(off[-1] + c)
    keys = np.concatenate(parts)
    off = np.array(off, np.int64)
    G = gf.FilterGroup(gf.FILTER_GQF, logs, 8, seeds, max_total=len(keys))
    O = [oracle.GQF(int(logs[m]), 8, seed=int(seeds[m])) for m in range(len(logs))]
    st = zeros_u8(len(keys))
    G.insert(dev_off(off), dev_u64(keys), st)
    st = host(st)
    for m in range(len(logs)):
        st_o = O[m].insert(keys[off[m]:off[m + 1]])
        assert np.array_equal(st[off[m]:off[m + 1]], st_o), m
    assert (st[off[1]:off[2]] == 1).any()
    check_images(G, O)
    assert G.stats(1)["failed_keys"] > 0 and G.stats(0)["failed_keys"] == 0


def test_group_edge_cases(gf, oracle):
    """A call with no keys, a one-member group, and members without keys."""
    import torch

    G = gf.FilterGroup(gf.FILTER_GQF, [12], 8, [9], max_total=5000)
    O = oracle.GQF(12, 8, seed=9)
    G.insert(dev_off([0, 0]), torch.zeros(0, dtype=torch.int64, device="cuda"))
    k = W.uniform_keys(1400, 3000)
    G.insert(dev_off([0, 3000]), dev_u64(k))
    O.insert(k)
    assert first_diff(G.export(0), O.export()) is None
    T = gf.FilterGroup(gf.FILTER_TCF, [10, 12, 10], 16, [1, 2, 3], max_total=3000)
    OT = [oracle.TCF(lg, 16, seed=s) for lg, s in ((10, 1), (12, 2), (10, 3))]
    k = W.uniform_keys(1401, 3000)
    T.insert(dev_off([0, 0, 3000, 3000]), dev_u64(k))
    OT[1].insert(k)
    for m in range(3):
        assert first_diff(T.export(m), OT[m].export()) is None
    found = zeros_u8(3000)
    T.query(dev_off([0, 0, 3000, 3000]), dev_u64(k), found)
    assert host(found).all()
    with pytest.raises(gf.FilterError):
        T.count(dev_off([0, 0, 3000, 3000]), dev_u64(k), zeros_u64(3000))
    with pytest.raises(gf.FilterError):
        T.insert(dev_off([0, 0, 3001, 3001]), dev_u64(W.uniform_keys(1402, 3001)))  # above max_total


@pytest.mark.slow
def test_batched_workload_full_size_sampled(gf, oracle):
    """The 4096-filter workload at full size (2048 TCF-16 + 2048 GQF-8, 2^10..2^20
    slots each, 85-95% load): every member's answers are checked for the
    properties that hold at any size, and a sample of members, including the
    largest of each kind, is compared with the oracle byte for byte."""
    import torch

    w = W.batched_workload()
    off, keys, logs, seeds = w["offsets"], w["insert"], w["log2_slots"], w["hash_seeds"]
    nt = w["n_tcf"]
    rounds = w["tcf_rounds"]
    # TCF half, in rounds
    toff = off[: nt + 1]
    chunks = W.round_chunks(toff, rounds)
    mt = max(int((chunks[j, :, 1] - chunks[j, :, 0]).sum()) for j in range(rounds))
    T = gf.FilterGroup(gf.FILTER_TCF, logs[:nt], 16, seeds[:nt], max_total=mt)
    dk = dev_u64(keys[: toff[-1]])
    ok = np.zeros(int(toff[-1]), bool)
    for j in range(rounds):
        o, k = call_arrays(keys, chunks[j])
        st = zeros_u8(len(k))
        T.insert(dev_off(o), dev_u64(k), st)
        st = host(st)
        for m in range(nt):  # back to filter order
            s, e = chunks[j, m]
            ok[s:e] = st[o[m]:o[m + 1]] == 0
    found = zeros_u8(int(toff[-1]))
    T.query(dev_off(toff), dk, found)
    found = host(found).astype(bool)
    assert found[ok].all()  # no false negatives among the stored keys
    assert (~ok).mean() < 1e-3  # keys rejected as FULL near 95% load are rare
    sample_t = sorted({0, 1, nt - 1, int(np.argmax(logs[:nt])), int(np.argmin(logs[:nt]))})
    for m in sample_t:
        O = oracle.TCF(int(logs[m]), 16, seed=int(seeds[m]))
        for j in range(rounds):
            s, e = chunks[j, m]
            O.insert(keys[s:e])
        assert first_diff(T.export(m), O.export()) is None, m
    del T, dk, found
    torch.cuda.empty_cache()
    # GQF half, one batch
    goff = off[nt:] - off[nt]
    gk = keys[off[nt]:]
    G = gf.FilterGroup(gf.FILTER_GQF, logs[nt:], 8, seeds[nt:], max_total=len(gk))
    dk = dev_u64(gk)
    G.insert(dev_off(goff), dk)
    cnt = zeros_u64(len(gk))
    G.count(dev_off(goff), dk, cnt)
    assert (host(cnt) >= 1).all()
    sample_g = sorted({0, len(logs) - nt - 1, int(np.argmax(logs[nt:])), int(np.argmin(logs[nt:]))})
    for m in sample_g:
        O = oracle.GQF(int(logs[nt + m]), 8, seed=int(seeds[nt + m]))
        O.insert(gk[goff[m]:goff[m + 1]])
        assert first_diff(G.export(m), O.export()) is None, m


def test_tcf_group_calls_capture_in_a_cuda_graph(gf, oracle):
    """TCF group inserts and queries enqueue no host synchronisation, so a
    sequence of them can be captured once in a CUDA graph and replayed; the
    replay gives the same tables and answers as the oracle."""
    import torch

    w = W.batched_workload(n_filters=24, seed=43, emin=10, emax=12, tcf_rounds=2)
    logs, seeds, keys, off = w["log2_slots"], w["hash_seeds"], w["insert"], w["offsets"]
    n = len(logs)
    chunks = W.round_chunks(off, 2)
    calls = [call_arrays(keys, chunks[j]) for j in range(2)]
    G = gf.FilterGroup(gf.FILTER_TCF, logs, 16, seeds, max_total=len(keys))
    d_calls = [(dev_off(o), dev_u64(k)) for o, k in calls]
    d_q = dev_u64(keys)
    d_qo = dev_off(off)
    found = zeros_u8(len(keys))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        G.clear(stream=s)  # the first call of each kernel happens outside the capture
        G.insert(*d_calls[0], stream=s)
        G.query(d_qo, d_q, found, stream=s)
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            G.clear(stream=s)
            for o, k in d_calls:
                G.insert(o, k, stream=s)
            G.query(d_qo, d_q, found, stream=s)
    found.zero_()
    graph.replay()
    torch.cuda.synchronize()
    O = [oracle.TCF(int(logs[m]), 16, seed=int(seeds[m])) for m in range(n)]
    for j in range(2):
        o, k = calls[j]
        for m in range(n):
            O[m].insert(k[o[m]:o[m + 1]])
    check_images(G, O)
    fh = host(found)
    for m in range(n):
        assert np.array_equal(fh[off[m]:off[m + 1]], O[m].query(keys[off[m]:off[m + 1]])), m
