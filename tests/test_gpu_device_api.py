"""Device-side point operations (include/gpufilter_device.cuh) called from
kernels compiled outside the library: query answers equal filter_query /
filter_count on the same filters and keys (TCF bulk and point mode, 16- and
8-bit tags, with the backing table in use; GQF with 8- and 16-bit remainders);
point-mode TCF inserts and removes from a user kernel leave answers equal to
membership in the live fingerprint multiset."""
import collections
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, zeros_u64, host, first_diff

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


@pytest.fixture(scope="module")
def example(tmp_path_factory):
    """The example kernel, built like a user of the header would build it."""
    out = str(tmp_path_factory.mktemp("device_api") / "libdevice_query_example.so")
    src = os.path.join(ROOT, "tests", "device_api", "device_query_example.cu")
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared", "-Xcompiler",
           "-fPIC", "-I", os.path.join(ROOT, "include"), "-o", out, src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    lib.device_query_example.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.device_query_example.restype = C.c_int
    lib.device_update_example.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p]
    lib.device_update_example.restype = C.c_int
    lib.device_update_serial_example.argtypes = lib.device_update_example.argtypes
    lib.device_update_serial_example.restype = C.c_int
    return lib


def run_example(example, view, keys, found=None, counts=None):
    import torch

    assert example.device_query_example(C.byref(view), C.c_void_p(keys.data_ptr()), keys.numel(),
                                        C.c_void_p(found.data_ptr()) if found is not None else None,
                                        C.c_void_p(counts.data_ptr()) if counts is not None else None, None) == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("f,mode", [(16, "bulk"), (8, "bulk"), (16, "point")])
def test_tcf_device_queries_equal_bulk_queries(gf, example, f, mode):
    q = 16
    keys = W.uniform_keys(81, int(0.93 * (1 << q)))
    T = gf.TCF(q, f, gf.MODE_BULK if mode == "bulk" else gf.MODE_POINT, seed=17, max_batch=len(keys))
    T.insert(dev_u64(keys))
    if mode == "point":
        T.remove(dev_u64(keys[::5]))
    if mode == "bulk" and f == 16:
        assert T.stats()["backing_used"] > 0, "the load should put keys in the backing table"
    probe = dev_u64(np.concatenate([keys, W.uniform_keys(82, 1 << 16)]))
    want, got = zeros_u8(probe.numel()), zeros_u8(probe.numel())
    T.query(probe, want)
    run_example(example, T.device_view(), probe, found=got)
    assert np.array_equal(host(got), host(want))


@pytest.mark.parametrize("q,r", [(16, 8), (15, 16)])
def test_gqf_device_counts_equal_bulk_counts(gf, example, q, r):
    keys = W.zipf_keys(83, int(0.6 * (1 << q)), 1.0, 1 << 20)
    G = gf.GQF(q, r, seed=19, max_batch=len(keys))
    G.insert(dev_u64(keys[: len(keys) // 2]))
    G.insert(dev_u64(keys[len(keys) // 2:]))  # the view must follow the second table buffer
    probe = dev_u64(np.concatenate([np.unique(keys), W.uniform_keys(84, 1 << 14)]))
    want, got = zeros_u64(probe.numel()), zeros_u64(probe.numel())
    G.count(probe, want)
    run_example(example, G.device_view(), probe, counts=got)
    assert np.array_equal(host(got), host(want))
    assert host(want)[: len(np.unique(keys))].min() >= 1


def run_update(example, view, keys, remove, status):
    import torch

    assert example.device_update_example(C.byref(view), C.c_void_p(keys.data_ptr()), keys.numel(), int(remove),
                                         C.c_void_p(status.data_ptr()), None) == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("f", [16, 8])
def test_point_tcf_updates_from_a_user_kernel(gf, oracle, example, f):
    """Keys inserted and removed by a user kernel, concurrently across threads:
    the filter then answers membership in the live fingerprint multiset (with
    the paired blocks, answers depend only on it, whatever the placement)."""
    q = 14
    keys = W.uniform_keys(85, int(0.8 * (1 << q)))
    T = gf.TCF(q, f, gf.MODE_POINT, seed=23, max_batch=len(keys))
    O = oracle.TCF(q, f, seed=23)  # hash only: fingerprints (min(b1, b2), tag)

    def membership(live, probe):
        c = collections.Counter(O.fingerprints(live).tolist())
        return np.array([c.get(int(x), 0) > 0 for x in O.fingerprints(probe)], np.uint8)

    st = zeros_u8(len(keys))
    run_update(example, T.device_view(), dev_u64(keys), False, st)
    s = host(st)
    ok = keys[s == 0]
    assert set(np.unique(s).tolist()) <= {0, 1} and len(ok) >= 0.99 * len(keys)
    assert T.stats()["failed_keys"] == int((s == 1).sum())
    probe_np = np.concatenate([keys, W.uniform_keys(86, 1 << 15)])
    probe = dev_u64(probe_np)
    got = zeros_u8(len(probe_np))
    T.query(probe, got)
    assert np.array_equal(host(got), membership(ok, probe_np))
    gone, kept = ok[::3], np.delete(ok, np.arange(0, len(ok), 3))
    st2 = zeros_u8(len(gone))
    run_update(example, T.device_view(), dev_u64(gone), True, st2)
    assert not host(st2).any()
    T.query(probe, got)
    assert np.array_equal(host(got), membership(kept, probe_np))
    # a bulk-mode filter refuses device updates, which would break its sorted blocks
    B = gf.TCF(q, f, gf.MODE_BULK, seed=23, max_batch=16)
    st3 = zeros_u8(16)
    run_update(example, B.device_view(), dev_u64(keys[:16]), False, st3)
    assert (host(st3) == 1).all() and B.stats()["failed_keys"] == 0


@pytest.mark.parametrize("q,r", [(12, 8), (12, 16)])
def test_point_gqf_updates_one_thread(gf, oracle, example, q, r):
    """The point insert and remove, key after key from one thread: the
    table equals the oracle's after each stage."""
    import torch

    G = gf.GQF(q, r, seed=q + 2 * r, max_batch=1 << 14)
    n = int(0.68 * (1 << q))  # with the repeats (3 slots each): 85 % of the home slots
    base = W.uniform_keys(5000 + q, n * 3 // 4)
    keys = np.concatenate([base, base[: n // 4]])
    view = G.device_view()
    st = torch.zeros(keys.size, dtype=torch.uint8, device="cuda")
    assert example.device_update_serial_example(C.byref(view), C.c_void_p(dev_u64(keys).data_ptr()), keys.size, 0,
                                                C.c_void_p(st.data_ptr()), None) == 0
    torch.cuda.synchronize()
    O = oracle.GQF(q, r, seed=q + 2 * r)
    want = O.insert(keys)
    assert np.array_equal(host(st), want), np.unique(host(st), return_counts=True)
    assert first_diff(G.export(), O.export()) is None
    rem = np.concatenate([base[::2], base[: n // 8], W.uniform_keys(5050 + q, 300)])
    d = dev_u64(rem)
    st = torch.zeros(rem.size, dtype=torch.uint8, device="cuda")
    assert example.device_update_serial_example(C.byref(view), C.c_void_p(d.data_ptr()), rem.size, 1,
                                                C.c_void_p(st.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert np.array_equal(host(st), O.remove(rem))
    assert first_diff(G.export(), O.export()) is None


@pytest.mark.parametrize("q,r", [(18, 8), (17, 16), (14, 8)])
def test_point_gqf_updates_from_a_user_kernel(gf, oracle, example, q, r):
    """Locked point GQF (Sec. 5.2): one key per thread, many threads on the
    same regions at once (repeated keys, neighbouring quotients). The table
    of a GQF is a function of its fingerprint multiset, so after the point
    inserts the image equals the oracle's after a bulk insert of the same
    keys, and after point removes the oracle's after the same removes."""
    import torch

    G = gf.GQF(q, r, seed=q + r, max_batch=1 << 16)
    n = int(0.68 * (1 << q))  # with the repeats (3 slots each): 85 % of the home slots
    base = W.uniform_keys(5100 + q, n * 3 // 4)
    keys = np.concatenate([base, base[: n // 4]])  # repeated keys: counters, and contention on one run
    keys = keys[W.sample_without_replacement(5200 + q, keys.size, keys.size)]  # interleave the copies
    view = G.device_view()
    st = torch.zeros(keys.size, dtype=torch.uint8, device="cuda")
    run_update(example, view, dev_u64(keys), False, st)
    assert not host(st).any(), np.unique(host(st), return_counts=True)
    O = oracle.GQF(q, r, seed=q + r)
    O.insert(keys)
    assert first_diff(G.export(), O.export()) is None
    probe = np.concatenate([base[::5], W.uniform_keys(5300 + q, 3000)])
    c = torch.zeros(probe.size, dtype=torch.int64, device="cuda")
    run_example(example, view, dev_u64(probe), counts=c)
    assert np.array_equal(host(c), O.count(probe))
    # removes: stored keys (some twice), and absent ones
    rem = np.concatenate([base[::2], base[: n // 8], W.uniform_keys(5400 + q, 500)])
    st = torch.zeros(rem.size, dtype=torch.uint8, device="cuda")
    run_update(example, view, dev_u64(rem), True, st)
    fpr = O.fingerprints(rem)
    want = O.remove(rem)
    # which copy of a repeated remove finds nothing depends on the threads'
    # order: compare the statuses per fingerprint
    got = collections.Counter(zip(fpr.tolist(), host(st).tolist()))
    assert got == collections.Counter(zip(fpr.tolist(), want.tolist()))
    assert first_diff(G.export(), O.export()) is None
    assert G.stats()["status_word"] == 0


def test_point_gqf_full_table_reports_full_without_damage(gf, oracle, example):
    """Point inserts into a table without room for all of them: the keys
    reported OK are exactly the stored multiset, the table is the canonical
    layout of that multiset (a consistent table, whatever order the threads
    took), and the FULL ones are counted."""
    import torch

    q, r = 10, 8
    G = gf.GQF(q, r, seed=3, max_batch=1 << 12)
    view = G.device_view()
    keys = W.uniform_keys(5500, 2 << q)
    st = torch.zeros(keys.size, dtype=torch.uint8, device="cuda")
    run_update(example, view, dev_u64(keys), False, st)
    s = host(st)
    assert set(np.unique(s)) <= {gf.KEY_OK, gf.KEY_FULL}
    assert (s == gf.KEY_FULL).any()
    O = oracle.GQF(q, r, seed=3)
    fu, cnt = np.unique(O.fingerprints(keys[s == gf.KEY_OK]), return_counts=True)
    fps, cnts = (host(t) for t in G.enumerate())
    assert np.array_equal(fps, fu) and np.array_equal(cnts, cnt.astype(np.uint64))
    assert O.insert_groups(fu, cnt) == fu.size
    assert first_diff(G.export(), O.export()) is None
    assert G.stats()["failed_keys"] == int((s == gf.KEY_FULL).sum())
