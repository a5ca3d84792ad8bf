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
from gpu_util import dev_u64, zeros_u8, zeros_u64, host

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
