"""Device-side point queries (include/gpufilter_device.cuh) called from a
kernel compiled outside the library: their answers equal filter_query /
filter_count on the same filters and keys (TCF bulk and point mode, 16- and
8-bit tags, with the backing table in use; GQF with 8- and 16-bit remainders)."""
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
