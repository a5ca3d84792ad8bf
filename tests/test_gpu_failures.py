"""Failure detection without a device fault: a bounded device wait that runs
out reports FILTER_ERR_TIMEOUT through the filter's status word and leaves
the filter usable; an allocation that fails (injected on the host) makes the
create calls return FILTER_ERR_OOM without leaking what they had already
allocated."""
import time

import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u64, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def test_bounded_wait_gives_up_with_timeout_status(gf):
    G = gf.GQF(12, 8, seed=1, max_batch=4096)
    keys = W.uniform_keys(61, 3000)
    G.insert(dev_u64(keys))
    assert G.stats()["status_word"] & gf.STATUS_TIMEOUT == 0
    t0 = time.perf_counter()
    gf.debug_wait_timeout(G, 10_000)  # the predecessor never publishes: the wait must give up
    st = G.stats()  # synchronises the stream
    assert time.perf_counter() - t0 < 10
    assert st["status_word"] & gf.STATUS_TIMEOUT
    # the table is untouched and the filter keeps working
    c = zeros_u64(len(keys))
    G.count(dev_u64(keys), c)
    assert (host(c) >= 1).all()
    G.insert(dev_u64(W.uniform_keys(62, 500)))
    assert G.stats()["failed_keys"] == 0
    with pytest.raises(gf.FilterError):
        gf.debug_wait_timeout(G, 0)


def test_allocation_failure_reports_oom_without_leaks(gf):
    base = gf.debug_live_allocations()
    try:
        # filter_create makes two allocations (table + scratch, counters): fail each in turn
        for nth in (1, 2):
            gf.debug_fail_alloc(nth)
            with pytest.raises(gf.FilterError, match="code 2"):
                gf.GQF(14, 8, seed=2, max_batch=1 << 12)
            assert gf.debug_live_allocations() == base
            gf.debug_fail_alloc(nth)
            with pytest.raises(gf.FilterError, match="code 2"):
                gf.TCF(14, 16, gf.MODE_BULK, seed=2, max_batch=1 << 12)
            assert gf.debug_live_allocations() == base
        gf.debug_fail_alloc(1)
        with pytest.raises(gf.FilterError, match="code 2"):
            gf.FilterGroup(gf.FILTER_GQF, [10, 11], 8, [1, 2], max_total=1 << 12)
        assert gf.debug_live_allocations() == base
        ok = gf.GQF(12, 8, seed=3, max_batch=1 << 12)
        assert gf.debug_live_allocations() == base + 2
        gf.debug_fail_alloc(1)
        with pytest.raises(gf.FilterError, match="code 2"):
            gf.FilterServer([ok], workers=2, max_keys=1 << 12)
        assert gf.debug_live_allocations() == base + 2
    finally:
        gf.debug_fail_alloc(0)
    # with nothing injected everything works again, and destroying frees all
    G = gf.GQF(12, 8, seed=3, max_batch=1 << 12)
    G.insert(dev_u64(W.uniform_keys(63, 1000)))
    assert G.stats()["failed_keys"] == 0
    del G, ok
    import gc

    gc.collect()
    assert gf.debug_live_allocations() == base
