"""The batched workload's oracle baseline on all host cores (CPU only): the
sample takes every k-th filter, each in its own oracle filter, one spawned
process per core, and counts three operations per inserted key."""
import numpy as np


def test_batched_oracle_baseline_on_all_cores():
    import bench
    from paper_2212_09005_gb300 import workloads as W

    w = W.batched_workload(n_filters=12, seed=4, emin=10, emax=12)
    r = bench.cpu_batched_sample(w, target_keys=1 << 13)
    k = max(1, int(w["offsets"][-1]) // (1 << 13))
    picked = np.arange(0, 12, k)
    nk = int(sum(w["n_keys"][i] for i in picked))
    assert r["kind"] == "oracle" and r["unit"] == "Gops/s"
    assert r["ops"] == 3 * nk
    assert 1 <= r["cores"] <= len(picked)
    assert r["value"] > 0 and r["seconds"] >= 0  # (a small sample can round to 0 s)
    assert f"{len(picked)} filters" in r["sample"]


def test_worker_counts_tcf_rounds_and_gqf_batches():
    import bench

    tasks = [("tcf", 10, 7, 0, 800, 8, 4), ("gqf", 10, 9, 800, 700, 8, 4)]
    ops, sec = bench._oracle_filters_worker(tasks)
    assert ops == 3 * 1500 and sec > 0
