"""The workload samplers: uniform doubles in [0, 1), samples with and without
replacement (distinct, in range, uniform by chi-square, reproducible), and the
batched workload's documented shape (sizes, loads, per-filter key ranges)."""
import numpy as np
from scipy import stats

from paper_2212_09005_gb300 import workloads as W


def test_uniform01_range_and_moments():
    u = W.uniform01(7, 0, 1 << 20)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert stats.kstest(u[:200_000], "uniform").pvalue > 1e-4


def test_sample_without_replacement():
    s = W.sample_without_replacement(11, 1000, 600)
    assert s.dtype == np.int64 and len(set(s.tolist())) == 600
    assert s.min() >= 0 and s.max() < 1000
    assert np.array_equal(s, W.sample_without_replacement(11, 1000, 600))
    assert np.array_equal(np.sort(W.sample_without_replacement(12, 50, 50)), np.arange(50))
    # each index is picked with probability k / population
    hits = np.zeros(40)
    for seed in range(400):
        hits[W.sample_without_replacement(1000 + seed, 40, 10)] += 1
    assert stats.chisquare(hits).pvalue > 1e-4


def test_sample_with_replacement_is_uniform():
    s = W.sample_with_replacement(13, 97, 500_000)
    assert s.min() >= 0 and s.max() < 97
    assert stats.chisquare(np.bincount(s, minlength=97)).pvalue > 1e-4


def test_batched_workload_shape():
    w = W.batched_workload(n_filters=64, seed=4, emin=10, emax=14)
    e, nk, off = w["log2_slots"], w["n_keys"], w["offsets"]
    assert e.min() >= 10 and e.max() <= 14 and w["n_tcf"] == 32
    load = nk / np.power(2.0, e)
    assert load.min() >= 0.85 - 1e-3 and load.max() < 0.95
    assert off[0] == 0 and np.array_equal(np.diff(off), nk)
    assert w["insert"].size == off[-1] == w["negatives"].size
    assert len(set(w["insert"].tolist())) == off[-1]  # distinct keys
    ch = W.round_chunks(off, w["tcf_rounds"])
    assert np.array_equal(ch[0, :, 0], off[:-1]) and np.array_equal(ch[-1, :, 1], off[1:])
    assert np.array_equal(ch[1:, :, 0], ch[:-1, :, 1])


def test_tcf_and_gqf_workload_shapes():
    t = W.tcf_workload(log2_slots=14, batch=1 << 11, n_query=1 << 12)
    n = int(0.9 * (1 << 14))
    ins = t["insert"]
    assert ins.size == n and len(set(ins.tolist())) == n
    assert len(set(t["pos_idx"].tolist())) == 1 << 12 and t["pos_idx"].max() < n
    assert len(set(t["del_idx"].tolist())) == n // 2 and t["del_idx"].max() < n
    assert not (set(t["negatives"].tolist()) & set(ins.tolist()))
    g = W.gqf_zipf_workload(q=16, n=200_000, n_query=5000)
    keys = g["insert"]
    assert keys.size == 200_000 and int(keys.max()) < (1 << 32)
    assert set(g["query"].tolist()) <= set(keys.tolist())
    u, c = np.unique(keys, return_counts=True)
    assert u[np.argmax(c)] == 0  # rank 1 (key 0) is the hottest
