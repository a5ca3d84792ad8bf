"""The serving workload's request stream, replayed on Python sets: inserts
bring keys never seen before, deletes take distinct live keys of their own
filter, no filter passes its cap, half of each query comes from the keys the
filter was given, sizes are powers of two within the range (or capped), the
stream stops at the target load, and Poisson arrivals have the right rate."""
import numpy as np

from paper_2212_09005_gb300 import workloads as W


def test_request_stream_invariants():
    lg, nf, bmin, bmax = 10, 6, 3, 8
    w = W.serving_workload(n_filters=nf, log2_slots=lg, seed=5, bmin=bmin, bmax=bmax)
    slots, cap = 1 << lg, int(0.95 * (1 << lg))
    live = [set(b.tolist()) for b in w["prefill"]]
    given = [set(s) for s in live]
    seen = set().union(*live)
    assert all(len(s) == slots // 2 for s in live) and len(seen) == nf * slots // 2
    ops = [0, 0, 0]
    for f, op, keys in w["requests"]:
        k = keys.tolist()
        ops[op] += 1
        assert 1 <= len(k) <= 1 << bmax
        if op == 0:
            assert not (set(k) & seen) and len(set(k)) == len(k)
            seen |= set(k)
            live[f] |= set(k)
            given[f] |= set(k)
            assert len(live[f]) <= cap
        elif op == 1:
            h = len(k) // 2
            assert set(k[:h]) <= given[f]
        else:
            assert len(set(k)) == len(k) and set(k) <= live[f]
            live[f] -= set(k)
    # the stream ends with the insert that brings the live keys to 90% of all slots
    goal = int(0.9 * slots * nf)
    total = sum(len(s) for s in live)
    last_f, last_op, last_keys = w["requests"][-1]
    assert last_op == 0 and total >= goal > total - len(last_keys)
    n = len(w["requests"])
    assert ops[0] > 0.3 * n and ops[1] > 0.3 * n and ops[2] > 0


def test_poisson_arrivals_rate():
    t = W.poisson_arrivals(29, 200_000, rate=5000.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 5000.0) < 5 * (1 / 5000.0) / np.sqrt(gaps.size)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.02  # exponential: coefficient of variation 1
