"""CPU tests of the serving loop's scheduler (csrc/gf_sched.h) with a fake
device-memory budget: per-filter order and one batch in flight per filter,
which requests merge, admission as staging memory frees up, refusal of
requests larger than the pool, the anti-starvation rule, and a randomized run
that checks the invariants against a replay of the trace."""
import ctypes as C
import os
import random
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INS, QRY, REM, CNT = 0, 1, 2, 3


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("sched") / "libsched.so")
    src = os.path.join(ROOT, "tests", "sched", "sched_shim.cpp")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                        os.path.join(ROOT, "paper_2212_09005_gb300", "csrc"), "-o", out, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(out)
    u64, u32 = C.c_uint64, C.c_uint32
    L.sched_new.argtypes = [u32, C.POINTER(C.c_uint8), C.POINTER(u64), u64, u32]
    L.sched_new.restype = C.c_void_p
    L.sched_free.argtypes = [C.c_void_p]
    L.sched_submit.argtypes = [C.c_void_p, u64, u32, u32, u64]
    L.sched_next.argtypes = [C.c_void_p, C.POINTER(u64), u32]
    L.sched_finish.argtypes = [C.c_void_p, u32, u32, u64, u64, u64]
    L.sched_pool_available.argtypes = [C.c_void_p]
    L.sched_pool_available.restype = u64
    L.sched_waiting.argtypes = [C.c_void_p]
    L.sched_waiting.restype = u64
    L.sched_staging_bytes.argtypes = [u32, u64]
    L.sched_staging_bytes.restype = u64
    return L


class Sched:
    def __init__(self, L, gqf, max_merge, pool, max_skips=8):
        n = len(gqf)
        self.L = L
        mr = (C.c_uint8 * n)(*[1 if g else 0 for g in gqf])
        mm = (C.c_uint64 * n)(*max_merge)
        self.h = L.sched_new(n, mr, mm, pool, max_skips)

    def submit(self, t, f, op, n):
        return bool(self.L.sched_submit(self.h, t, f, op, n))

    def next(self):
        buf = (C.c_uint64 * 4096)()
        if not self.L.sched_next(self.h, buf, 4096):
            return None
        k = int(buf[5])
        return {"filter": int(buf[0]), "op": int(buf[1]), "n": int(buf[2]), "offset": int(buf[3]),
                "bytes": int(buf[4]), "tickets": [int(buf[6 + i]) for i in range(k)]}

    def finish(self, b):
        self.L.sched_finish(self.h, b["filter"], b["op"], b["n"], b["offset"], b["bytes"])

    def __del__(self):
        self.L.sched_free(self.h)


def test_one_batch_per_filter_in_submission_order(lib):
    S = Sched(lib, [False, False], [1 << 20] * 2, 1 << 30)
    for t, (f, op) in enumerate([(0, INS), (0, INS), (1, INS), (0, REM)], start=1):
        assert S.submit(t, f, op, 100)
    a = S.next()
    b = S.next()
    assert (a["filter"], a["tickets"]) == (0, [1])  # oldest first
    assert (b["filter"], b["tickets"]) == (1, [3])  # filter 0 is busy: another worker takes filter 1
    assert S.next() is None                         # nothing else may start
    S.finish(a)
    c = S.next()
    assert c["tickets"] == [2]                      # TCF inserts never merge
    S.finish(c)
    assert S.next()["tickets"] == [4]


def test_merge_rules(lib):
    S = Sched(lib, [False, True], [1000, 1000], 1 << 30)
    reqs = [(0, QRY, 100), (0, QRY, 200), (0, CNT, 10), (1, REM, 300), (1, REM, 300), (1, REM, 500),
            (0, REM, 5), (0, REM, 5)]
    for t, (f, op, n) in enumerate(reqs, start=1):
        S.submit(t, f, op, n)
    a = S.next()
    assert a["tickets"] == [1, 2] and a["n"] == 300   # queries merge, the count does not join them
    b = S.next()
    assert b["tickets"] == [4, 5] and b["n"] == 600   # GQF removes merge up to max_merge (1000)
    S.finish(a)
    assert S.next()["tickets"] == [3]
    S.finish(b)
    assert S.next()["tickets"] == [6]
    S2 = Sched(lib, [False], [1000], 1 << 30)
    S2.submit(1, 0, REM, 5)
    S2.submit(2, 0, REM, 5)
    assert S2.next()["tickets"] == [1]                # TCF removes never merge


def test_admission_waits_for_staging_memory(lib):
    per = lib.sched_staging_bytes(QRY, 1000)
    S = Sched(lib, [False] * 3, [1 << 20] * 3, 2 * per)  # room for two 1000-key batches
    for t, f in enumerate([0, 1, 2], start=1):
        S.submit(t, f, QRY, 1000)
    a, b = S.next(), S.next()
    assert a and b and lib.sched_pool_available(S.h) == 0
    assert S.next() is None                          # the third waits for memory
    S.finish(b)
    c = S.next()
    assert c["filter"] == 2 and c["offset"] == b["offset"]
    assert not S.submit(9, 0, QRY, 3000)             # larger than the whole pool: refused


def test_merged_batch_that_does_not_fit_runs_its_head_alone(lib):
    per = lib.sched_staging_bytes(QRY, 1000)
    S = Sched(lib, [False] * 2, [1 << 20] * 2, 2 * per)
    S.submit(1, 1, QRY, 1000)
    x = S.next()                                     # half of the pool is taken
    S.submit(2, 0, QRY, 1000)
    S.submit(3, 0, QRY, 1000)
    a = S.next()
    assert a["tickets"] == [2]                       # merged would need the whole pool: the head alone
    S.finish(x)
    S.finish(a)
    assert S.next()["tickets"] == [3]


def test_large_request_is_not_starved(lib):
    small = lib.sched_staging_bytes(QRY, 100)
    big = lib.sched_staging_bytes(QRY, 4000)
    S = Sched(lib, [False] * 4, [1 << 20] * 4, big, max_skips=3)
    S.submit(1, 1, QRY, 100)
    run = [S.next()]                                 # a small batch holds part of the pool
    S.submit(2, 0, QRY, 4000)                        # the big one needs all of it
    t = 3
    admitted_ahead = 0
    for _ in range(10):                              # small requests keep arriving on other filters
        S.submit(t, 2 + (t % 2), QRY, 100)
        t += 1
        b = S.next()
        if b is not None:
            assert b["filter"] != 0
            admitted_ahead += 1
            run.append(b)
        for r in run[1:]:
            S.finish(r)
        run = run[:1]
    assert admitted_ahead == 3                       # passed over max_skips times, then nothing more
    S.finish(run[0])
    b = S.next()
    assert b["filter"] == 0 and b["tickets"] == [2]


def test_randomized_invariants(lib):
    rng = random.Random(7)
    nf, pool = 6, 1 << 16
    gqf = [f % 2 == 1 for f in range(nf)]
    S = Sched(lib, gqf, [3000] * nf, pool)
    submitted = {f: [] for f in range(nf)}
    info = {}
    ran = {f: [] for f in range(nf)}
    running = []
    t = 1
    for step in range(4000):
        if rng.random() < 0.55:
            f, op, n = rng.randrange(nf), rng.choice([INS, QRY, REM, CNT]), rng.randrange(1, 2500)
            if S.submit(t, f, op, n):
                submitted[f].append(t)
                info[t] = (f, op, n)
            t += 1
        if running and rng.random() < 0.4:
            S.finish(running.pop(rng.randrange(len(running))))
        b = S.next()
        if b is not None:
            f = b["filter"]
            assert all(r["filter"] != f for r in running), "two batches of one filter in flight"
            assert sum(r["bytes"] for r in running) + b["bytes"] <= pool
            spans = sorted([(r["offset"], r["offset"] + r["bytes"]) for r in running + [b]])
            assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1)), "staging overlaps"
            ops = {info[x][1] for x in b["tickets"]}
            assert len(ops) == 1 and b["n"] == sum(info[x][2] for x in b["tickets"])
            if len(b["tickets"]) > 1:
                op = ops.pop()
                assert op in (QRY, CNT) or (op == REM and gqf[f])
                assert b["n"] <= 3000
            ran[f].extend(b["tickets"])
            running.append(b)
    while lib.sched_waiting(S.h) or running:
        if running:
            S.finish(running.pop())
        b = S.next()
        if b is not None:
            ran[b["filter"]].extend(b["tickets"])
            running.append(b)
    for f in range(nf):
        assert ran[f] == submitted[f], "a filter's requests ran out of order or not at all"
    assert lib.sched_pool_available(S.h) == pool
