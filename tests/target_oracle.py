"""Oracle side of the target-size parity tests (2^28 slots, 90 % load).

At this size the oracle takes minutes, so each filter's oracle run happens in
a spawned process (safe after CUDA is up) that regenerates the seeded inputs
itself and returns what the GPU side is compared with: per-MiB digests of the
table images, per-key statuses and answers. `start()` launches both runs once
per test session; conftest calls it as soon as a target test is selected, so
the oracle works while the other GPU tests run.

TCF: the incremental oracle, batch by batch (2^24-key batches), exactly as
the GPU receives them. GQF: brute force and the oracle's independent
canonical builder (gqf_build) on the fingerprint multiset, because the table
of a GQF is a function of that multiset alone."""
from __future__ import annotations

import hashlib

import numpy as np

CHUNK = 1 << 20
TCF_LOG2, TCF_SEED, TCF_BATCH = 28, 8, 1 << 24
GQF_Q, GQF_SEED = 28, 9

_futures = {}
_pool = None


def digests(img: np.ndarray) -> list:
    """blake2b digest of every MiB of a byte image (the last chunk may be short)."""
    img = np.ascontiguousarray(img).view(np.uint8)
    return [hashlib.blake2b(img[i:i + CHUNK].tobytes(), digest_size=16).digest() for i in range(0, img.size, CHUNK)]


def first_chunk_diff(a: list, b: list):
    if len(a) != len(b):
        return f"{len(a)} vs {len(b)} chunks"
    for i, (x, y) in enumerate(zip(a, b)):
        if x != y:
            return f"first differing MiB chunk: {i} of {len(a)}"
    return None


def tcf_inputs():
    from paper_2212_09005_gb300 import workloads as W

    w = W.tcf_workload(log2_slots=TCF_LOG2, seed=TCF_SEED, batch=TCF_BATCH, n_query=1 << 24)
    ins = w["insert"]
    probe = np.concatenate([ins[w["pos_idx"]], w["negatives"]])
    return ins, probe, ins[w["del_idx"]]


def gqf_inputs():
    from paper_2212_09005_gb300 import workloads as W

    w = W.gqf_target_workload(q=GQF_Q, seed=GQF_SEED)
    ins = w["insert"]
    probe = np.concatenate([ins[w["pos_idx"]], w["negatives"]])
    return ins, probe, ins[w["del_idx"]]


def tcf_run() -> dict:
    import oracle as O

    ins, probe, dels = tcf_inputs()
    T = O.TCF(TCF_LOG2, 16, seed=TCF_SEED)
    st_ins = np.concatenate([T.insert(ins[i:i + TCF_BATCH]) for i in range(0, len(ins), TCF_BATCH)])
    out = {"ins_failed": int(np.count_nonzero(st_ins)), "ins_status_digest": digests(st_ins),
           "img_ins": digests(T.export()), "q1": T.query(probe), "backing": T.backing_count()}
    st_del = np.concatenate([T.remove(dels[i:i + TCF_BATCH]) for i in range(0, len(dels), TCF_BATCH)])
    out.update({"del_status_digest": digests(st_del), "img_del": digests(T.export()), "q2": T.query(probe)})
    return out


def gqf_run() -> dict:
    import oracle as O

    ins, probe, dels = gqf_inputs()
    G = O.GQF(GQF_Q, 8, seed=GQF_SEED)  # used for its fingerprint function only
    fu, cnt = np.unique(G.fingerprints(ins), return_counts=True)
    cnt = cnt.astype(np.uint64)
    img1 = O.gqf_build(GQF_Q, 8, fu, cnt)

    def counts_of(keys, fu, cnt):
        fp = G.fingerprints(keys)
        j = np.searchsorted(fu, fp)
        j[j == fu.size] = 0
        return np.where(fu[j] == fp, cnt[j], 0).astype(np.uint64)

    c1 = counts_of(probe, fu, cnt)
    # every deleted key is a distinct inserted key: each delete finds a copy
    fd = G.fingerprints(dels)
    np.subtract.at(cnt, np.searchsorted(fu, fd), np.uint64(1))
    keep = cnt > 0
    fu2, cnt2 = fu[keep], cnt[keep]
    img2 = O.gqf_build(GQF_Q, 8, fu2, cnt2)
    return {"img_ins": digests(img1), "c1": c1, "img_del": digests(img2), "c2": counts_of(probe, fu2, cnt2),
            "groups": int(fu.size)}


def start():
    """Launch both oracle runs (once per process) in spawned workers."""
    global _pool
    if _futures:
        return _futures
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    _pool = ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn"))
    _futures["tcf"] = _pool.submit(tcf_run)
    _futures["gqf"] = _pool.submit(gqf_run)
    return _futures


def result(name: str, timeout: float = 1800.0) -> dict:
    return start()[name].result(timeout=timeout)
