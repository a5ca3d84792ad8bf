"""Per-size kernel choices, measured on the device they are used on.

None of these choices changes a result: both TCF bulk paths apply the same
phased insert and remove (Section 4.2) and leave the same table, and the GQF
in-place and merge paths both leave the canonical table of the stored
multiset (Section 5). They only trade launch count against memory traffic,
and where the trade-off turns over is a property of the device, so it is
measured rather than assumed:

  tcf_path            per-block counting sort (one CTA per 2^k blocks, keys
                      sorted in shared memory) or tiled (one partition of the
                      whole batch by tile, one CTA per tile of blocks);
  tcf_tile_target     candidates per tile the tiled path aims for;
  gqf_region_groups   how many 64-slot groups a batch may touch per key
                      before the GQF leaves the in-place path for a merge.

`autotune()` times each choice on synthetic filters of every size class and
writes `tuning.json` next to this file; `Filter` and `FilterGroup` apply the
entry of the largest size class not above their own at creation. Without the
file every knob keeps its built-in default."""
from __future__ import annotations

import json
import os
import time

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
KNOBS = ("tcf_path", "tcf_tile_target", "gqf_region_groups", "tcf_tiled_min_blocks")

_table = None


def table() -> dict:
    """The measured table ({} when none was written)."""
    global _table
    if _table is None:
        try:
            with open(TABLE_PATH) as f:
                _table = json.load(f)
        except (OSError, ValueError):
            _table = {}
    return _table


def _pick(rows: dict, log2_slots: int):
    best, knobs = -1, None
    for k, v in rows.items():
        lg = int(k)
        if best < lg <= log2_slots:
            best, knobs = lg, {n: int(x) for n, x in v.items() if n in KNOBS}
    return knobs


def lookup(kind: int, log2_slots: int, group: bool = False) -> dict:
    """Knobs for a filter, or (group) for a filter group of that many slots in
    all: a TCF group takes the measured group rows when one covers its size
    (many small members behave unlike one table of their total size), else
    the single-filter rows."""
    from . import FILTER_TCF

    t = table()
    name = "tcf" if kind == FILTER_TCF else "gqf"
    if group:
        k = _pick(t.get(name + "_group", {}), log2_slots)
        if k is not None:
            return k
    return _pick(t.get(name, {}), log2_slots) or {}


def struct(knobs: dict):
    from . import FilterError, FilterTuning

    bad = set(knobs) - set(KNOBS)
    if bad:
        raise FilterError(f"unknown tuning knobs {sorted(bad)}")
    return FilterTuning(int(knobs.get("tcf_path", 0)), int(knobs.get("tcf_tile_target", 0)),
                        int(knobs.get("gqf_region_groups", 0)), 0, int(knobs.get("tcf_tiled_min_blocks", 0)))


# ---------------------------------------------------------------------------
# Measurement
# ---------------------------------------------------------------------------
TCF_CANDIDATES = ((1, 0), (2, 256), (2, 512), (2, 1024))  # (tcf_path, tile target)
GQF_CANDIDATES = (4, 8, 16, 32, 64, 128)                  # region groups


def _timed(torch, fn, reps=2):
    """Best of `reps` runs of fn (which returns a list of (start, end) CUDA
    event pairs): milliseconds per pair, summed."""
    best = None
    for _ in range(reps):
        pairs = fn()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in pairs)
        best = ms if best is None else min(best, ms)
    return best


def tune_tcf(lg: int, keys, torch) -> dict:
    """A 2^lg-slot bulk TCF filled to 90 % in batches of one key per block
    (2^(lg-4) keys), then half of the keys removed in batches of the same
    size: the path and tile target with the least total time."""
    from . import MODE_BULK, TCF

    nb = 1 << (lg - 4)
    n = int(0.9 * (1 << lg))
    b = min(nb, n)
    ins = [keys[i:min(i + b, n)] for i in range(0, n, b)]
    dels = [keys[i:min(i + b, n // 2)] for i in range(0, n // 2, b)]
    F = TCF(lg, 16, MODE_BULK, seed=lg, max_batch=b)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for path, target in TCF_CANDIDATES:
        F.set_tuning(tcf_path=path, tcf_tile_target=target)

        def run():
            F.clear()
            a, m, z = ev(), ev(), ev()
            a.record()
            for k in ins:
                F.insert(k)
            m.record()
            for k in dels:
                F.remove(k)
            z.record()
            return [(a, m), (m, z)]

        run()  # warm-up
        res[f"{'block' if path == 1 else 'tiled'}{'' if path == 1 else '_' + str(target)}"] = round(
            _timed(torch, run), 3)
    F.close()
    best = min(res, key=res.get)
    if best == "block":
        knobs = {"tcf_path": 1}
    else:  # tiled when a batch has at least one key per block, else per-block
        knobs = {"tcf_path": 0, "tcf_tiled_min_blocks": nb, "tcf_tile_target": int(best.split("_")[1])}
    return {**knobs, "ms": res, "batch": b}


def tune_tcf_group(torch, n_filters: int = 2048, rounds: int = 8, seed: int = 78) -> tuple:
    """A TCF group shaped like the batched workload (members of 2^10 .. 2^20
    slots at 85-95 % load, keys in `rounds` per-member chunks), then a removal
    of every member's first chunk: the path with the least total time.
    Returns (log2 of the group's slots, entry)."""
    import numpy as np

    from . import FILTER_TCF, FilterGroup
    from . import workloads as W

    w = W.batched_workload(n_filters=2 * n_filters, seed=seed, tcf_rounds=rounds)
    nt = w["n_tcf"]
    off = w["offsets"][: nt + 1]
    logs, seeds = w["log2_slots"][:nt], w["hash_seeds"][:nt]
    keys = w["insert"][: off[-1]]
    chunks = W.round_chunks(off, rounds)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()
    calls = []
    for j in range(rounds):
        lens = chunks[j, :, 1] - chunks[j, :, 0]
        o = np.zeros(nt + 1, np.int64)
        np.cumsum(lens, out=o[1:])
        calls.append((dev(o), dev(np.concatenate([keys[a:b] for a, b in chunks[j]]))))
    mt = max(int(k.numel()) for _, k in calls)
    G = FilterGroup(FILTER_TCF, logs, 16, seeds, max_total=mt)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for path in (1, 2):
        G.set_tuning(tcf_path=path, tcf_tile_target=1024 if path == 2 else 0)

        def run():
            G.clear()
            a, m, z = ev(), ev(), ev()
            a.record()
            for o, k in calls:
                G.insert(o, k)
            m.record()
            G.remove(*calls[0])
            z.record()
            return [(a, m), (m, z)]

        run()
        res["block" if path == 1 else "tiled_1024"] = round(_timed(torch, run), 3)
    G.close()
    lg = int(sum(1 << int(x) for x in logs)).bit_length() - 1
    best = min(res, key=res.get)
    return lg, {**({"tcf_path": 1} if best == "block" else {"tcf_path": 2, "tcf_tile_target": 1024}), "ms": res,
                "members": int(nt)}


def tune_gqf(q: int, keys, torch) -> dict:
    """A GQF with 2^q home slots filled to 90 % in one batch; then a batch
    of min(2^24, n/16) distinct stored keys is removed and inserted again:
    the region bound with the least total time for the two."""
    from . import GQF

    n = int(0.9 * (1 << q))
    b = min(1 << 24, n // 16)
    F = GQF(q, 8, seed=q, max_batch=n)
    sub = keys[:b]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for g in GQF_CANDIDATES:
        F.set_tuning(gqf_region_groups=g)
        F.clear()
        F.insert(keys[:n])

        def run():
            a, m, z = ev(), ev(), ev()
            a.record()
            F.remove(sub)
            m.record()
            F.insert(sub)
            z.record()
            return [(a, m), (m, z)]

        run()  # warm-up
        res[str(g)] = round(_timed(torch, run), 3)
    F.close()
    best = min(res, key=res.get)
    return {"gqf_region_groups": int(best), "ms": res, "batch": b}


def autotune(tcf_classes=(20, 22, 24, 26, 27, 28), gqf_classes=(20, 22, 24, 26, 28), path: str = TABLE_PATH,
             seed: int = 77) -> dict:
    """Measure every size class on the current CUDA device and write the
    table (the classes' uniform keys are prefixes of one seeded stream)."""
    global _table
    import torch

    from . import workloads as W

    n_max = int(0.9 * (1 << max(max(tcf_classes), max(gqf_classes))))
    keys = torch.from_numpy(W.uniform_keys(seed, n_max).view("int64")).cuda()
    out = {"device": torch.cuda.get_device_name(), "tcf": {}, "gqf": {}}
    for lg in tcf_classes:
        out["tcf"][str(lg)] = tune_tcf(lg, keys, torch)
    for q in gqf_classes:
        out["gqf"][str(q)] = tune_gqf(q, keys, torch)
    del keys
    torch.cuda.empty_cache()
    lg, entry = tune_tcf_group(torch)
    out["tcf_group"] = {str(lg): entry}
    torch.cuda.empty_cache()
    if path:
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        _table = None
    return out


if __name__ == "__main__":
    print(json.dumps(autotune(), indent=1))
