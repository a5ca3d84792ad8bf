#!/usr/bin/env python
"""Throughput benchmark of the filter hot path on GB300.

One step = every operation of the hot path over one pass of the paper-scale
workloads, all through the C ABI:
  TCF, 2^26 slots, 16-bit tags, bulk mode: empty the table; insert
    floor(0.9 * 2^26) uniform keys in 2^22-key batches; query 2^24 inserted
    keys and 2^24 fresh keys; delete a random half of the inserted keys in
    2^22-key batches; query the 2^25 probes again.
  Counting GQF, 2^28 slots, 8-bit remainders: empty the table; insert 2.4e8
    Zipf(1.0) keys over a 2^32 universe in one batch; count 2^24 keys sampled
    from the stream; delete those 2^24 keys (one copy each); count them again.
value = operations per second over the whole step (inserts + queries +
deletes + counts), inputs resident in HBM. Inputs (2.9 GB of keys) exceed the
L2 (129 MB), so no explicit L2 flush is done between steps.

--impl reference times the CPU oracle (tests only, single thread) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "insert & query Gops/s at 90% load, % of HBM/L2 roofline; batched/served p99"
UNIT = "Gops/s"
WORKLOAD = ("TCF 2^26 slots f=16 bulk: 15 x 2^22-key insert batches to 90% load, 2^24 pos + 2^24 neg "
            "queries, delete random half, re-query; counting GQF 2^28 slots r=8: insert 2.4e8 "
            "Zipf(1.0) keys over 2^32, count 2^24 sampled keys, delete them, re-count")

# Algorithmic bytes per work unit of each kernel (units are what the library
# records per launch: keys, slots, blocks or buckets).
BYTES_PER_UNIT = {
    "rs_scatter": 16.0,          # key read + key write
    "rs_scatter_kv": 24.0,       # key + index read and write
    "rs_hist": 8.0,              # key read
    "scan_kernel": 8.0,          # u32 read + write
    "rs_fp_hist": 16.0,          # key read + fingerprint write (the first pass's histogram comes free)
    "rle_kernel": 8.0,           # sorted fingerprint read (group writes not counted)
    "gqf_merge_kernel": 1.0,     # unit = algorithmic byte, counted on the device: old table read + new
                                 # table write (r / 8 + 1 / 2 B per slot each) + 12 B per group read
    "gqf_count_kernel": 80.0,    # key + metadata sector + remainder sector + count
    "gqf_status_kernel": 13.0,
    "tcf_query_kernel": 73.0,    # key + two 32-byte blocks + found byte
    "tcf_query_values_kernel": 73.0,  # key + two 32-byte blocks + value byte (bucket reads not counted)
    "gqf_counts_sorted": 8.0,    # counts carried by the sort: sorted count read + write
    "gqf_counts_gather": 12.0,   # with statuses: sorted index read + count gather + sorted count write
    "tcf_group_hist": 8.0,       # key read
    "tcf_group_scatter": 16.0,   # key read + record write
    "tcf_group_hist_sparse": 12.0,     # per candidate (counted on the device): pending entry + key read
    "tcf_group_scatter_sparse": 20.0,  # per candidate: pending entry + key read + record write
    "tcf_alloc": 24.0,           # per touched destination: list + count read, offset + list + segment write
    "tcf_block_insert": 74.0,    # per block with candidates (counted on the device): offsets + fill
                                 # read and write + 32-byte block read and write (records not counted)
    "tcf_block_remove": 74.0,
    "tcf_block_insert_sparse": 74.0,
    "tcf_block_remove_sparse": 74.0,
    "tcf_bucket_insert": 136.0,  # per bucket with candidates: segment + 64-byte bucket read and write
    "tcf_bucket_remove": 136.0,
    "tcf_tile_hist": 8.0,        # key read (tile histogram through shared memory)
    "tcf_tile_hist_pend": 12.0,  # pending record read
    "tcf_tile_part": 20.0,       # key read + 12-byte record write
    "tcf_tile_part_pend": 24.0,  # record read + record write
    "tcf_tile_part2": 24.0,      # record read + record write (second partition pass)
    "tcf_tile_insert": 1.0,      # unit = algorithmic byte, counted on the device: 12 per candidate read and
    "tcf_tile_remove": 1.0,      # per candidate left, 32 per block read, 32 per block written, 2 per fill
    "batch_gather": 16.0,        # key read + key write
    "batch_scatter": 9.0,        # result read + write (1 byte; counts: 16)
    "gqf_group_commit": 192.0,   # per 64-slot block: 32 B metadata + 64 B remainders, read and written (r = 8)
    "gqf_group_reject": 8.0,
    "tcf_point_insert": 104.0,
    "tcf_point_remove": 104.0,
    # filter groups
    "tcf_group_prep": 32.0,            # key read + 24-byte prepared key write
    "tcf_group_query_kernel": 73.0,
    "gqf_group_fp_kernel": 16.0,
    "gqf_merge_group_kernel": 1.0,
    "gqf_group_count_kernel": 73.0,    # key + metadata sector + remainder sector + found byte
}

# Algorithmic bytes of one operation (the sectors it must touch, plus its key
# and result; sort traffic excluded): 32-byte sectors as the filters lay them
# out, and the same count with every 32-byte sector taken as a 64-byte DRAM
# access (a random 32-byte read can cost a whole 64-byte burst).
OP_BYTES = {
    "tcf_insert": (104, 200),   # key + two 32 B blocks read + one written
    "tcf_query": (73, 137),     # key + two 32 B blocks + found byte
    "tcf_delete": (104, 200),
    "gqf_insert": (136, 264),   # key + metadata and remainder sectors read and written
    "gqf_query": (73, 137),     # key + metadata sector + remainder sector + found byte
    "gqf_count": (80, 144),     # key + metadata sector + remainder sector + 8-byte count
    "gqf_delete": (136, 264),
}


class OpTimer:
    """CUDA events around every operation call of the timed steps, on the
    stream the library launches on (torch's current stream). Per operation:
    the keys it processed and its summed device time, which includes any
    host round trip inside the call (the GQF insert and delete read their
    group count back)."""

    def __init__(self, torch):
        self.torch = torch
        self.rec = []
        self.on = False

    def op(self, name, n):
        timer = self

        class _Scope:
            def __enter__(self_):
                if timer.on:
                    self_.e = (timer.torch.cuda.Event(enable_timing=True), timer.torch.cuda.Event(enable_timing=True))
                    self_.e[0].record()

            def __exit__(self_, *a):
                if timer.on:
                    self_.e[1].record()
                    timer.rec.append((name, int(n), self_.e))

        return _Scope()

    def summary(self, peak_gbs):
        self.torch.cuda.synchronize()
        agg = {}
        for name, n, (a, b) in self.rec:
            x = agg.setdefault(name, [0, 0.0])
            x[0] += n
            x[1] += a.elapsed_time(b)
        out = {}
        for name, (n, ms) in agg.items():
            b32, b64 = OP_BYTES[name]
            rate = n / (ms / 1e3)
            out[name] = {"keys": n, "ms": round(ms, 3), "gops": round(rate / 1e9, 3),
                         "bytes_per_op": b32, "achieved_gbs": round(rate * b32 / 1e9, 1),
                         "frac": round(rate * b32 / 1e9 / peak_gbs, 4),
                         "bytes_per_op_64b": b64, "frac_64b": round(rate * b64 / 1e9 / peak_gbs, 4)}
        return out


BATCHED_WORKLOAD = ("4096 filters: 2048 TCF f=16 bulk + 2048 counting GQF r=8, 2^e slots with e uniform in "
                    "10..20, 85-95% load (7.2e8 keys in total); TCF keys inserted in 8 rounds, GQF keys in "
                    "one batch; then every filter's own keys and as many fresh keys are queried; one group "
                    "call per kind and operation")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batched", action="store_true", help="skip the 4096-filter group measurement")
    ap.add_argument("--no-target", action="store_true", help="skip the 2^28-slot, 90%%-load measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the reduced serving-loop measurement")
    ap.add_argument("--no-tcf-point", action="store_true", help="skip the point-mode TCF (Alg. 1) measurement")
    ap.add_argument("--no-geometry", action="store_true", help="skip the TCF block-geometry sweep and the GQF point updates")
    ap.add_argument("--case", default="full", choices=["full", "profile", "target", "batched", "serving", "kmer", "values"],
                    help="profile: a reduced copy of the workload (TCF 2^24, GQF 2^25 with 3e7 Zipf "
                         "keys) that fits an ncu capture; its line is not the benchmark figure")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# ranks: one process per GPU, replicas of the whole step (weak scaling)
# ---------------------------------------------------------------------------
def rank_env():
    """(rank, world, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(ops_per_step: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput in Gops/s: every rank did `steps` full steps."""
    return ops_per_step * steps * world / (ms_max / 1e3) / 1e9


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
PROFILE_WORKLOAD = ("reduced copy for ncu captures: TCF 2^24 slots f=16 bulk, 2^20-key batches, 2^22 + 2^22 "
                    "queries; counting GQF 2^25 slots r=8, 3e7 Zipf(1.0) keys, 2^22 counts")


def make_inputs(case: str = "full"):
    from paper_2212_09005_gb300 import workloads as W

    if case == "target":
        t = W.tcf_workload(log2_slots=28, seed=8, batch=1 << 24, n_query=1 << 24)
        g = W.gqf_target_workload(q=28, seed=9, n_query=1 << 24)
        ins = t["insert"]
        gi = g["insert"]
        return {
            "tcf_ins": ins, "tcf_batch": t["batch"], "tcf_probe": np.concatenate([ins[t["pos_idx"]], t["negatives"]]),
            "tcf_del": ins[t["del_idx"]], "tcf_log2": 28, "tcf_seed": 8, "gqf_qbits": 28, "gqf_seed": 9,
            "gqf_ins": gi, "gqf_q": np.concatenate([gi[g["pos_idx"]], g["negatives"]]), "gqf_del": gi[g["del_idx"]],
            "n_pos": len(t["pos_idx"]), "n_gpos": len(g["pos_idx"]),
        }
    if case == "profile":
        t = W.tcf_workload(log2_slots=24, batch=1 << 20, n_query=1 << 22)
        g = W.gqf_zipf_workload(q=25, n=30_000_000, n_query=1 << 22)
    else:
        t = W.tcf_workload()
        g = W.gqf_zipf_workload()
    ins = t["insert"]
    probe = np.concatenate([ins[t["pos_idx"]], t["negatives"]])
    dels = ins[t["del_idx"]]
    return {
        "tcf_ins": ins, "tcf_batch": t["batch"], "tcf_probe": probe, "tcf_del": dels,
        "tcf_log2": t["log2_slots"], "gqf_qbits": g["q"],
        "gqf_ins": g["insert"], "gqf_q": g["query"], "n_pos": len(t["pos_idx"]),
    }


def ops_per_step(inp):
    n = len(inp["tcf_ins"]) + 2 * len(inp["tcf_probe"]) + len(inp["tcf_del"]) + len(inp["gqf_ins"])
    if "gqf_del" in inp:  # count, query, delete, count
        return n + 3 * len(inp["gqf_q"]) + len(inp["gqf_del"])
    return n + 3 * len(inp["gqf_q"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic():
    """Per-kernel DRAM bytes per work unit from the committed ncu summary."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    out = {}
    if os.path.exists(p):
        for line in open(p):
            line = line.split("#", 1)[0].split()
            if len(line) >= 3:
                out[line[0]] = (float(line[1]), float(line[2]))  # units per launch, bytes per launch
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
class Runner:
    def __init__(self, inp, device):
        import torch

        import paper_2212_09005_gb300 as gf

        self.gf, self.torch, self.inp = gf, torch, inp
        self.dev = device
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
        self.target = "gqf_del" in inp
        names = ("tcf_ins", "tcf_probe", "tcf_del", "gqf_ins", "gqf_q") + (("gqf_del",) if self.target else ())
        self.d = {k: to(inp[k]) for k in names}
        self.found = torch.zeros(len(inp["tcf_probe"]), dtype=torch.uint8, device=device)
        self.found2 = torch.zeros_like(self.found)
        self.cnt = torch.zeros(len(inp["gqf_q"]), dtype=torch.int64, device=device)
        self.cnt2 = torch.zeros_like(self.cnt)
        self.gfound = torch.zeros(len(inp["gqf_q"]), dtype=torch.uint8, device=device)
        self.timer = OpTimer(torch)
        self.B = inp["tcf_batch"]
        self.tcf = gf.TCF(inp["tcf_log2"], 16, gf.MODE_BULK, seed=inp.get("tcf_seed", 2), max_batch=self.B)
        self.gqf = gf.GQF(inp["gqf_qbits"], 8, seed=inp.get("gqf_seed", 3), max_batch=len(inp["gqf_ins"]))

    def step(self, src=None, wait=None):
        """One pass of the hot path. `src` maps input names to device tensors;
        `wait(name, k)` (optional) is called before input `name` (batch k) is
        first used, so that its host->device copy can still be in flight."""
        d = src or self.d
        w = wait or (lambda name, k=0: None)
        op = self.timer.op
        tcf, gqf, B = self.tcf, self.gqf, self.B
        tcf.clear()
        ins = d["tcf_ins"]
        for k, s in enumerate(range(0, ins.numel(), B)):
            w("tcf_ins", k)
            b = ins[s:s + B]
            with op("tcf_insert", b.numel()):
                tcf.insert(b)
        w("tcf_probe")
        with op("tcf_query", d["tcf_probe"].numel()):
            tcf.query(d["tcf_probe"], self.found)
        dl = d["tcf_del"]
        for k, s in enumerate(range(0, dl.numel(), B)):
            w("tcf_del", k)
            b = dl[s:s + B]
            with op("tcf_delete", b.numel()):
                tcf.remove(b)
        with op("tcf_query", d["tcf_probe"].numel()):
            tcf.query(d["tcf_probe"], self.found2)
        gqf.clear()
        w("gqf_ins")
        with op("gqf_insert", d["gqf_ins"].numel()):
            gqf.insert(d["gqf_ins"])
        w("gqf_q")
        q = d["gqf_q"]
        with op("gqf_count", q.numel()):
            gqf.count(q, self.cnt)
        if self.target:
            with op("gqf_query", q.numel()):
                gqf.query(q, self.gfound)
            dq = d["gqf_del"]
        else:
            dq = q
        with op("gqf_delete", dq.numel()):
            gqf.remove(dq)
        with op("gqf_count", q.numel()):
            gqf.count(q, self.cnt2)

    def _recount_ok(self):
        if self.target:
            # distinct inserted keys were deleted: counts only fall, and the
            # query answers are count > 0
            c1, c2 = self.cnt.cpu().numpy(), self.cnt2.cpu().numpy()
            f = self.gfound.cpu().numpy()
            return bool((c2 <= c1).all() and np.array_equal(f != 0, c1 > 0))
        # each sampled key was deleted once per occurrence in the sample
        q = self.inp["gqf_q"]
        u, inv, occ = np.unique(q, return_inverse=True, return_counts=True)
        before = self.cnt.cpu().numpy()
        after = self.cnt2.cpu().numpy()
        return bool((after == np.maximum(before - occ[inv], 0)).all())

    def checks(self):
        """Cheap correctness guards on the last step's results."""
        t = self.torch
        t.cuda.synchronize()
        npos = self.inp["n_pos"]
        st_t, st_g = self.tcf.stats(), self.gqf.stats()
        ok = {
            "tcf_pos_found": bool(self.found[:npos].all().item()),
            "tcf_fpr": float(self.found[npos:].float().mean().item()),
            "gqf_counts_pos": bool((self.cnt[:self.inp.get("n_gpos", len(self.cnt))] >= 1).all().item()),
            "gqf_recount_ok": self._recount_ok(),
            "tcf_status_word": st_t["status_word"], "gqf_status_word": st_g["status_word"],
            "tcf_backing_used": st_t["backing_used"],
        }
        return ok


def traced_steps(step, steps):
    """Per-kernel split: the same steps again with the library's kernel trace
    on (CUDA events around every launch, on the launching stream). Kept out
    of the timed region, whose step time the extra event records would
    lengthen."""
    import torch

    import paper_2212_09005_gb300 as gf

    torch.cuda.synchronize()
    gf.trace_reset()
    gf.trace_enable(True)
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    gf.trace_enable(False)
    return gf.trace_summary()


def run_ours(args, rank, world, device_index):
    import torch
    import torch.distributed as dist

    import paper_2212_09005_gb300 as gf

    torch.cuda.set_device(device_index)
    device = torch.device("cuda", device_index)
    inp = make_inputs(args.case)
    R = Runner(inp, device)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        R.step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(device_index)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    R.timer.on = True
    e0.record(stream)
    for _ in range(args.steps):
        R.step()
    e1.record(stream)
    torch.cuda.synchronize()
    R.timer.on = False
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    per_op = R.timer.summary(peaks()[0])
    trace = traced_steps(R.step, args.steps)
    if world > 1:
        dist.barrier()
    checks = R.checks()
    ops = ops_per_step(inp)
    value = aggregate_rate(ops, args.steps, world, ms)

    kern, roof = roofline_from_trace(trace)
    launches = sum(v["launches"] for v in trace.values())
    gather = query_vs_gather(kern, {"tcf_query_kernel": R.tcf.stats()["table_bytes"],
                                    "gqf_count_kernel": R.gqf.stats()["table_bytes"]}, device)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(R, args, world, device)

    tcf_point = None
    if args.case == "full" and not args.no_tcf_point:
        tcf_point = run_tcf_point(inp, device)

    target = None
    if args.case == "full" and not args.no_target:
        del R
        torch.cuda.empty_cache()
        target = run_target(args, device)

    batched = None
    if args.case == "full" and not args.no_batched:
        R = None
        torch.cuda.empty_cache()
        batched = run_batched(args, device)

    serving = None
    if args.case == "full" and not args.no_serving:
        R = None
        torch.cuda.empty_cache()
        serving = run_serving(args, device, log2_slots=20, bmax=20, workload=SERVING_SMALL)

    geometry = None
    if args.case == "full" and not args.no_geometry:
        R = None
        torch.cuda.empty_cache()
        geometry = run_geometry(args, device)

    point = None
    if args.case == "full" and not args.no_geometry:
        torch.cuda.empty_cache()
        point = run_point_gqf(args, device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.case == "full":
        cpu = cpu_sample(inp)

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded SplitMix64 uniform keys, Zipf rejection-inversion keys)",
        "config": {"workload": {"full": WORKLOAD, "profile": PROFILE_WORKLOAD, "target": TARGET_WORKLOAD}[args.case],
                   "ops_per_step": ops, "tcf_mode": "bulk (deterministic)",
                   "l2": "inputs larger than L2 (2.9 GB of keys), no flush", "parallelism": f"replicas x{world}"},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
        "cpu_baseline": cpu, "random_gather": gather, "per_op": per_op, "kernels": kern, "checks": checks,
        "target_2_28": target, "batched": batched, "serving": serving, "tcf_geometry": geometry, "gqf_point": point,
        "tcf_point": tcf_point,
    }
    return line


TARGET_WORKLOAD = ("target size, 2^28 slots at 90% load: TCF f=16 bulk, floor(0.9 * 2^28) uniform keys in 2^24-key "
                   "batches, 2^24 pos + 2^24 neg queries, delete a random half in 2^24-key batches, re-query; GQF "
                   "r=8, as many uniform keys in one batch, count and query 2^24 inserted + 2^24 fresh keys, delete "
                   "2^24 distinct inserted keys, re-count")


POINT_WORKLOAD = ("GQF point updates (paper Sec. 5.2 point API, one thread per key, region locks) against the bulk "
                  "path on the same keys: 2^24 home slots, r=8, 2^20 distinct uniform keys (6 % load) inserted in one "
                  "call into an empty table, then half of them removed in one call. Point updates serialise per "
                  "8192-quotient region and shift clusters slot by slot, so they suit small scattered updates; "
                  "filling 2^24 home slots to 85 % this way takes 2.3 s against 0.9 ms in bulk "
                  "(tests/test_gpu_gqf_point.py covers that load for parity)")


def run_point_gqf(args, device, q=24, n=1 << 20):
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    k = torch.from_numpy(W.uniform_keys(41, n).view(np.int64)).to(device)
    half = k[: n // 2]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": POINT_WORKLOAD}
    imgs = []
    for mode in ("point", "bulk"):
        G = gf.GQF(q, 8, seed=42, max_batch=n)
        best = None
        for rep in range(3):
            G.clear()
            torch.cuda.synchronize()
            a, m, z = ev(), ev(), ev()
            a.record()
            if mode == "point":
                G.point_update(k)
            else:
                G.insert(k)
            m.record()
            if mode == "point":
                G.point_update(half, remove=True)
            else:
                G.remove(half)
            z.record()
            torch.cuda.synchronize()
            t = (a.elapsed_time(m), m.elapsed_time(z))
            best = t if best is None or sum(t) < sum(best) else best
        st = G.stats()
        imgs.append(G.export())
        out[mode] = {"insert_ms": round(best[0], 3), "insert_gops": round(n / best[0] / 1e6, 3),
                     "remove_ms": round(best[1], 3), "remove_gops": round((n // 2) / best[1] / 1e6, 3),
                     "status_word": st["status_word"], "failed_keys": st["failed_keys"]}
        G.close()
    out["tables_equal"] = bool(np.array_equal(imgs[0], imgs[1]))
    return out


TCF_POINT_WORKLOAD = ("TCF point mode (paper Alg. 1: one thread per key, a compare-and-swap into the first empty "
                      "slot of b1 under the shortcut, else of the less full of b1 and b2, else a backing bucket; "
                      "delete swaps in a tombstone) on the main step's TCF keys: 2^26 slots f=16, the same 15 "
                      "insert batches, 2^24 pos + 2^24 neg queries, the same random-half delete, re-query")


def run_tcf_point(inp, device, reps: int = 3):
    """Per-operation rates of the point-mode TCF on the main step's TCF
    inputs, best of `reps` passes after one warm-up pass. The table of a
    point-mode TCF depends on the order of the threads' compare-and-swaps,
    so the checks are the ones that hold for any order: every inserted key
    is found before the delete, every key not deleted after it, and no
    key is refused."""
    import torch

    import paper_2212_09005_gb300 as gf

    to = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
    ins, probe, dels, B = to(inp["tcf_ins"]), to(inp["tcf_probe"]), to(inp["tcf_del"]), inp["tcf_batch"]
    npos = inp["n_pos"]
    f1 = torch.zeros(probe.numel(), dtype=torch.uint8, device=device)
    f2 = torch.zeros_like(f1)
    T = gf.TCF(inp["tcf_log2"], 16, gf.MODE_POINT, seed=inp.get("tcf_seed", 2), max_batch=B)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    best = None
    for rep in range(reps + 1):
        T.clear()
        torch.cuda.synchronize()
        e = [ev() for _ in range(5)]
        e[0].record()
        for s in range(0, ins.numel(), B):
            T.insert(ins[s:s + B])
        e[1].record()
        T.query(probe, f1)
        e[2].record()
        for s in range(0, dels.numel(), B):
            T.remove(dels[s:s + B])
        e[3].record()
        T.query(probe, f2)
        e[4].record()
        torch.cuda.synchronize()
        t = [e[k].elapsed_time(e[k + 1]) for k in range(4)]
        if rep > 0 and (best is None or sum(t) < sum(best)):
            best = t
    st = T.stats()
    peak = peaks()[0]
    n_ops = {"tcf_insert": (ins.numel(), best[0]), "tcf_query": (2 * probe.numel(), best[1] + best[3]),
             "tcf_delete": (dels.numel(), best[2])}
    per_op = {}
    for name, (n, ms) in n_ops.items():
        b32, b64 = OP_BYTES[name]
        rate = n / (ms / 1e3)
        per_op[name] = {"keys": n, "ms": round(ms, 3), "gops": round(rate / 1e9, 3), "bytes_per_op": b32,
                        "frac": round(rate * b32 / 1e9 / peak, 4), "frac_64b": round(rate * b64 / 1e9 / peak, 4)}
    # the positives are a sample of the inserted keys; deleted ones are
    # those of the sample that appear in the delete set
    pos = inp["tcf_probe"][:npos]
    kept = ~np.isin(pos, inp["tcf_del"])
    f1h, f2h = f1.cpu().numpy(), f2.cpu().numpy()
    checks = {"pos_found": bool(f1h[:npos].all()), "kept_found_after_delete": bool(f2h[:npos][kept].all()),
              "fpr": round(float(f1h[npos:].mean()), 6), "failed_keys": st["failed_keys"],
              "status_word": st["status_word"], "backing_used": st["backing_used"]}
    T.close()
    total_ms = sum(best)
    total_ops = ins.numel() + 2 * probe.numel() + dels.numel()
    return {"workload": TCF_POINT_WORKLOAD, "gops": round(total_ops / total_ms / 1e6, 3),
            "ms": round(total_ms, 3), "per_op": per_op, "checks": checks}


GEOMETRY_WORKLOAD = ("TCF block-geometry sweep (paper Sec. 4.1 block sizes, Sec. 4.2 128-slot blocks, 12-bit tags): "
                     "per (tag bits, slots per block), a bulk TCF of 2^24 slots (nb the largest power of two with "
                     "nb * B <= 2^24) filled to 90% with uniform keys in 2^21-key batches, 2^22 positive + 2^22 "
                     "fresh queries, then a random half deleted in 2^21-key batches")
GEOMETRIES = [(16, 16), (16, 8), (16, 32), (16, 64), (16, 128), (12, 21), (8, 32), (8, 64)]


def run_geometry(args, device, log2_slots=24, batch=1 << 21, nq=1 << 22):
    """Insert, query and delete rates per block geometry, with the measured
    false-positive rate; one timed pass after one warm-up pass per geometry."""
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    keys = torch.from_numpy(W.uniform_keys(31, int(0.9 * (1 << log2_slots))).view(np.int64)).to(device)
    neg = torch.from_numpy(W.uniform_keys(32, nq).view(np.int64)).to(device)
    found = torch.zeros(nq, dtype=torch.uint8, device=device)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    rows = []
    for f, B in GEOMETRIES:
        F = gf.TCF(log2_slots, f, gf.MODE_BULK, seed=33, max_batch=batch, block_slots=0 if B * f == 256 and f != 12 else B)
        n = min(int(0.9 * F.stats()["nslots"]), keys.numel())
        ins = [keys[i:min(i + batch, n)] for i in range(0, n, batch)]
        dels = [keys[i:min(i + batch, n // 2)] for i in range(0, n // 2, batch)]
        pos = keys[: min(nq, n)]
        for rep in range(2):  # warm-up, then the timed pass
            F.clear()
            t = [ev() for _ in range(5)]
            t[0].record()
            for k in ins:
                F.insert(k)
            t[1].record()
            F.query(pos, found[: pos.numel()])
            t[2].record()
            F.query(neg, found)
            t[3].record()
            for k in dels:
                F.remove(k)
            t[4].record()
            torch.cuda.synchronize()
        fpr = float(found.float().mean().item())
        ms = [t[i].elapsed_time(t[i + 1]) for i in range(4)]
        st = F.stats()
        rows.append({"tag_bits": f, "block_slots": B, "block_bytes": int((f * B + 255) // 256 * 32),
                     "nslots": st["nslots"], "keys": n,
                     "insert_gops": round(n / ms[0] / 1e6, 3), "query_gops": round((pos.numel() + nq) / (ms[1] + ms[2]) / 1e6, 3),
                     "delete_gops": round((n // 2) / ms[3] / 1e6, 3), "fpr": round(fpr, 6),
                     "backing_used": st["backing_used"], "failed_keys": st["failed_keys"]})
        F.close()
    return {"workload": GEOMETRY_WORKLOAD, "rows": rows}


def run_target(args, device):
    """Both filters at the target size, every operation timed on its own
    (same step structure as the main workload)."""
    import torch

    import paper_2212_09005_gb300 as gf

    inp = make_inputs("target")
    R = Runner(inp, device)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        R.step()
    torch.cuda.synchronize()
    clocks = ClockSampler(device.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R.timer.on = True
    e0.record(stream)
    for _ in range(args.steps):
        R.step()
    e1.record(stream)
    torch.cuda.synchronize()
    R.timer.on = False
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    trace = traced_steps(R.step, args.steps)
    ops = ops_per_step(inp)
    kern, roof = roofline_from_trace(trace, with_traffic=False)
    out = {"workload": TARGET_WORKLOAD, "value": round(aggregate_rate(ops, args.steps, 1, ms), 4), "unit": UNIT,
           "ms_per_step": round(ms / args.steps, 3), "ops_per_step": ops, "clocks": clk,
           "per_op": R.timer.summary(peaks()[0]), "gpu_launches": sum(v["launches"] for v in trace.values()),
           "roofline": roof, "kernels": kern[:12], "checks": R.checks()}
    del R
    torch.cuda.empty_cache()
    return out


def gather_peak(footprint_bytes: int, device, sectors_per_key: int = 2, n: int = 1 << 24) -> float:
    """Throughput (GB/s of 8 + 32 * spk + 1 bytes per key) of random 32-byte
    gathers over a table of the given footprint: the query access pattern
    without filter arithmetic, timed with CUDA events (best of 5)."""
    import torch

    import paper_2212_09005_gb300 as gf

    table = torch.zeros(footprint_bytes, dtype=torch.uint8, device=device)
    keys = torch.randint(-(1 << 62), 1 << 62, (n,), dtype=torch.int64, device=device)
    out = torch.empty(n, dtype=torch.uint8, device=device)
    for _ in range(3):
        gf.calibrate_gather(table, keys, out, sectors_per_key)
    best = float("inf")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        e0.record()
        gf.calibrate_gather(table, keys, out, sectors_per_key)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del table, keys, out
    return (8 + 32 * sectors_per_key + 1) * n / (best / 1e3) / 1e9


def query_vs_gather(kern, footprints, device):
    """The query kernels against the random-gather roofline at their table footprint."""
    out = {}
    for name, fp in footprints.items():
        k = next((x for x in kern if x["kernel"] == name), None)
        if k is None or not k["achieved_gbs"]:
            continue
        g = gather_peak(fp, device)
        out[name] = {"footprint_mib": round(fp / 2**20, 1), "gather_gbs": round(g, 1),
                     "kernel_gbs": k["achieved_gbs"], "frac": round(k["achieved_gbs"] / g, 4)}
    return out


def roofline_from_trace(trace, with_traffic: bool = True):
    """Per-kernel shares and the roofline of the dominant kernel, from the live
    CUDA-event trace of the timed region. with_traffic: attach the ncu DRAM
    traffic recorded for this workload (cases without their own capture pass
    False and report null)."""
    peak, peak_src = peaks()
    traffic = ncu_traffic() if with_traffic else {}
    kern = []
    tot_ms = sum(v["ms"] for v in trace.values())
    for name, v in trace.items():
        bpu = BYTES_PER_UNIT.get(name)
        gbs = (bpu * v["units"] / (v["ms"] / 1e3) / 1e9) if (bpu and v["ms"] > 0) else None
        kern.append({"kernel": name, "launches": v["launches"], "units": v["units"], "ms": round(v["ms"], 3),
                     "share": round(v["ms"] / tot_ms, 4) if tot_ms else None,
                     "achieved_gbs": round(gbs, 1) if gbs else None})
    kern.sort(key=lambda k: -k["ms"])
    top = kern[0] if kern else None
    roof = None
    if top and top["achieved_gbs"]:
        name = top["kernel"]
        per_launch_units = trace[name]["units"] / trace[name]["launches"]
        tr = None
        if name in traffic:
            u, b = traffic[name]
            tr = round(b * per_launch_units / u) if u else None
        roof = {"bound": "hbm", "kernel": name, "achieved": top["achieved_gbs"], "peak": peak,
                "unit": "GB/s", "frac": round(top["achieved_gbs"] / peak, 4), "peak_source": peak_src,
                "traffic": tr, "algorithmic_bytes_per_launch": BYTES_PER_UNIT[name] * per_launch_units}
    return kern, roof


# ---------------------------------------------------------------------------
# batched filters (filter groups)
# ---------------------------------------------------------------------------
class BatchedRunner:
    """One step: empty both groups; insert the TCF keys in rounds and the GQF
    keys in one batch; query every filter's own keys and as many fresh keys."""

    def __init__(self, w, device):
        import torch

        import paper_2212_09005_gb300 as gf
        from paper_2212_09005_gb300 import workloads as W

        self.torch, self.w = torch, w
        off, keys, neg = w["offsets"], w["insert"], w["negatives"]
        logs, seeds, nt = w["log2_slots"], w["hash_seeds"], w["n_tcf"]
        to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
        toff = off[: nt + 1]
        goff = off[nt:] - off[nt]
        self.toff, self.goff = to_dev(toff), to_dev(goff)
        self.tkeys, self.tneg = to_dev(keys[: toff[-1]]), to_dev(neg[: toff[-1]])
        self.gkeys, self.gneg = to_dev(keys[off[nt]:]), to_dev(neg[off[nt]:])
        chunks = W.round_chunks(toff, w["tcf_rounds"])
        self.rounds = []
        for j in range(w["tcf_rounds"]):
            lens = chunks[j, :, 1] - chunks[j, :, 0]
            o = np.zeros(nt + 1, np.int64)
            np.cumsum(lens, out=o[1:])
            idx = np.concatenate([np.arange(a, b) for a, b in chunks[j]])
            self.rounds.append((to_dev(o), to_dev(keys[idx])))
        mt = max(int(r[1].numel()) for r in self.rounds)
        self.T = gf.FilterGroup(gf.FILTER_TCF, logs[:nt], 16, seeds[:nt], max_total=mt)
        self.G = gf.FilterGroup(gf.FILTER_GQF, logs[nt:], 8, seeds[nt:], max_total=int(self.gkeys.numel()))
        u8 = lambda n: torch.zeros(n, dtype=torch.uint8, device=device)
        self.tf, self.tfn = u8(self.tkeys.numel()), u8(self.tneg.numel())
        self.gf_, self.gfn = u8(self.gkeys.numel()), u8(self.gneg.numel())
        self.ops = int(off[-1]) * 3  # inserts, own-key queries, fresh-key queries
        # the same step as work lists: one list per TCF round, then one with the
        # TCF queries, the GQF insert and the GQF queries
        # the last list queries each group's own keys and as many fresh keys in one class
        self.B = gf.FilterBatch(self.T, self.G, max_keys=max(mt, 2 * int(self.tkeys.numel()), 2 * int(self.gkeys.numel())),
                                max_items=4 * len(logs))
        TB, GB = gf.BATCH_TCF, gf.BATCH_GQF
        self.lists = []
        for o, k in self.rounds:
            oh = o.cpu().numpy()
            self.lists.append([(TB, m, gf.OP_INSERT, k[oh[m]:oh[m + 1]], None) for m in range(nt)])
        last = []
        for m in range(nt):
            a, b = int(toff[m]), int(toff[m + 1])
            last.append((TB, m, gf.OP_QUERY, self.tkeys[a:b], self.tf[a:b]))
            last.append((TB, m, gf.OP_QUERY, self.tneg[a:b], self.tfn[a:b]))
        for m in range(len(logs) - nt):
            a, b = int(goff[m]), int(goff[m + 1])
            last.append((GB, m, gf.OP_INSERT, self.gkeys[a:b], None))
            last.append((GB, m, gf.OP_QUERY, self.gkeys[a:b], self.gf_[a:b]))
            last.append((GB, m, gf.OP_QUERY, self.gneg[a:b], self.gfn[a:b]))
        self.lists.append(last)
        self.graph = None

    def step_batch(self):
        self.T.clear()
        self.G.clear()
        for items in self.lists:
            self.B.run(items)

    def capture(self):
        torch = self.torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step_batch()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step_batch()

    def step_graph(self):
        self.graph.replay()

    def outputs(self):
        self.torch.cuda.synchronize()
        return [t.clone() for t in (self.tf, self.tfn, self.gf_, self.gfn)]

    def step(self):
        T, G = self.T, self.G
        T.clear()
        for o, k in self.rounds:
            T.insert(o, k)
        T.query(self.toff, self.tkeys, self.tf)
        T.query(self.toff, self.tneg, self.tfn)
        G.clear()
        G.insert(self.goff, self.gkeys)
        G.query(self.goff, self.gkeys, self.gf_)
        G.query(self.goff, self.gneg, self.gfn)

    def checks(self):
        self.torch.cuda.synchronize()
        st = self.T.stats(0)
        return {"tcf_own_found": float(self.tf.float().mean().item()),
                "tcf_failed_keys": st["failed_keys"],
                "tcf_fpr": float(self.tfn.float().mean().item()),
                "gqf_own_found": bool(self.gf_.all().item()),
                "gqf_fpr": float(self.gfn.float().mean().item())}


def run_single_filters(w, device, args):
    """The batched workload through one standalone filter per member and one
    call per filter and operation (the plain path the groups replace): one
    timed step after one warm-up step; sampled members' images are compared
    with a group's."""
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    off, keys, neg = w["offsets"], w["insert"], w["negatives"]
    logs, seeds, nt, rounds = w["log2_slots"], w["hash_seeds"], w["n_tcf"], w["tcf_rounds"]
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
    dk, dn = to_dev(keys), to_dev(neg)
    found = torch.zeros(int(off[-1]), dtype=torch.uint8, device=device)
    chunks = W.round_chunks(off[: nt + 1], rounds)
    fs = []
    for m in range(len(logs)):
        n = int(off[m + 1] - off[m])
        if m < nt:
            mb = max(1, int((chunks[:, m, 1] - chunks[:, m, 0]).max()))
            fs.append(gf.TCF(int(logs[m]), 16, gf.MODE_BULK, seed=int(seeds[m]), max_batch=mb))
        else:
            fs.append(gf.GQF(int(logs[m]), 8, seed=int(seeds[m]), max_batch=max(1, n)))

    def step():
        for f in fs:
            f.clear()
        for j in range(rounds):
            for m in range(nt):
                a, b = int(chunks[j, m, 0]), int(chunks[j, m, 1])
                if b > a:
                    fs[m].insert(dk[a:b])
        for m in range(len(logs)):
            a, b = int(off[m]), int(off[m + 1])
            if b == a:
                continue
            if m >= nt:
                fs[m].insert(dk[a:b])
            fs[m].query(dk[a:b], found[a:b])
            fs[m].query(dn[a:b], found[a:b])

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ops = int(off[-1]) * 3
    # members sampled against a group built the same way
    T = gf.FilterGroup(gf.FILTER_TCF, logs[:nt], 16, seeds[:nt], max_total=int(off[nt]))
    G = gf.FilterGroup(gf.FILTER_GQF, logs[nt:], 8, seeds[nt:], max_total=int(off[-1] - off[nt]))
    for j in range(rounds):
        lens = chunks[j, :, 1] - chunks[j, :, 0]
        o = np.zeros(nt + 1, np.int64)
        np.cumsum(lens, out=o[1:])
        idx = np.concatenate([np.arange(a, b) for a, b in chunks[j]])
        T.insert(to_dev(o), to_dev(keys[idx]))
    G.insert(to_dev(off[nt:] - off[nt]), dk[int(off[nt]):])
    same = all(np.array_equal(fs[m].export(), T.export(m)) for m in range(0, nt, 97)) and \
        all(np.array_equal(fs[m].export(), G.export(m - nt)) for m in range(nt, len(logs), 97))
    del fs, T, G, dk, dn, found
    torch.cuda.empty_cache()
    return {"seconds_per_step": round(sec, 3), "value": round(ops / sec / 1e9, 4), "filters": len(logs),
            "member_images_equal_group": bool(same), "sample": "every 97th member of each kind"}


def run_batched(args, device):
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    R = BatchedRunner(W.batched_workload(), device)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        R.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        R.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    trace = traced_steps(R.step, args.steps)
    kern, roof = roofline_from_trace(trace)
    gather = query_vs_gather(kern, {"tcf_group_query_kernel": sum(R.T.export_size(m) for m in range(R.T.n)),
                                    "gqf_group_count_kernel": sum(R.G.export_size(m) for m in range(R.G.n))}, device)
    out = {"workload": BATCHED_WORKLOAD, "value": round(aggregate_rate(R.ops, args.steps, 1, ms), 4), "unit": UNIT,
           "ms_per_step": round(ms / args.steps, 3), "ops_per_step": R.ops,
           "gpu_launches": sum(v["launches"] for v in trace.values()), "roofline": roof,
           "random_gather": gather, "kernels": kern, "checks": R.checks()}
    ref = R.outputs()
    img_t, img_g = R.T.export(0), R.G.export(0)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    # the work-list form of the same step, run directly and replayed from one CUDA graph
    ms_b = timed(R.step_batch)
    same_b = all(torch.equal(x, y) for x, y in zip(R.outputs(), ref))
    R.capture()
    ms_g = timed(R.step_graph)
    same_g = all(torch.equal(x, y) for x, y in zip(R.outputs(), ref))
    same_img = bool(np.array_equal(R.T.export(0), img_t) and np.array_equal(R.G.export(0), img_g))
    out["work_list"] = {"ms_per_step": round(ms_b, 3), "value": round(R.ops / (ms_b / 1e3) / 1e9, 4),
                        "answers_equal_group_calls": bool(same_b),
                        "graph": {"ms_per_step": round(ms_g, 3), "value": round(R.ops / (ms_g / 1e3) / 1e9, 4),
                                  "answers_equal_group_calls": bool(same_g), "member_images_equal": same_img},
                        "calls_per_step": len(R.lists)}
    w = R.w
    R.graph = None
    R.B.close()
    del R
    torch.cuda.empty_cache()
    out["single_filter_calls"] = run_single_filters(w, device, args)
    if not args.no_cpu:
        try:
            out["cpu_baseline"] = cpu_batched_sample(w)
        except Exception as e:  # the GPU figures stand without it
            out["cpu_baseline"] = {"error": f"{type(e).__name__}: {e}"}
    return out


KMER_WORKLOAD = ("k-mer counting: counting GQF 2^28 slots r=8; one batch of 2e8 canonical 28-mers of synthetic "
                 "100-base reads (random genome of 2^25 bases, about 6x k-mer coverage, 0.5% substitution errors), "
                 "then 2^24 count queries on k-mers sampled from the batch")
KMER_N = 200_000_000
PAPER_KMER_2_28 = 507.373  # M k-mers/s, the paper's GQF counting table at 2^28 slots (other hardware)


def run_kmer(args, device):
    """GQF counting insert of synthetic k-mers: the paper's k-mer count column
    (Table of GQF counting inserts), on generated reads."""
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    kmers = W.kmer_workload(KMER_N)
    qpos = W.sample_with_replacement(6 * 1000 + 3, len(kmers), 1 << 24)
    kd = torch.from_numpy(kmers.view(np.int64)).to(device)
    qd = torch.from_numpy(kmers[qpos].view(np.int64)).to(device)
    cnt = torch.zeros(len(qpos), dtype=torch.int64, device=device)
    G = gf.GQF(28, 8, seed=6, max_batch=len(kmers))
    stream = torch.cuda.current_stream()

    ins_ev = []

    def step(timed=False):
        G.clear()
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        G.insert(kd)
        if timed:
            b.record(stream)
            ins_ev.append((a, b))
        G.count(qd, cnt)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    gf.trace_reset()
    gf.trace_enable(True)
    clocks = ClockSampler(device.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(timed=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    gf.trace_enable(False)
    trace = gf.trace_summary()
    ms = e0.elapsed_time(e1)
    kern, roof = roofline_from_trace(trace, with_traffic=False)
    ins_ms = sum(a.elapsed_time(b) for a, b in ins_ev) / len(ins_ev)
    st = G.stats()
    c = cnt.cpu().numpy()
    out = {"workload": KMER_WORKLOAD, "value": round(aggregate_rate(len(kmers) + len(qpos), args.steps, 1, ms), 4),
           "unit": UNIT, "ms_per_step": round(ms / args.steps, 3), "ops_per_step": len(kmers) + len(qpos),
           "insert_mkmers_per_s": round(len(kmers) / ins_ms / 1e3, 1),
           "paper_kmer_count_2_28_mkmers_per_s": PAPER_KMER_2_28,
           "clocks": clk, "gpu_launches": sum(v["launches"] for v in trace.values()), "roofline": roof,
           "kernels": kern,
           "checks": {"counts_positive": bool((c >= 1).all()), "failed_keys": st["failed_keys"],
                      "status_word": st["status_word"]}}
    del G, kd, qd, cnt
    torch.cuda.empty_cache()
    return out


VALUES_WORKLOAD = ("values: TCF 2^26 slots f=16 bulk with 4-bit values (12-bit tags): 15 x 2^22-key insert "
                   "batches with values to 90% load, then 2^25 value queries (half inserted keys, half fresh); "
                   "counting GQF 2^28 slots r=8: one counted insert of 2^25 + 2^24 uniform keys below 2^32 "
                   "with counts 1..8 (about 66% of the slots: a count of 2 or more takes 3 or 4), then 2^24 "
                   "counts of inserted keys")


def run_values(args, device):
    """Value association in both filters: TCF slots carrying 4-bit values, and
    the GQF's counted insert (values through the counters)."""
    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    nt = 15 * (1 << 22)
    tk = W.uniform_keys(7001, nt)
    tv = (W.uniform_keys(7002, nt) & np.uint64(15)).astype(np.uint8)
    tq = np.concatenate([tk[W.sample_with_replacement(7003, nt, 1 << 24)], W.uniform_keys(7004, 1 << 24)])
    ng = (1 << 25) + (1 << 24)
    gk = W.uniform_keys(7005, ng) & np.uint64(0xFFFFFFFF)
    gc = (1 + (W.uniform_keys(7006, ng) & np.uint64(7))).astype(np.uint32)
    gpos = W.sample_with_replacement(7007, ng, 1 << 24)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    tkd, tvd, tqd = to_dev(tk.view(np.int64)), to_dev(tv), to_dev(tq.view(np.int64))
    gkd, gcd, gqd = to_dev(gk.view(np.int64)), to_dev(gc.view(np.int32)), to_dev(gk[gpos].view(np.int64))
    tout = torch.zeros(len(tq), dtype=torch.uint8, device=device)
    gout = torch.zeros(len(gpos), dtype=torch.int64, device=device)
    T = gf.TCF(26, 16, gf.MODE_BULK, seed=21, max_batch=1 << 22, value_bits=4)
    G = gf.GQF(28, 8, seed=22, max_batch=ng)
    B = 1 << 22

    def step():
        T.clear()
        for o in range(0, nt, B):
            T.insert(tkd[o:o + B], values=tvd[o:o + B])
        T.query_values(tqd, tout)
        G.clear()
        G.insert_counts(gkd, gcd)
        G.count(gqd, gout)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    gf.trace_reset()
    gf.trace_enable(True)
    clocks = ClockSampler(device.index or 0)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    gf.trace_enable(False)
    trace = gf.trace_summary()
    ms = e0.elapsed_time(e1)
    kern, roof = roofline_from_trace(trace, with_traffic=False)
    ops = nt + len(tq) + ng + len(gpos)
    tv_got = tout.cpu().numpy()
    # the true counts of the probed keys (keys below 2^32 < 2^36: the fingerprint
    # is injective), reduced with torch outside the timed region
    sk, order = torch.sort(gkd)
    uk, inv = torch.unique_consecutive(sk, return_inverse=True)
    tot = torch.zeros(len(uk), dtype=torch.int64, device=device).index_add_(0, inv, gcd[order].to(torch.int64))
    exact = bool(torch.equal(tot[torch.searchsorted(uk, gqd)], gout))
    del sk, order, uk, inv, tot
    st_t, st_g = T.stats(), G.stats()
    per_kind = {k["kernel"]: k for k in kern}
    out = {"workload": VALUES_WORKLOAD, "value": round(aggregate_rate(ops, args.steps, 1, ms), 4), "unit": UNIT,
           "ms_per_step": round(ms / args.steps, 3), "ops_per_step": ops,
           "tcf_query_values_gops": round(len(tq) / (per_kind["tcf_query_values_kernel"]["ms"] / args.steps) / 1e6, 2),
           "clocks": clk, "gpu_launches": sum(v["launches"] for v in trace.values()), "roofline": roof,
           "kernels": kern,
           "checks": {"tcf_inserted_found": float((tv_got[:1 << 24] != 0xFF).mean()),
                      "tcf_value_equal": float((tv_got[:1 << 24] == tv[W.sample_with_replacement(7003, nt, 1 << 24)]).mean()),
                      "gqf_counts_exact": exact,
                      "tcf_failed_keys": st_t["failed_keys"], "gqf_failed_keys": st_g["failed_keys"],
                      "status_word": st_t["status_word"] | st_g["status_word"]}}
    del T, G
    torch.cuda.empty_cache()
    return out


SERVING_WORKLOAD = ("serving loop: 64 filters of 2^24 slots (32 TCF f=16 bulk + 32 counting GQF r=8, "
                    "2^30 slots in all) pre-filled to 50%; batches of 2^10..2^24 keys (log-uniform) for a "
                    "uniformly chosen filter, 50/45/5 insert/query/delete, until 90% aggregate load; host "
                    "keys in, host results out (page-locked buffers); 8 worker streams; Poisson arrivals at 0.5x and "
                    "0.8x of the back-to-back capacity")
SERVING_SMALL = ("serving loop, reduced: 64 filters of 2^20 slots (32 TCF f=16 bulk + 32 counting GQF r=8, 2^26 "
                 "slots in all) pre-filled to 50%; batches of 2^10..2^20 keys (log-uniform), 50/45/5 "
                 "insert/query/delete, until 90% aggregate load; otherwise as the full serving case")


def run_serving(args, device, log2_slots: int = 24, bmax: int = 24, workload: str = SERVING_WORKLOAD):
    """Capacity (every request submitted at once) and latency under Poisson
    arrivals at 0.5x and 0.8x of that capacity, from the same pre-filled
    state; then the same request sequence run back to back through the plain
    single-filter calls (host keys in, host results out, one stream), whose
    results must equal the served ones."""
    import time as _t

    import torch

    import paper_2212_09005_gb300 as gf
    from paper_2212_09005_gb300 import workloads as W

    w = W.serving_workload(log2_slots=log2_slots, bmax=bmax)
    reqs, nt, lg = w["requests"], w["n_tcf"], w["log2_slots"]
    mb = max(max(len(b) for b in w["prefill"]), max(len(k) for _, _, k in reqs))
    fs = [gf.TCF(lg, 16, gf.MODE_BULK, seed=5000 + i, max_batch=mb) if i < nt else
          gf.GQF(lg, 8, seed=5000 + i, max_batch=mb) for i in range(w["n_filters"])]
    pre = [torch.from_numpy(b.view(np.int64)).to(device) for b in w["prefill"]]

    def prefill():
        for f, b in zip(fs, pre):
            f.clear()
            f.insert(b)
        torch.cuda.synchronize()

    ops = sum(len(k) for _, _, k in reqs)
    # request keys and results in page-locked host memory, as a server's
    # receive buffers would be
    kbuf = torch.empty(ops, dtype=torch.int64).pin_memory()
    obuf = torch.empty(ops, dtype=torch.uint8).pin_memory()
    kv, ov = kbuf.numpy().view(np.uint64), obuf.numpy()
    spans, at = [], 0
    for _, _, k in reqs:
        kv[at:at + len(k)] = k
        spans.append((at, at + len(k)))
        at += len(k)
    S = gf.FilterServer(fs, workers=8, max_keys=max(len(k) for _, _, k in reqs))

    def run(arrivals):
        prefill()
        t0 = _t.perf_counter()
        tickets = []
        for j, (f, op, keys) in enumerate(reqs):
            if arrivals is not None:
                while _t.perf_counter() - t0 < arrivals[j]:
                    pass
            a, b = spans[j]
            tickets.append(S.submit(f, op, kv[a:b], out=ov[a:b]))
        lat = [S.wait(t)[1] for t in tickets]
        sec = _t.perf_counter() - t0
        return sec, np.array(lat)

    run(None)  # warm-up
    clocks = ClockSampler(device.index or 0)
    clocks.start()
    st0 = S.stats()
    sec, lat = run(None)
    st1 = S.stats()
    served = ov.copy()
    cap = ops / sec
    # where the time goes: summed latency per filter kind and operation
    brk = {}
    for (f, op, keys), l in zip(reqs, lat):
        k = ("tcf" if f < nt else "gqf") + "_" + ("insert", "query", "delete")[op]
        b = brk.setdefault(k, [0, 0, 0.0])
        b[0] += 1
        b[1] += len(keys)
        b[2] += float(l)
    breakdown = {k: {"requests": v[0], "keys": v[1], "latency_s_sum": round(v[2], 3)} for k, v in brk.items()}
    out = {"workload": workload, "requests": len(reqs), "ops": ops, "capacity_gops": round(cap / 1e9, 4),
           "capacity_p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
           "capacity_p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3), "capacity_breakdown": breakdown,
           "server": {k: st1[k] - st0[k] if k in ("batches", "requests", "merged_requests") else st1[k] for k in st1},
           "loads": []}
    mean_ops = ops / len(reqs)
    for frac in (0.5, 0.8):
        rate = frac * cap / mean_ops
        arr = W.poisson_arrivals(25, len(reqs), rate)
        sec, lat = run(arr)
        out["loads"].append({"load": frac, "offered_gops": round(frac * cap / 1e9, 4),
                             "achieved_gops": round(ops / sec / 1e9, 4),
                             "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                             "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3)})
    out["clocks"] = clocks.stop()
    S.close()
    # the plain path: the same requests back to back through the single-filter
    # calls, host keys in and host results out on one stream
    prefill()
    dk = torch.empty(max(len(k) for _, _, k in reqs), dtype=torch.int64, device=device)
    dr = torch.empty(dk.numel(), dtype=torch.uint8, device=device)
    pout = torch.empty(ops, dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    for j, (f, op, keys) in enumerate(reqs):
        a, b = spans[j]
        n = b - a
        dk[:n].copy_(kbuf[a:b], non_blocking=True)
        call = fs[f].insert if op == 0 else (fs[f].query if op == 1 else fs[f].remove)
        call(dk[:n], dr[:n])
        pout[a:b].copy_(dr[:n], non_blocking=True)
    torch.cuda.synchronize()
    psec = _t.perf_counter() - t0
    out["plain_gops"] = round(ops / psec / 1e9, 4)
    out["served_over_plain"] = round(cap / (ops / psec), 3)
    out["results_equal_plain"] = bool(np.array_equal(pout.numpy(), served))
    del fs, pre, kbuf, obuf, dk, dr, pout
    torch.cuda.empty_cache()
    return out


def run_e2e(R, args, world, device):
    """Same step through the C ABI with inputs in pinned host memory: every step
    copies its keys host->device and its results device->host inside the timed
    region. Inputs and results each have two device sets that alternate from
    step to step. The host->device copies run on a second stream in the order
    the step consumes them, each batch behind an event, so a step's copies
    overlap its own earlier batches and the previous step's work; a step's
    results are read back on a third stream, overlapping the next step."""
    import torch
    import torch.distributed as dist

    inp = R.inp
    B = R.B
    names = tuple(R.d.keys())
    onames = ("found", "found2", "cnt", "cnt2") + (("gfound",) if R.target else ())
    hostb = {k: torch.from_numpy(np.ascontiguousarray(inp[k]).view(np.int64)).pin_memory() for k in names}
    sets = [{k: torch.empty(hostb[k].shape, dtype=torch.int64, device=device) for k in names} for _ in range(2)]
    osets = [{k: torch.empty_like(getattr(R, k)) for k in onames} for _ in range(2)]
    hosto = [{k: torch.empty(getattr(R, k).shape, dtype=getattr(R, k).dtype).pin_memory() for k in onames}
             for _ in range(2)]
    h2d = sum(hostb[k].numel() * 8 for k in names)
    d2h = sum(t.numel() * t.element_size() for t in hosto[0].values())
    main = torch.cuda.current_stream(device)
    cs = torch.cuda.Stream(device)  # host->device
    ds = torch.cuda.Stream(device)  # device->host, so that both directions overlap
    done = [None, None]   # per input set: recorded on the compute stream after the step that read it
    rdone = [None, None]  # per result set: recorded on the copy stream after its results were read back

    def copies(si):
        ev = {}
        with torch.cuda.stream(cs):
            if done[si] is not None:
                cs.wait_event(done[si])
            for k in names:
                batched = k in ("tcf_ins", "tcf_del")
                n = hostb[k].numel()
                for j, s0 in enumerate(range(0, n, B if batched else max(n, 1))):
                    e = min(n, s0 + (B if batched else n))
                    sets[si][k][s0:e].copy_(hostb[k][s0:e], non_blocking=True)
                    ev[(k, j)] = torch.cuda.Event()
                    ev[(k, j)].record(cs)
        return ev

    def run(si, ev):
        if rdone[si] is not None:
            main.wait_event(rdone[si])  # the results of two steps ago have reached the host
        for k in onames:
            setattr(R, k, osets[si][k])
        R.step(sets[si], wait=lambda name, k=0: main.wait_event(ev[(name, k)]))
        e = torch.cuda.Event()
        e.record(main)
        done[si] = e
        with torch.cuda.stream(ds):
            ds.wait_event(e)
            for k in onames:
                hosto[si][k].copy_(osets[si][k], non_blocking=True)
            r = torch.cuda.Event()
            r.record(ds)
        rdone[si] = r

    run(0, copies(0))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    ev = copies(0)
    for i in range(args.steps):
        si = i % 2
        nxt = copies(1 - si) if i + 1 < args.steps else None
        run(si, ev)
        ev = nxt
    torch.cuda.synchronize()
    sec = max_over_ranks(time.perf_counter() - t0, world, device)
    v = aggregate_rate(ops_per_step(inp), args.steps, world, sec * 1e3)
    return {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "overlap": "host->device copies and result read-back on their own streams, two alternating device "
                       "sets of inputs and of results, each input batch behind an event"}


# ---------------------------------------------------------------------------
# CPU oracle (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def cpu_sample(inp, frac_gqf: int = 16):
    """Time the oracle on: the first 2^22-key TCF batch into the 2^26-slot table,
    2^21 + 2^21 TCF queries, 2^21 TCF deletes; 1/16 of the Zipf stream into the
    2^28-slot GQF, and 2^19 counts, deletes and re-counts."""
    import oracle as O

    B = inp["tcf_batch"]
    t_ins = inp["tcf_ins"][:B]
    npos = inp["n_pos"]
    probe = np.concatenate([inp["tcf_probe"][: B // 2], inp["tcf_probe"][npos:npos + B // 2]])
    t_del = t_ins[: B // 2]
    g_ins = inp["gqf_ins"][: len(inp["gqf_ins"]) // frac_gqf]
    g_q = g_ins[: 1 << 19]
    T = O.TCF(26, 16, seed=2)
    G = O.GQF(28, 8, seed=3)
    t0 = time.perf_counter()
    T.insert(t_ins)
    T.query(probe)
    T.remove(t_del)
    G.insert(g_ins)
    G.count(g_q)
    G.remove(g_q)
    G.count(g_q)
    sec = time.perf_counter() - t0
    ops = len(t_ins) + len(probe) + len(t_del) + len(g_ins) + 3 * len(g_q)
    return {"value": round(ops / sec / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"TCF 2^26: one 2^22-key insert batch, {len(probe)} queries, {len(t_del)} deletes; "
                       f"GQF 2^28: {len(g_ins)} Zipf keys, {len(g_q)} counts + deletes + re-counts"),
            "seconds": round(sec, 2), "ops": ops}


def _oracle_filters_worker(tasks):
    """One host core's share of the batched workload's filters, each in its
    own oracle filter: TCF keys in the same rounds as on the GPU, GQF keys in
    one batch, then queries of the filter's own and of fresh keys. Returns
    (ops, seconds of the oracle calls alone)."""
    import oracle as O
    from paper_2212_09005_gb300 import workloads as W

    ready = []
    for kind, lg, hseed, start, n, rounds, wseed in tasks:
        ready.append((kind, lg, hseed, W.uniform_keys_range(wseed + 2, start, n),
                      W.uniform_keys_range(wseed + 1000, start, n), rounds))
    ops = 0
    t0 = time.perf_counter()
    for kind, lg, hseed, keys, neg, rounds in ready:
        n = len(keys)
        if kind == "tcf":
            F = O.TCF(lg, 16, seed=hseed)
            for j in range(rounds):
                F.insert(keys[n * j // rounds:n * (j + 1) // rounds])
            F.query(keys)
            F.query(neg)
        else:
            F = O.GQF(lg, 8, seed=hseed)
            F.insert(keys)
            F.count(keys)
            F.count(neg)
        ops += 3 * n
    return ops, time.perf_counter() - t0


def cpu_batched_sample(w, target_keys: int = 1 << 25, wseed: int = 4):
    """The batched workload's oracle baseline on all host cores: every k-th
    filter of each kind (about target_keys inserted keys in all), one oracle
    filter per filter, spread over one process per core (spawned, so safe
    after CUDA is up; a worker that dies or stalls raises instead of hanging).
    Rate = sample ops / the slowest core's oracle time."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    off, logs, seeds, nt = w["offsets"], w["log2_slots"], w["hash_seeds"], w["n_tcf"]
    total = int(off[-1])
    k = max(1, total // target_keys)
    tasks = []
    for i in range(0, len(logs), k):
        n = int(off[i + 1] - off[i])
        tasks.append(("tcf" if i < nt else "gqf", int(logs[i]), int(seeds[i]), int(off[i]), n,
                      int(w["tcf_rounds"]), wseed))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    shares = [[] for _ in range(cores)]
    load = [0] * cores
    for t in sorted(tasks, key=lambda t: -t[4]):  # largest first, onto the least loaded core
        c = load.index(min(load))
        shares[c].append(t)
        load[c] += t[4]
    shares = [x for x in shares if x]
    ex = ProcessPoolExecutor(max_workers=len(shares), mp_context=mp.get_context("spawn"))
    try:
        futs = [ex.submit(_oracle_filters_worker, sh) for sh in shares]
        res = [f.result(timeout=600) for f in futs]
    finally:
        ex.shutdown(wait=False, cancel_futures=True)
    ops = sum(r[0] for r in res)
    sec = max(r[1] for r in res)
    nk = sum(t[4] for t in tasks)
    return {"value": round(ops / sec / 1e9, 6), "unit": UNIT, "cores": len(shares), "kind": "oracle",
            "sample": (f"every {k}-th filter of the batched workload ({len(tasks)} filters, {nk} keys), one oracle "
                       f"filter each, TCF keys in {w['tcf_rounds']} rounds, own + fresh queries; one process per "
                       f"core, rate over the slowest core's oracle time"),
            "seconds": round(sec, 4), "ops": ops}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    inp = make_inputs()
    for _ in range(max(3, args.warmup)):
        cpu_sample(inp, frac_gqf=64)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_sample(inp, frac_gqf=64)
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = float(np.mean(vals))
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(1e3 * float(np.mean(secs)), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded SplitMix64 uniform keys, Zipf rejection-inversion keys)",
        "config": {"workload": WORKLOAD, "sample": r["sample"], "parallelism": "single host thread"},
        "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]},
        "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    rank, world, local = rank_env()
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.case == "serving":
        import torch

        torch.cuda.set_device(local)
        sv = run_serving(args, torch.device("cuda", local))
        hi = sv["loads"][-1]
        line = {"metric": METRIC, "value": hi["achieved_gops"], "unit": UNIT, "n_gpus": 1, "steps": 1,
                "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": {"workload": SERVING_WORKLOAD},
                "serving": sv}
    elif args.case == "kmer":
        import torch

        torch.cuda.set_device(local)
        km = run_kmer(args, torch.device("cuda", local))
        line = {"metric": METRIC, "value": km["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": km["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": KMER_WORKLOAD}, "clocks": km["clocks"], "gpu_launches": km["gpu_launches"],
                "roofline": km["roofline"], "kmer": km}
    elif args.case == "values":
        import torch

        torch.cuda.set_device(local)
        vl = run_values(args, torch.device("cuda", local))
        line = {"metric": METRIC, "value": vl["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": vl["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": VALUES_WORKLOAD}, "clocks": vl["clocks"], "gpu_launches": vl["gpu_launches"],
                "roofline": vl["roofline"], "values": vl}
    elif args.case == "batched":
        import torch

        torch.cuda.set_device(local)
        b = run_batched(args, torch.device("cuda", local))
        line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": b["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": BATCHED_WORKLOAD}, "gpu_launches": b["gpu_launches"],
                "roofline": b["roofline"], "kernels": b["kernels"], "checks": b["checks"], "batched": b}
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
