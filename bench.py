"""Benchmark: greedy multi-hit WSC solves per second on one or more GB300s.

A step is one whole greedy solve (every round of Algorithm 1 with its P-DFS
argmax, §III-D) of the synthetic cohort "c2" (h=3, G=5,000, Nt=500, Nn=300,
seed 1; see synth/), with the cohort already resident on the device.  Between
timed steps a 256 MiB buffer is written to flush L2 (the cohort is far smaller
than L2).  Each step is timed with CUDA events on the solving stream; the timed
region is bracketed by barrier + synchronize; the result is the max over ranks.
On one GPU the line also carries the batched workload (16 uneven cohorts in one
launch against one after another) and the served one (a request trace replayed
against the continuous-batching server and against a plain loop).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank solves its own copy of the workload (weak
scaling, no collective on the data path).  --impl reference times the CPU oracle
(the paper's P-DFS restated in plain C, single-threaded) on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wsc_solves_per_s"
UNIT = "solves/s"
WORKLOAD = "c2"
H, ALPHA = 3, (1, 10)


def _dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_max(values, world):
    """Max over ranks of each value (identity on one rank)."""
    if world == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once nvidia-smi is sampling (at most 3 s)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Integer pipe of one SM per clock (32-bit results): logical / add ops and popcount.
INT32_OPS_PER_SM_CLK = 64
SMS = 152


def algorithmic_ops(r, Nt, Nn):
    """32-bit integer operations the P-DFS of §III-D performs for a solve's counters.

    Per unit, with w_t = 2 * ceil(Nt / 64) and w_n = 2 * ceil(Nn / 64) 32-bit words
    per tumor / normal row: every visited node at every depth costs w_t LOP3 (the
    AND with the parent's intersection fused with the zero test) + 1 compare; every
    scored leaf (TP > 0) additionally w_t AND + w_t POPC + w_n AND + w_n POPC + 6
    (score, key and compare).  Returns (ops of the whole solve, ops of the leaves)."""
    wt = 2 * ((Nt + 63) // 64)
    wn = 2 * ((Nn + 63) // 64)
    visited_all = int(r.visited.sum())
    visited_leaf = int(r.visited[:, -1].sum())
    scored = int((r.visited[:, -1] - r.pruned[:, -1]).sum())
    per_scored = 2 * wt + 2 * wn + 6
    return visited_all * (wt + 1) + scored * per_scored, visited_leaf * (wt + 1) + scored * per_scored


def _profiled_fields(kernel_file="k_solve_c2.md"):
    """Fields of the committed ncu summary of the solve kernel ("- `key`: `value`"
    lines), if that summary was taken from the kernel source as it is now (else {})."""
    import hashlib
    src = os.path.join(ROOT, "paper_2603_16721_gb300", "csrc", "mh_kernels.cu")
    try:
        text = open(os.path.join(ROOT, "profiles", kernel_file)).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return {}
    fields = {k: v.strip("`") for k, v in (ln.strip("- `").split(": ", 1) for ln in text.splitlines()
                                             if ln.startswith("- `") and ": " in ln)}
    return fields if fields.get("kernel_source_sha256") == sha else {}


def _profiled_traffic(kernel_file="k_solve_c2.md"):
    """DRAM bytes per launch of the solve kernel from the committed ncu summary (or None)."""
    try:
        return int(_profiled_fields(kernel_file)["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def solve_roofline(res_list, Nt, Nn, peaks, source):
    """Integer-pipe roofline of the persistent solve kernel (the dominant kernel:
    one cooperative launch runs every round of a solve).

    achieved = algorithmic 32-bit ops of a solve (algorithmic_ops: the per-node and
    per-leaf cost of the paper's search, applied to the solve's exact counters) /
    the kernel's duration (CUDA events around its launch on the solving stream);
    peak = SMs x 64 int32 ops/clk x max SM clock.  The kernel reaches the same
    counters and argmax with far fewer operations (64 siblings per OR of a sample
    column word; single-sample subtrees counted in closed form; TP = 1 leaves
    represented by per-sample champions), so `achieved` is a work-equivalent rate.
    What the hardware did is in `ncu` (from the committed profile of this kernel
    source): integer-pipe and issue utilisation over the launch."""
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = SMS * INT32_OPS_PER_SM_CLK * clk / 1e12
    ops = [algorithmic_ops(r, Nt, Nn) for r in res_list]
    kernel_s = sum(r.kernel_ms for r in res_list) / 1e3
    launches = sum(max(1, r.kernel_launches - 1) for r in res_list)  # minus the init kernel
    if kernel_s <= 0:
        return None
    achieved = sum(o[0] for o in ops) / kernel_s / 1e12
    leaf_s = sum(r.leaf_ms for r in res_list) / 1e3
    leaf = None
    if leaf_s > 0:
        # the kernel's own work in the leaf phase: 2 int32 ops per 64-bit column word
        # OR-ed in a sibling test (counted by the kernel) + ~14 per leaf scored exactly
        issued = sum(2 * r.leaf_words + 14 * r.leaf_scored for r in res_list) / leaf_s / 1e12
        leaf = {"ms_per_solve": round(leaf_s * 1e3 / len(res_list), 4),
                "issued": round(issued, 4), "issued_frac": round(issued / peak, 5)}
    prof = _profiled_fields()
    ncu = {k: float(prof[k]) for k in ("alu_pipe_active_pct", "issue_active_pct", "warps_active_pct",
                                       "barrier_stall_per_issue") if k in prof} or None
    return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 2), "unit": "Tops/s (int32)",
            "frac": round(achieved / peak, 4), "traffic": _profiled_traffic(),
            "kernel": "k_solve (persistent solve, one launch per solve)", "launches": launches,
            "avg_launch_us": round(kernel_s / launches * 1e6, 2),
            "ops_per_launch": round(sum(o[0] for o in ops) / launches),
            "leaf_phase": leaf, "ncu": ncu,
            "peak_source": f"derived: {SMS} SMs x {INT32_OPS_PER_SM_CLK} int32/clk x {clk / 1e6:.0f} MHz "
                           f"({source} max SM clock); no measured integer peak exists"}


def cpu_baseline_sample(c, full_visited_total, seconds_target=10.0):
    """Oracle P-DFS on the first rounds of the workload, scaled to solves/s by visited nodes."""
    import oracle
    rounds = 1
    t0 = time.perf_counter()
    sol = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, H, ALPHA, max_rounds=rounds)
    dt = time.perf_counter() - t0
    while dt < seconds_target / 3 and rounds < 8:
        rounds *= 2
        t0 = time.perf_counter()
        sol = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, H, ALPHA, max_rounds=rounds)
        dt = time.perf_counter() - t0
    vis = int(sol.visited.sum())
    frac = vis / full_visited_total
    solves_per_s = frac / dt
    return {"value": solves_per_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle P-DFS (single-threaded C) on the first {rounds} greedy rounds of {WORKLOAD} "
                      f"({vis} of {full_visited_total} visited nodes of the solve, {100 * frac:.1f}%), "
                      f"{dt:.2f} s, scaled to whole solves by visited nodes"}, dt


def run_reference(args):
    rank, world, _ = _dist_env()
    if world > 1 and rank != 0:
        return 0
    import synth
    c = synth.generate(synth.c2())
    total = _full_visited_total(c)
    if total is None:  # stored oracle result does not match this machine's cohort: count once
        import oracle
        total = int(oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, H, ALPHA).visited.sum())
    vals = []
    for i in range(args.warmup + args.steps):
        cb, dt = cpu_baseline_sample(c, total, seconds_target=3.0)
        if i >= args.warmup:
            vals.append((cb, dt))
    value = statistics.median(v[0]["value"] for v in vals)
    ms = 1e3 / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "c2: h=3, G=5000, Nt=500, Nn=300, seed 1, alpha=1/10"},
            "cpu_baseline": vals[-1][0], "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _full_visited_total(c):
    """Visited nodes of the whole c2 solve (from the stored oracle result when it matches)."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", "c2_pdfs.json")
    try:
        g = json.load(open(path))
        if g["cohort_sha256"] == hashlib.sha256(c.bitmaps.tobytes()).hexdigest():
            return int(sum(sum(r) for r in g["visited"]))
    except (OSError, ValueError, KeyError):
        pass
    return None


def run_ours(args):
    import torch
    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2603_16721_gb300 import mh

    c = synth.generate(synth.c2())
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    H = mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn)
    mh.mh_set_stream(H, stream.cuda_stream)
    for _ in range(args.warmup):
        mh.mh_solve_ex(H, H_HITS, ALPHA, max_rounds=args.max_rounds, mode=MODES[args.mode])
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    results, step_ms = [], []
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r = mh.mh_solve_ex(H, H_HITS, ALPHA, max_rounds=args.max_rounds, time_kernels=True, mode=MODES[args.mode])
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        results.append(r)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    total_ms = sum(step_ms)
    total_ms_max, = aggregate_max([total_ms], world)
    value = world * args.steps / (total_ms_max / 1e3)

    if args.kernels_only:  # profiling run: the timed solves only
        H.close()
        if rank == 0:
            print(json.dumps({"kernels_only": True, "ms_per_step": total_ms / args.steps}))
        return 0

    # end to end through the C ABI with host buffers: create (H2D), solve, read back
    e2e_ms = []
    d2h = 0
    for _ in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H2:
            r2 = mh.mh_solve(H2, H_HITS, ALPHA)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        d2h = r2.genes.nbytes + r2.tp.nbytes + r2.fp.nbytes + r2.visited.nbytes + r2.pruned.nbytes
    e2e_max, = aggregate_max([statistics.median(e2e_ms)], world)
    H.close()

    if rank == 0:
        peaks, src = _peaks()
        r0 = results[-1]
        scored = int((r0.visited[:, -1] - r0.pruned[:, -1]).sum())
        vis_leaves = int(r0.visited[:, -1].sum())
        pruned_prefixes = int(r0.pruned[:, :-1].sum())
        cb = None
        total_vis = _full_visited_total(c) or int(r0.visited.sum())
        if world == 1:
            cb, _ = cpu_baseline_sample(c, total_vis)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "c2: h=3, G=5000, Nt=500, Nn=300, seed 1, alpha=1/10",
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MiB write)",
                       "rounds_per_solve": r0.rounds, "selected": r0.k},
            "breakdown_ms_per_solve": {k: round(sum(getattr(r, k) for r in results) / len(results), 3)
                                       for k in ("level1_ms", "expand_ms", "leaf_ms", "finalize_ms")},
            "mode": "persistent" if r0.mode == mh.MH_MODE_PERSISTENT else "launches",
            "warp_balance": {k: {"mean_warp_cycles": round(r0.diag[i] / max(1, r0.diag[4 + i]), 1),
                                 "longest_warp_cycles_per_round": round(r0.diag[2 + i] / max(1, r0.rounds), 1)}
                             for i, k in enumerate(("expand", "leaf"))},
            "extra": {"p50_ms": statistics.median(step_ms), "p99_ms": sorted(step_ms)[int(0.99 * (len(step_ms) - 1))],
                      "combos_scored_per_s": scored * value / world, "leaves_tested_per_s": vis_leaves * value / world,
                      "prefixes_pruned_per_s": pruned_prefixes * value / world,
                      "visited_fraction": vis_leaves / (r0.rounds * _comb(c.G, H_HITS))},
            "roofline": solve_roofline(results, c.Nt, c.Nn, peaks, src),
            "cpu_baseline": cb,
            "e2e": {"value": world / (e2e_max / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(c.bitmaps.nbytes), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(sum(r.kernel_launches for r in results)),
            "clocks": clocks,
        }
        if world == 1 and not args.no_extras:
            # the other two parts of the metric, after the timed c2 steps: batched
            # (16 uneven cohorts in one launch vs one after another) and served
            # (request trace: continuous batching vs a plain loop)
            b16 = batch16_comparison(argparse.Namespace(steps=3, warmup=1))
            line["batched"] = {k: b16[k] for k in ("value", "unit", "sequential_value", "speedup_vs_sequential",
                                                   "identical_to_sequential", "config")}
            line["served"] = served_comparison(argparse.Namespace(requests=200, slots=8, large_slots=0))
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _comb(n, k):
    import math
    return math.comb(n, k)


H_HITS = H
MODES = {"persistent": 0, "launches": 1}


def run_batch16(args):
    print(json.dumps(batch16_comparison(args)))
    return 0


def batch16_comparison(args):
    """Batched workload: 16 cohorts of uneven size (seeds 100-115, h=3 for 12, h=4 for 4)
    solved in one persistent launch, against the same 16 solved one after another."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2603_16721_gb300 import mh
    specs = synth.batch16()
    cohorts = [synth.generate(sp) for sp in specs]
    stream = torch.cuda.Stream()
    handles = [mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) for c in cohorts]
    for H in handles:
        mh.mh_set_stream(H, stream.cuda_stream)
    hs = [sp.h for sp in specs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # sequential plain solves (one persistent launch per solve)
    seq = []
    for _ in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rs = [mh.mh_solve(H, h) for H, h in zip(handles, hs)]
        seq.append(time.perf_counter() - t0)
    seq_t = statistics.median(seq[args.warmup:])
    # batched solves (the first call autotunes the block split)
    bat = []
    for _ in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = mh.mh_solve_batch(handles, hs)
        bat.append(time.perf_counter() - t0)
    bat_t = statistics.median(bat[args.warmup:])
    same = all(a.records() == b.records() for a, b in zip(rs, rb))
    out = ({
        "metric": "batched_wsc_solves_per_s", "value": len(handles) / bat_t, "unit": "solves/s",
        "sequential_value": len(handles) / seq_t, "speedup_vs_sequential": seq_t / bat_t,
        "identical_to_sequential": same, "steps": args.steps, "warmup": args.warmup,
        "config": {"workload": "batch16: 16 cohorts, seeds 100-115, G~U[2000,19000], Nt~U[100,1000], "
                               "Nn~U[50,500], h=3 x12 and h=4 x4, alpha=1/10"},
        "per_cohort": [{"G": c.G, "Nt": c.Nt, "Nn": c.Nn, "h": sp.h, "k": r.k, "rounds": r.rounds,
                        "solo_ms": round(r.solve_ms, 3)} for c, sp, r in zip(cohorts, specs, rs)],
    })
    for H in handles:
        H.close()
    return out


def run_served(args):
    print(json.dumps(served_comparison(args)))
    return 0


def served_comparison(args):
    """Served workload: a trace of requests (c3-law cohorts, Poisson arrivals at 5/s,
    h from {2: .3, 3: .5, 4: .2}) replayed in real time against (i) the served
    runtime (continuous batching) and (ii) a plain FIFO loop of one solve (one
    persistent launch) per request; latency = arrival to result.  Then the same
    requests all at once (saturated), for throughput at full load."""
    import threading
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2603_16721_gb300 import mh
    specs, gaps = synth.served200()
    n = min(args.requests, len(specs))
    specs = specs[:n]
    arrivals = np.cumsum(gaps[:n]) - gaps[0]
    cohorts = [synth.generate(sp) for sp in specs]
    torch.cuda.synchronize()
    # warm-up: one request of each h, both paths
    for h in (2, 3, 4):
        c = next(c for c, sp in zip(cohorts, specs) if sp.h == h)
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            mh.mh_solve(H, h)

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]

    # (ii) plain FIFO loop
    plain_res, plain_lat, service = [], [], []
    t0 = time.perf_counter()
    for i, (c, sp) in enumerate(zip(cohorts, specs)):
        now = time.perf_counter() - t0
        if now < arrivals[i]:
            time.sleep(arrivals[i] - now)
        ts = time.perf_counter()
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            plain_res.append(mh.mh_solve(H, sp.h))
        te = time.perf_counter()
        service.append(te - ts)
        plain_lat.append(te - t0 - arrivals[i])
    plain_span = time.perf_counter() - t0

    # (i) served: requests submitted at their arrival times
    with mh.Server(slots=args.slots, large_slots=args.large_slots) as S:
        tickets = [None] * n
        t0 = time.perf_counter()

        def submitter():
            for i, (c, sp) in enumerate(zip(cohorts, specs)):
                now = time.perf_counter() - t0
                if now < arrivals[i]:
                    time.sleep(arrivals[i] - now)
                tickets[i] = S.submit(c.bitmaps, c.G, c.Nt, c.Nn, sp.h)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        served_res = [S.wait(t) for t in tickets]
        served_span = time.perf_counter() - t0
        stats = S.stats()
        # saturated: every request submitted at once (throughput at full load; the
        # plain loop's is 1 / mean service time)
        t0 = time.perf_counter()
        burst_tickets = [S.submit(c.bitmaps, c.G, c.Nt, c.Nn, sp.h) for c, sp in zip(cohorts, specs)]
        burst_res = [S.wait(t) for t in burst_tickets]
        burst_span = time.perf_counter() - t0
    served_lat = [r.solve_ms / 1e3 for r in served_res]
    same = all(a.records() == b.records() for a, b in zip(plain_res, served_res))
    same = same and all(a.records() == b.records() for a, b in zip(plain_res, burst_res))
    mean_service = sum(service) / n
    plain_done = np.cumsum(service)  # the plain loop fed all requests at once
    return ({
        "metric": "served_wsc_solves_per_s", "value": n / served_span, "unit": "solves/s",
        "p50_ms": 1e3 * pct(served_lat, 0.50), "p99_ms": 1e3 * pct(served_lat, 0.99),
        "plain": {"value": n / plain_span, "p50_ms": 1e3 * pct(plain_lat, 0.50), "p99_ms": 1e3 * pct(plain_lat, 0.99),
                  "mean_service_ms": 1e3 * mean_service, "capacity_solves_per_s": 1.0 / mean_service},
        "saturated": {"served_solves_per_s": n / burst_span, "plain_solves_per_s": 1.0 / mean_service,
                      "served_p50_ms": 1e3 * pct([r.solve_ms / 1e3 for r in burst_res], 0.50),
                      "served_p99_ms": 1e3 * pct([r.solve_ms / 1e3 for r in burst_res], 0.99),
                      "plain_p50_ms": 1e3 * pct(list(plain_done), 0.50),
                      "plain_p99_ms": 1e3 * pct(list(plain_done), 0.99)},
        "offered_load_req_per_s": n / max(arrivals[-1], 1e-9), "requests": n, "slots": args.slots,
        "identical_to_plain": same, "server_launches": stats["launches"],
        "config": {"workload": f"served: first {n} of 200 requests, c3-law cohorts (G=19000, Nt=800, Nn=400), "
                               "seeds 1000-1199, Poisson 5 req/s, h from {2:.3,3:.5,4:.2}, trace seed 5000"},
    })


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--max-rounds", type=int, default=0, help="stop each solve after R rounds (profiling)")
    ap.add_argument("--kernels-only", action="store_true", help="time the solves only (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="c2: leave out the batched and served comparisons appended to the line")
    ap.add_argument("--mode", choices=["persistent", "launches"], default="persistent",
                    help="one persistent kernel per solve, or one launch per phase")
    ap.add_argument("--workload", choices=["c2", "batch16", "served200"], default="c2",
                    help="c2: the headline single-cohort solve; batch16: the batched workload; "
                         "served200: the served request trace")
    ap.add_argument("--requests", type=int, default=200, help="served200: requests replayed")
    ap.add_argument("--slots", type=int, default=8, help="served200: concurrent requests")
    ap.add_argument("--large-slots", type=int, default=0,
                    help="served200: large requests solved concurrently (0: the library default)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch16":
        return run_batch16(args)
    if args.workload == "served200":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
