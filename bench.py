"""Throughput of batched Smith-Waterman (affine gaps, BLOSUM62, open 11 /
extend 1) on one GB300, on the seeded 2,000,000-pair log-normal workload.

One step = one pass of the whole hot path (device bucketing, forward DP for
score and end, reverse DP for start, records in pair order) over all pairs,
inputs resident in HBM, replayed from a CUDA graph captured once
(swgb_plan_create; --no-graph times direct swgb_align calls).  Prints one
JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on the host cores
    python bench.py --workload families_200k   # many-against-many block:
        one step = candidate discovery by shared 6-mers + alignment of every
        candidate + identity / pass-fail, on 200,000 resident sequences

Under torchrun every rank aligns its own copy of the workload (weak scaling,
no collective on the data path); the step time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS & alignments/s on 1 GB300 (bit-exact); filter recall; p50/p99 latency"
ADDMAX_OPS_PER_CELL = 2.5     # five packed 16x2 add-max per two cells
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "dp_forward_traffic.json")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2303_01845_gb300", "csrc", "swgb_kernels.cu")
KERNEL_HEADER = os.path.join(ROOT, "paper_2303_01845_gb300", "csrc", "swgb_internal.cuh")
LANE_HEADER = os.path.join(ROOT, "paper_2303_01845_gb300", "csrc", "swgb_lane.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_2m")
    ap.add_argument("--pairs", type=int, default=0,
                    help="use an evenly strided subset of N pairs (profiling cases)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="time direct swgb_align calls instead of replaying a captured CUDA graph")
    ap.add_argument("--tune-pairs", type=int, default=0,
                    help="pairs of the batch the tile and band selection is tuned on "
                         "(0 = the whole batch; a smaller number = an evenly strided sample)")
    ap.add_argument("--tile-overhead", type=int, default=-1,
                    help="fixed tile-cost overhead instead of tuning (profiling runs)")
    ap.add_argument("--band-min", type=int, default=-1,
                    help="fixed band threshold (0 = no banded reverse pass) with --tile-overhead")
    ap.add_argument("--filter-epochs", type=int, default=20,
                    help="family blocks: training epochs of the learned filter")
    ap.add_argument("--filter-recall", type=float, default=0.995,
                    help="family blocks: recall of the training positives the threshold keeps")
    ap.add_argument("--no-tune", action="store_true",
                    help="family blocks: keep the context's aligner knobs for the filtered pipeline "
                         "instead of tuning them (untimed) on the block's kept pairs")
    ap.add_argument("--serve-refs", type=int, default=1_000_000, help="serving: resident references")
    ap.add_argument("--serve-requests", type=int, default=400, help="serving: timed requests")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="serving: requests per second")
    ap.add_argument("--serve-slots", type=int, default=3, help="serving: batches in flight")
    ap.add_argument("--no-next-rows", action="store_true",
                    help="batched run: skip the other workloads' figures (next_rows)")
    ap.add_argument("--next-steps", type=int, default=3,
                    help="timed steps of the family block in next_rows")
    ap.add_argument("--next-requests", type=int, default=200,
                    help="serving requests timed in next_rows")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's step time); value itself
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, steps, total_ms):
    """Whole-job throughput: units every rank processed in `steps` steps
    divided by the (max over ranks) time of those steps."""
    return world * units_per_rank * steps / (total_ms / 1e3)


def sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def dp_source_sha():
    """Hash of what the DP kernels' DRAM traffic depends on: the DP section of
    swgb_kernels.cu (the kernel, its dispatch and launch sizes), the lane
    arithmetic of swgb_lane.cuh and swgb_internal.cuh (tile shapes,
    arguments)."""
    src = open(KERNEL_SOURCE).read()
    a = src.index("// The DP kernel")
    b = src.index("// Issue-rate probe")
    return hashlib.sha256(src[a:b].encode() + open(LANE_HEADER, "rb").read() +
                          open(KERNEL_HEADER, "rb").read()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p))
    return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def make_workload(name, mat, pairs=0):
    import numpy as np

    from paper_2303_01845_gb300 import workload
    wl = workload.generate(name, mat)
    if pairs and pairs < len(wl.pairs):
        # an evenly strided subset keeps the mix of lengths and relatedness
        wl = wl.subset(np.linspace(0, len(wl.pairs) - 1, pairs).astype(np.int64))
    return wl


def workload_name(args):
    return args.workload + ("[%d strided]" % args.pairs if args.pairs else "")


def cpu_oracle_sample(wl, mat, target_s, seed=7):
    """Times the oracle (as it stands) on a seeded random subset of the pairs
    sized to take about target_s seconds on all host cores."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(wl.pairs))
    # calibrate on a small subset
    n0 = min(len(perm), 2000)
    sub = wl.subset(np.sort(perm[:n0]))
    t = time.perf_counter()
    oracle.align_batch(sub.q_res, sub.q_off, sub.r_res, sub.r_off, sub.pairs, mat, 11, 1,
                       n_threads=cores)
    dt = time.perf_counter() - t
    rate = sub.cells() / max(dt, 1e-6)
    mean_cells = sub.cells() / n0
    n = int(min(len(perm), max(n0, target_s * rate / mean_cells)))
    sub = wl.subset(np.sort(perm[:n]))
    t = time.perf_counter()
    oracle.align_batch(sub.q_res, sub.q_off, sub.r_res, sub.r_off, sub.pairs, mat, 11, 1,
                       n_threads=cores)
    dt = time.perf_counter() - t
    return {"gcups": sub.cells() / dt / 1e9, "aln_per_s": n / dt, "cores": cores, "pairs": n,
            "cells": sub.cells(), "seconds": dt}


def run_reference(args):
    """The CPU oracle on the host cores, same workload and metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    mat = oracle.blosum62()
    wl = make_workload(args.workload, mat, args.pairs)
    cores = os.cpu_count() or 1
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    # size one step's sample from a calibration run
    cal = cpu_oracle_sample(wl, mat, per_step / 4, seed=99)
    mean_cells = cal["cells"] / cal["pairs"]
    n = int(min(len(wl.pairs), per_step * cal["gcups"] * 1e9 / mean_cells))
    rng = np.random.default_rng(3)
    times, cells, pairs = [], 0, 0
    for step in range(args.warmup + args.steps):
        sub = wl.subset(np.sort(rng.choice(len(wl.pairs), size=n, replace=False)))
        t = time.perf_counter()
        oracle.align_batch(sub.q_res, sub.q_off, sub.r_res, sub.r_off, sub.pairs, mat, 11, 1,
                           n_threads=cores)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            cells += sub.cells()
            pairs += n
    total = sum(times)
    value = cells / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(args), "pairs_per_step": n,
                   "sample": "seeded random subset of the workload's pairs per step"},
        "alignments_per_s": pairs / total,
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d random pairs of %s per step" % (n, workload_name(args))},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def traffic_for_current_kernel():
    """DRAM bytes per forward pass from the committed ncu summary, if it was
    taken on the current DP kernel source (else None)."""
    try:
        rec = json.load(open(PROFILE_SUMMARY))
    except (OSError, ValueError):
        return None
    if rec.get("dp_source_sha") != dp_source_sha():
        return None
    return rec.get("dram_bytes_per_forward_pass")


def run_ours(args):
    import numpy as np
    import torch

    from paper_2303_01845_gb300 import swgb

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mat = swgb.swgb_blosum62()
    wl = make_workload(args.workload, mat, args.pairs)
    al = swgb.Aligner(local)
    stream = torch.cuda.current_stream(dev)
    q = al.seqset(torch.from_numpy(wl.q_res).to(dev), torch.from_numpy(wl.q_off).to(dev))
    r = al.seqset(torch.from_numpy(wl.r_res).to(dev), torch.from_numpy(wl.r_off).to(dev))
    pairs = torch.from_numpy(wl.pairs).to(dev)
    out = torch.empty((len(wl.pairs), 5), dtype=torch.int32, device=dev)
    params = swgb.make_params(mat, 11, 1, timing=True)
    P = len(wl.pairs)

    # tile and band selection tuned on the batch, or an evenly strided sample
    # of it (untimed): the band's extra rounds weigh more on a small sample
    tuning = None
    if args.band_min >= 0:
        swgb.swgb_set_band_min(al.ctx, args.band_min)
    if args.tile_overhead >= 0:
        swgb.swgb_set_tile_overhead(al.ctx, args.tile_overhead)
        tile_overhead = args.tile_overhead
    else:
        tune_n = P if args.tune_pairs <= 0 else min(P, args.tune_pairs)
        tune_idx = torch.from_numpy(np.linspace(0, P - 1, tune_n).astype(np.int64)).to(dev)
        tune_pairs = pairs[tune_idx].contiguous()
        tune_out = torch.empty((tune_n, 5), dtype=torch.int32, device=dev)
        tile_overhead, _ = swgb.swgb_autotune(al.ctx, q.handle, r.handle, tune_pairs, params,
                                              tune_out, stream)
        tuning = swgb.swgb_last_tuning(al.ctx)
        tuning["pairs"] = int(tune_n)
        del tune_pairs, tune_out

    # the timed step replays the whole pipeline captured once into a CUDA graph
    # (swgb_plan_*): same kernels and records as swgb_align, no per-launch host work
    plan = None if args.no_graph else swgb.swgb_plan_create(al.ctx, q.handle, r.handle, pairs, params, out)
    launch_kind = "direct calls" if plan is None else "CUDA graph (swgb_plan)"

    def step():
        if plan is not None:
            swgb.swgb_plan_launch(al.ctx, plan, stream)
        else:
            swgb.swgb_align(al.ctx, q.handle, r.handle, pairs, params, out, stream)

    for _ in range(args.warmup):
        step()
        swgb.swgb_sync(al.ctx, stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    step_ms, fwd_ms, rev_ms = [], [], []
    launches = 0
    stats = None

    def barrier():
        if dist is not None:
            dist.barrier()

    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            swgb.swgb_sync(al.ctx, stream)
            stats = swgb.swgb_last_stats(al.ctx)
            fwd_ms.append(stats["forward_ms"])
            rev_ms.append(stats["reverse_ms"])
            launches += stats["kernel_launches"]
        torch.cuda.synchronize()
        barrier()
    clock = clocks.summary()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    cells = stats["forward_cells"]
    value = job_rate(cells, world, args.steps, total_ms) / 1e9
    aln_per_s = job_rate(P, world, args.steps, total_ms)
    fwd_mean = statistics.mean(fwd_ms)
    achieved = cells / (fwd_mean / 1e3) / 1e9
    # the cells the reverse pass needs: the prefixes up to the end, from the
    # start's query row on (a pass cannot stop before the start)
    recs = out.cpu().numpy().astype(np.int64)
    scored = recs[:, 0] > 0
    rev_needed = int(((recs[scored, 2] - recs[scored, 1] + 1) * (recs[scored, 4] + 1)).sum())
    slot_split = {"forward_slots": stats["forward_slots"], "reverse_slots": stats["reverse_slots"],
                  "reverse_needed_cells": rev_needed,
                  "forward_cells_per_slot": cells / max(stats["forward_slots"], 1),
                  "reverse_needed_per_slot": rev_needed / max(stats["reverse_slots"], 1)}

    # roofline of the forward DP: add-max issue rate x SMs x max clock
    ops_per_clk, sms = swgb.swgb_probe_addmax_rate(al.ctx)
    peaks = measured_peaks()
    sm_max_mhz = peaks.get("sm_max_mhz") or clock.get("sm_max_mhz") or 2070.0
    peak = sms * sm_max_mhz * 1e6 * ops_per_clk / ADDMAX_OPS_PER_CELL / 1e9

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(al, wl, mat, dev, stream, args, dist, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the host baseline: N = 1 only
        cpu = cpu_oracle_sample(wl, np.asarray(mat), args.cpu_seconds)

    next_rows = None
    if rank == 0 and world == 1 and not args.no_next_rows and not args.pairs:
        if plan is not None:
            swgb.swgb_plan_destroy(plan)
            plan = None
        next_rows = measure_next_rows(args, al, dev)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i16x2+i32", "data": "synthetic",
        "config": {"workload": workload_name(args), "pairs": P, "forward_cells": cells,
                   "reverse_cells": stats["reverse_cells"],
                   "int32_pairs": stats["n_int32_pairs"], "gap_open": 11, "gap_extend": 1,
                   "matrix": "BLOSUM62", "tile_overhead": tile_overhead,
                   "band_min": swgb.swgb_get_band_min(al.ctx),
                   "autotune": tuning,
                   "band_pairs": stats["n_band_pairs"], "band_certified": stats["n_band_certified"],
                   "dp_slots": slot_split,
                   "launch": launch_kind,
                   "l2": "inputs (%.2f GB of residues) exceed L2; no flush" %
                         ((len(wl.q_res) + len(wl.r_res)) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "alignments_per_s": aln_per_s,
        "gcups_forward_kernel": achieved,
        "forward_ms": fwd_mean, "reverse_ms": statistics.mean(rev_ms),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
                     "frac": achieved / peak, "traffic": traffic_for_current_kernel(),
                     "peak_basis": "%d SMs x %.0f MHz x %.1f add-max/clk/SM (measured) / %.1f per cell"
                                   % (sms, sm_max_mhz, ops_per_clk, ADDMAX_OPS_PER_CELL)},
        "cpu_baseline": None if cpu is None else {
            "value": cpu["gcups"], "unit": "GCUPS", "cores": cpu["cores"], "kind": "oracle",
            "sample": "%d random pairs (%.2e cells) of %s, %.1f s" %
                      (cpu["pairs"], cpu["cells"], workload_name(args), cpu["seconds"]),
            "alignments_per_s": cpu["aln_per_s"]},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clock["sm_mhz"], "sm_max_mhz": clock["sm_max_mhz"],
                   "reasons": clock["reasons"]},
    }
    if next_rows is not None:
        line["next_rows"] = next_rows
    print(json.dumps(line), flush=True)
    if plan is not None:
        swgb.swgb_plan_destroy(plan)
    if dist is not None:
        dist.destroy_process_group()


def measure_plain(al, dev, name, steps, warmup):
    """The small plain workload (10,000 pairs, lengths U[50,500]): every record
    checked against the oracle, then the same step as the batched line
    (CUDA-graph replay) timed on the device, and the oracle timed on all host
    cores over the whole workload."""
    import numpy as np
    import torch

    import oracle
    from paper_2303_01845_gb300 import swgb
    mat = swgb.swgb_blosum62()
    wl = make_workload(name, mat)
    stream = torch.cuda.current_stream(dev)
    q = al.seqset(torch.from_numpy(wl.q_res).to(dev), torch.from_numpy(wl.q_off).to(dev))
    r = al.seqset(torch.from_numpy(wl.r_res).to(dev), torch.from_numpy(wl.r_off).to(dev))
    pairs = torch.from_numpy(wl.pairs).to(dev)
    out = torch.empty((len(wl.pairs), 5), dtype=torch.int32, device=dev)
    params = swgb.make_params(mat, 11, 1, timing=True)
    plan = swgb.swgb_plan_create(al.ctx, q.handle, r.handle, pairs, params, out)
    for _ in range(warmup):
        swgb.swgb_plan_launch(al.ctx, plan, stream)
    swgb.swgb_sync(al.ctx, stream)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    want = oracle.align_batch(wl.q_res, wl.q_off, wl.r_res, wl.r_off, wl.pairs, np.asarray(mat), 11, 1,
                              n_threads=cores)
    cpu_s = time.perf_counter() - t
    exact = bool(np.array_equal(out.cpu().numpy(), want))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    fwd = []
    for k in range(steps):
        ev[k][0].record(stream)
        swgb.swgb_plan_launch(al.ctx, plan, stream)
        ev[k][1].record(stream)
        swgb.swgb_sync(al.ctx, stream)
        st = swgb.swgb_last_stats(al.ctx)
        fwd.append(st["forward_ms"])
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    swgb.swgb_plan_destroy(plan)
    q.close()
    r.close()
    cells = st["forward_cells"]
    return {"workload": name, "pairs": len(wl.pairs), "forward_cells": cells,
            "records_bit_exact_vs_oracle": exact, "ms_per_step": ms, "gcups": cells / ms / 1e6,
            "alignments_per_s": len(wl.pairs) / ms * 1e3,
            "gcups_forward_kernel": cells / statistics.mean(fwd) / 1e6, "steps": steps,
            "launch": "CUDA graph (swgb_plan)",
            "cpu_baseline": {"gcups": cells / cpu_s / 1e9, "alignments_per_s": len(wl.pairs) / cpu_s,
                             "cores": cores, "kind": "oracle", "sample": "the whole workload"}}


def measure_next_rows(args, al, dev):
    """The other workloads' figures, added to the batched line: the small plain
    workload, the many-against-many block with and without the learned filter,
    and the query server under Poisson load.  Each leg is fenced: a failure
    is reported in its place."""
    import traceback
    out = {}
    steps = max(1, args.next_steps)
    warm = max(1, min(args.warmup, 2))
    try:
        out["plain_10k"] = measure_plain(al, dev, "plain_10k", max(3, args.steps), warm)
    except Exception as e:   # noqa: BLE001 -- reported in the line
        out["plain_10k"] = {"error": "%s: %s" % (type(e).__name__, e), "trace": traceback.format_exc()[-800:]}
    mlp = thr = None
    try:
        line, mlp, thr = measure_families(args, al, dev, "families_200k", steps, warm,
                                          None if args.no_cpu_baseline else 4.0)
        f = line["filter"]
        out["families_200k"] = {
            "candidates": line["config"]["candidates"], "passing_pairs": line["config"]["passing_pairs"],
            "plain_ms_per_step": line["plain"]["ms_per_step"], "filtered_ms_per_step": line["ms_per_step"],
            "plain_candidates_per_s": line["plain"]["alignments_per_s"],
            "filtered_candidates_per_s": line["value"], "speedup": f["speedup_vs_plain"],
            "recall": f["recall"], "kept_fraction": f["kept_fraction"],
            "kept_results_exact": f["kept_results_exact"], "kmer_threshold_3": f["kmer_threshold_3"],
            "stage_ms": {"plain": {k: line["plain"][k] for k in ("discover_ms", "align_ms", "identity_ms")},
                         "filtered": f["ms"]},
            "gcups_forward_kernel": line["plain"]["gcups_forward_kernel"],
            "trained_on": f["trained_on"], "aligner_knobs": f["aligner_knobs"], "steps": steps,
            "cpu_baseline": line["cpu_baseline"],
            "clocks": line["clocks"]}
    except Exception as e:   # noqa: BLE001
        out["families_200k"] = {"error": "%s: %s" % (type(e).__name__, e), "trace": traceback.format_exc()[-800:]}
    if mlp is not None:
        try:
            line = measure_serving(args, al, dev, mlp, thr, 0.0, args.next_requests, args.serve_rate, warm)
            out["serving_1m"] = {
                "references": line["config"]["references"], "arrivals": line["config"]["arrivals"],
                "requests": line["config"]["requests"], "slots": line["config"]["slots"],
                "latency_ms": line["latency_ms"], "queue_ms": line["queue_ms"],
                "throughput": line["throughput"], "max_batches_in_flight": line["max_batches_in_flight"],
                "filter": "the network trained for families_200k", "clocks": line["clocks"]}
        except Exception as e:   # noqa: BLE001
            out["serving_1m"] = {"error": "%s: %s" % (type(e).__name__, e), "trace": traceback.format_exc()[-800:]}
    return out


def measure_e2e(al, wl, mat, dev, stream, args, dist=None, world=1):
    """Same metric through the public host-buffer API: every step loads both
    sequence sets from pinned host memory, copies the pairs in and the records
    out (swgb_seqset_load + swgb_align_host).  Whole-job figure: a barrier on
    both sides, the slowest rank's time, every rank's units."""
    import torch

    from paper_2303_01845_gb300 import swgb
    pin = lambda a: torch.from_numpy(a).pin_memory()
    q_res, q_off, r_res, r_off = pin(wl.q_res), pin(wl.q_off), pin(wl.r_res), pin(wl.r_off)
    pairs = pin(wl.pairs)
    out = torch.empty((len(wl.pairs), 5), dtype=torch.int32).pin_memory()
    params = swgb.make_params(mat, 11, 1)
    qs = al.seqset(q_res, q_off, stream=stream)
    rs = al.seqset(r_res, r_off, stream=stream)

    def step():
        swgb.swgb_seqset_load(al.ctx, qs.handle, q_res, q_off, stream=stream)
        swgb.swgb_seqset_load(al.ctx, rs.handle, r_res, r_off, stream=stream)
        swgb.swgb_align_host(al.ctx, qs.handle, rs.handle, pairs, params, out, stream)

    step()
    n = max(1, args.steps)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    dt = max_over_ranks((time.perf_counter() - t) / n, dist, dev)
    if dist is not None:
        dist.barrier()
    st = swgb.swgb_last_stats(al.ctx)
    h2d = sum(x.numel() * x.element_size() for x in (q_res, q_off, r_res, r_off, pairs))
    qs.close()
    rs.close()
    return {"value": world * st["forward_cells"] / dt / 1e9, "unit": "GCUPS", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": out.numel() * out.element_size(), "ms_per_step": dt * 1e3,
            "alignments_per_s": world * len(wl.pairs) / dt}


def search_oracle_sample(fs, mat, target_s, seed=5):
    """The oracle pipeline on sampled rows of a family block: k-mer-set merges
    of row i against every sequence, alignment of its partners j > i, identity
    and pass/fail; about target_s seconds."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    ix = oracle.KmerIndex(fs.res, fs.off, 6)
    index_s = time.perf_counter() - t0
    rows, pairs, t_rows = 0, 0, 0.0
    for i in rng.permutation(len(fs)):
        t = time.perf_counter()
        js, _ = ix.candidates_of(int(i), 2)
        js = js[js > i]
        if len(js):
            pr = np.stack([np.full(len(js), i, np.int32), js.astype(np.int32)], axis=1)
            rec = oracle.align_batch(fs.res, fs.off, fs.res, fs.off, pr, mat, 11, 1,
                                     n_threads=cores)
            for p in range(len(pr)):
                a, b = pr[p]
                qs = fs.res[fs.off[a]:fs.off[a + 1]]
                rs = fs.res[fs.off[b]:fs.off[b + 1]]
                mt, cols = oracle.span_identity(qs, rs, rec[p], mat, 11, 1)
                oracle.passes(rec[p], mt, cols, len(qs), len(rs))
        t_rows += time.perf_counter() - t
        rows += 1
        pairs += len(js)
        if t_rows > target_s:
            break
    ix.close()
    # the per-row work is a scan over all sequences, so the block's rate is the
    # sampled rows' candidate rate
    return {"aln_per_s": pairs / t_rows, "rows": rows, "pairs": pairs, "seconds": t_rows,
            "index_s": index_s, "cores": cores}


def run_search(args):
    """The many-against-many block as its own bench line (--workload
    families_200k)."""
    import torch

    from paper_2303_01845_gb300 import swgb

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    al = swgb.Aligner(local)
    line, _, _ = measure_families(args, al, dev, args.workload, args.steps, args.warmup,
                                  None if args.no_cpu_baseline or rank != 0 else args.cpu_seconds,
                                  dist, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def train_filter(al, dev, mat, spec, seed, epochs, recall):
    """The learned filter, trained (untimed) on a family block drawn with
    `seed`: exact labels, features, network, threshold.  Returns (MLP,
    threshold, summary)."""
    import dataclasses

    import torch

    from paper_2303_01845_gb300 import filter as F
    from paper_2303_01845_gb300 import swgb, workload
    t = time.perf_counter()
    fs = workload.generate_families(dataclasses.replace(spec, seed=seed), mat)
    s = al.seqset(torch.from_numpy(fs.res).to(dev), torch.from_numpy(fs.off).to(dev))
    cand, _ = al.discover(s, 6, 2)
    params = swgb.make_params(mat, 11, 1)
    _, ident = F.exact_labels(al, s, cand, params, swgb.make_thresholds())
    X = swgb.swgb_pair_features(al.ctx, s.handle, s.handle, cand)
    y = ident[:, 2].to(torch.float32).contiguous()
    net, losses = F.train(al, X, y, epochs=epochs, batch=8192, lr=3e-3, seed=1)
    threshold = F.calibrate(net, X, y, recall)
    torch.cuda.synchronize()
    summary = {"candidates": int(cand.shape[0]), "passing": int(y.sum().item()), "epochs": epochs,
               "seconds": time.perf_counter() - t, "final_loss": losses[-1], "seed": seed}
    del cand, ident, X, y
    s.close()
    return net, threshold, summary


def measure_families(args, al, dev, name, steps, warmup, cpu_seconds, dist=None, world=1):
    """The many-against-many block: discovery + alignment + identity, plain and
    with the learned filter (trained beforehand, untimed, on a block drawn
    with another seed).  Returns (bench line, trained network parameters,
    threshold)."""
    import ctypes
    import dataclasses

    import numpy as np
    import torch

    from paper_2303_01845_gb300 import swgb, workload

    mat = swgb.swgb_blosum62()
    spec = workload.FAMILY_SPECS[name]
    stream = torch.cuda.current_stream(dev)
    params = swgb.make_params(mat, 11, 1, timing=True)
    th = swgb.make_thresholds()
    lib = swgb.load()

    # ---- training block (untimed): exact labels, features, network, threshold
    net, threshold, trained = train_filter(al, dev, mat, spec, spec.seed + 1, args.filter_epochs,
                                           args.filter_recall)
    # the aligner's knobs (tile overhead, band threshold) of each pipeline:
    # plain keeps the context's; filtered is tuned (untimed) on this block's
    # kept pairs after the first warm-up step, as the batched line is tuned
    # on its own batch
    saved_knobs = (swgb.swgb_get_tile_overhead(al.ctx), swgb.swgb_get_band_min(al.ctx))
    knobs = {"plain": {"tile_overhead": saved_knobs[0], "band_min": saved_knobs[1]}}

    def use_knobs(pipeline):
        if pipeline in knobs:
            swgb.swgb_set_tile_overhead(al.ctx, knobs[pipeline]["tile_overhead"])
            swgb.swgb_set_band_min(al.ctx, knobs[pipeline]["band_min"])

    # ---- the measured block
    fs = workload.generate_families(dataclasses.replace(spec, seed=spec.seed), mat)
    s = al.seqset(torch.from_numpy(fs.res).to(dev), torch.from_numpy(fs.off).to(dev))
    cap = al.discover(s, 6, 2)[0].shape[0]
    cand = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    counts = torch.empty((cap,), dtype=torch.int32, device=dev)
    rec = torch.empty((cap, 5), dtype=torch.int32, device=dev)
    ident = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    feats = torch.empty((cap, 32), dtype=torch.float32, device=dev)
    logits = torch.empty((cap,), dtype=torch.float32, device=dev)
    kept = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    kept_index = torch.empty((cap,), dtype=torch.int64, device=dev)
    rec_k = torch.empty((cap, 5), dtype=torch.int32, device=dev)
    ident_k = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    n_found = ctypes.c_int64()
    n_kept = ctypes.c_int64()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    plain = {"discover": [], "align": [], "identity": [], "step": [], "fwd": []}
    filt = {"features": [], "network": [], "select": [], "align": [], "identity": [], "step": []}
    launches = {"plain": 0, "filtered": 0}
    band_stats = {}

    def discover():
        swgb._check(al.ctx, lib.swgb_discover(al.ctx, s.handle, 6, 2, cand.data_ptr(),
                                              counts.data_ptr(), cap, ctypes.byref(n_found),
                                              stream.cuda_stream))
        return lib.swgb_search_launches(al.ctx)

    def plain_step(timed):
        use_knobs("plain")
        ev[0].record(stream)
        nl = discover()
        ev[1].record(stream)
        swgb.swgb_align(al.ctx, s.handle, s.handle, cand, params, rec, stream)
        ev[2].record(stream)
        swgb.swgb_identity(al.ctx, s.handle, s.handle, cand, rec, params, th, ident, stream)
        nl += lib.swgb_search_launches(al.ctx)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if timed:
            plain["discover"].append(ev[0].elapsed_time(ev[1]))
            plain["align"].append(ev[1].elapsed_time(ev[2]))
            plain["identity"].append(ev[2].elapsed_time(ev[3]))
            plain["step"].append(ev[0].elapsed_time(ev[3]))
            st = swgb.swgb_last_stats(al.ctx)
            plain["fwd"].append(st["forward_ms"])
            launches["plain"] += nl + st["kernel_launches"]
            return st
        return None

    def filtered_step(timed):
        use_knobs("filtered")
        ev[0].record(stream)
        nl = discover()
        ev[1].record(stream)
        swgb.swgb_pair_features(al.ctx, s.handle, s.handle, cand, 6, feats, stream)
        nl += lib.swgb_search_launches(al.ctx)
        ev[2].record(stream)
        net.forward(feats, logits, stream)
        ev[3].record(stream)
        swgb._check(al.ctx, lib.swgb_select_pairs(al.ctx, cand.data_ptr(), logits.data_ptr(), cap,
                                                  ctypes.c_float(threshold), kept.data_ptr(),
                                                  kept_index.data_ptr(), ctypes.byref(n_kept),
                                                  stream.cuda_stream))
        nl += lib.swgb_search_launches(al.ctx) + 1
        ev[4].record(stream)
        k = n_kept.value
        kp = kept[:k]
        swgb.swgb_align(al.ctx, s.handle, s.handle, kp, params, rec_k[:k], stream)
        ev[5].record(stream)
        swgb.swgb_identity(al.ctx, s.handle, s.handle, kp, rec_k[:k], params, th, ident_k[:k], stream)
        nl += lib.swgb_search_launches(al.ctx)
        ev[6].record(stream)
        torch.cuda.synchronize()
        if timed:
            for key, a, b in (("features", 1, 2), ("network", 2, 3), ("select", 3, 4),
                              ("align", 4, 5), ("identity", 5, 6), ("step", 0, 6)):
                filt[key].append(ev[a].elapsed_time(ev[b]))
            filt.setdefault("discover", []).append(ev[0].elapsed_time(ev[1]))
            st = swgb.swgb_last_stats(al.ctx)
            launches["filtered"] += nl + st["kernel_launches"]
            filt.setdefault("align_forward", []).append(st["forward_ms"])
            filt.setdefault("align_reverse", []).append(st["reverse_ms"])
            band_stats.update(pairs=st["n_band_pairs"], certified=st["n_band_certified"])

    tune_s = 0.0
    for w_ in range(warmup):
        plain_step(False)
        filtered_step(False)
        if w_ == 0 and not args.no_tune:
            t_ = time.perf_counter()
            k = n_kept.value
            tmp = torch.empty((max(k, 1), 5), dtype=torch.int32, device=dev)
            swgb.swgb_autotune(al.ctx, s.handle, s.handle, kept[:k], params, tmp[:k])
            tu = swgb.swgb_last_tuning(al.ctx)
            knobs["filtered"] = {"tile_overhead": tu["tile_overhead"], "band_min": tu["band_min"],
                                 "tuned_ms": round(tu["best_ms"], 3), "band_off_ms": round(tu["band_off_ms"], 3),
                                 "tuned_pairs": int(k)}
            del tmp
            tune_s = time.perf_counter() - t_
    stats = None
    with ClockSampler(dev.index) as clocks:
        torch.cuda.synchronize()
        for _ in range(steps):
            stats = plain_step(True)
            filtered_step(True)
    clock = clocks.summary()
    assert n_found.value == cap
    plain_ms = max_over_ranks(sum(plain["step"]), dist, dev)
    filt_ms = max_over_ranks(sum(filt["step"]), dist, dev)
    plain_rate = job_rate(cap, world, steps, plain_ms)
    filt_rate = job_rate(cap, world, steps, filt_ms)
    # recall of the filter against the exact pass / fail of every candidate
    y = ident[:, 2].cpu().numpy() > 0
    keep = np.zeros(cap, bool)
    keep[kept_index[:n_kept.value].cpu().numpy()] = True
    same = bool(np.array_equal(ident_k[:n_kept.value].cpu().numpy(), ident.cpu().numpy()[keep]))
    recall = float(keep[y].mean()) if y.any() else None
    cnt = counts.cpu().numpy()
    cpu = None
    if cpu_seconds:
        cpu = search_oracle_sample(fs, np.asarray(mat), cpu_seconds)
    mlp_params = net.get()
    net.close()
    s.close()
    mean = lambda d, k: statistics.mean(d[k])
    line = {
        "metric": METRIC, "value": filt_rate, "unit": "alignments/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": filt_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i16x2+i32 align, bf16 net", "data": "synthetic",
        "config": {"workload": name, "sequences": len(fs), "residues": int(fs.off[-1]),
                   "k": 6, "min_shared": 2, "candidates": cap,
                   "forward_cells": stats["forward_cells"],
                   "passing_pairs": int(y.sum()),
                   "thresholds": "identity >= 3/10, coverage >= 7/10",
                   "value_is": "candidates judged per second by the filtered pipeline "
                               "(discovery, features, network, selection, exact alignment and "
                               "identity of the kept pairs)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "filter": {"recall": recall, "kept": int(n_kept.value), "kept_fraction": n_kept.value / cap,
                   "kept_results_exact": same, "threshold": threshold,
                   "trained_on": "%s seed %d: %d candidates, %d passing; %d epochs, %.1f s "
                                 "(labels, features, training)" %
                                 (name, trained["seed"], trained["candidates"], trained["passing"],
                                  trained["epochs"], trained["seconds"]),
                   "final_loss": trained["final_loss"],
                   "align_band": band_stats,
                   "aligner_knobs": dict(knobs, tuned_on=(
                       "filtered: this block's kept pairs, after the first warm-up step (untimed, "
                       "%.1f s), as the batched line is tuned on its batch; plain: the context's knobs"
                       % tune_s) if "filtered" in knobs else "not tuned: both pipelines on the context's knobs"),
                   "kmer_threshold_3": {"recall": float((cnt[y] >= 3).mean()) if y.any() else None,
                                        "kept_fraction": float((cnt >= 3).mean())},
                   "speedup_vs_plain": filt_rate / plain_rate,
                   "ms": {k: mean(filt, k) for k in filt}},
        "plain": {"alignments_per_s": plain_rate, "ms_per_step": plain_ms / steps,
                  "discover_ms": mean(plain, "discover"), "align_ms": mean(plain, "align"),
                  "identity_ms": mean(plain, "identity"), "forward_ms": mean(plain, "fwd"),
                  "gcups_forward_kernel": stats["forward_cells"] / (mean(plain, "fwd") / 1e3) / 1e9},
        "cpu_baseline": None if cpu is None else {
            "value": cpu["aln_per_s"], "unit": "alignments/s", "cores": cpu["cores"],
            "kind": "oracle",
            "sample": "%d random rows (%d candidates j > i): k-mer-set merges against all %d "
                      "sequences, alignment, identity; %.1f s (+ %.1f s k-mer index)" %
                      (cpu["rows"], cpu["pairs"], len(fs), cpu["seconds"], cpu["index_s"])},
        "gpu_launches": launches["filtered"],
        "clocks": {"sm_mhz": clock["sm_mhz"], "sm_max_mhz": clock["sm_max_mhz"],
                   "reasons": clock["reasons"]},
    }
    swgb.swgb_set_tile_overhead(al.ctx, saved_knobs[0])
    swgb.swgb_set_band_min(al.ctx, saved_knobs[1])
    return line, mlp_params, threshold


def run_serving(args):
    """The query server as its own bench line (--workload serving_1m)."""
    import torch

    from paper_2303_01845_gb300 import swgb, workload

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mat = swgb.swgb_blosum62()
    al = swgb.Aligner(local)
    net, threshold, trained = train_filter(al, dev, mat, workload.FAMILY_SPECS["families_200k"], 4,
                                           args.filter_epochs, args.filter_recall)
    mlp_params = net.get()
    net.close()
    line = measure_serving(args, al, dev, mlp_params, threshold, trained["seconds"],
                           args.serve_requests, args.serve_rate, args.warmup)
    print(json.dumps(line), flush=True)


def measure_serving(args, al, dev, mlp_params, threshold, train_s, n_requests, rate, warmup):
    """The query server over args.serve_refs resident references: requests of
    1 to 1,000 queries arrive as a Poisson process at `rate`; each goes
    through shared-6-mer candidates from the resident index, the learned
    filter, exact alignment and identity.  Latency = submission to completion
    of a request.  Returns the bench line."""
    import numpy as np
    import torch

    from paper_2303_01845_gb300 import swgb, workload

    mat = swgb.swgb_blosum62()
    params = swgb.make_params(mat, 11, 1)
    # ---- resident references: families x 10 copies; queries: an 11th copy
    n_fam = args.serve_refs // 10
    spec = workload.FamilySpec("serving_refs", n_fam, 11, "lognormal", 20, 5000, median=250.0,
                               sigma=0.7, seed=5)
    fs = workload.generate_families(spec, mat)
    n = len(fs)
    is_q = np.zeros(n, bool)
    is_q[np.arange(10, n, 11)] = True

    def pack(idx):
        lens = (fs.off[idx + 1] - fs.off[idx]).astype(np.int64)
        off = np.zeros(len(idx) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        take = np.repeat(fs.off[idx] - off[:-1], lens) + np.arange(int(off[-1]), dtype=np.int64)
        return fs.res[take].astype(np.uint8), off
    rr, ro = pack(np.nonzero(~is_q)[0])
    qr, qo = pack(np.nonzero(is_q)[0])
    t_index = time.perf_counter()
    refs = al.seqset(torch.from_numpy(rr).to(dev), torch.from_numpy(ro).to(dev))
    index = swgb.Index(al, refs, 6)
    torch.cuda.synchronize()
    t_index = time.perf_counter() - t_index
    srv = swgb.Server(refs, index, params, mlp_params, device=dev.index, slots=args.serve_slots,
                      threshold=threshold, max_batch_queries=4096, max_batch_residues=1 << 21,
                      max_inflight_bytes=8 << 30, candidates_per_query=1024)
    rng = np.random.default_rng(17)
    nq_pool = len(qo) - 1

    def make_request():
        size = int(rng.integers(1, 1001))
        q0 = int(rng.integers(0, nq_pool - size))
        off = qo[q0:q0 + size + 1] - qo[q0]
        return qr[qo[q0]:qo[q0 + size]], off

    for _ in range(warmup):
        srv.wait(srv.submit(*make_request()))
    reqs = [make_request() for _ in range(n_requests)]
    gaps = rng.exponential(1.0 / rate, len(reqs))
    tickets = []
    with ClockSampler(dev.index) as clocks:
        t0 = time.perf_counter()
        next_t = t0
        for (c, o), g in zip(reqs, gaps):
            next_t += g
            delay = next_t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(c, o))
        results = [srv.wait(tk) for tk in tickets]
        wall = time.perf_counter() - t0
    clock = clocks.summary()
    lat = np.array([r["latency_ms"] for r in results])
    queue = np.array([r["queue_ms"] for r in results])
    aligned = sum(len(r["records"]) for r in results)
    cands = sum(r["candidates"] for r in results)
    queries = sum(len(o) - 1 for _, o in reqs)
    passing = sum(int(r["identity"][:, 2].sum()) for r in results if len(r["identity"]))
    stats = srv.stats()
    info = index.info()
    srv.close()
    index.close()
    refs.close()
    return {
        "metric": METRIC, "value": aligned / wall, "unit": "alignments/s", "n_gpus": 1,
        "steps": len(reqs), "warmup": warmup, "ms_per_step": 1000 * wall / len(reqs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i16x2+i32 align, bf16 net", "data": "synthetic",
        "config": {"workload": "serving_%dk" % (args.serve_refs // 1000),
                   "references": int(len(ro) - 1), "reference_residues": int(ro[-1]),
                   "requests": len(reqs), "queries_per_request": "uniform 1..1000",
                   "arrivals": "Poisson, %.1f requests/s" % rate,
                   "slots": args.serve_slots, "index_bytes": info["bytes"],
                   "index_build_s": t_index, "filter_training_s": train_s,
                   "filter_threshold": threshold,
                   "step": "one request (submission to completion)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "queue_ms": {"p50": float(np.percentile(queue, 50)), "p99": float(np.percentile(queue, 99))},
        "batch_stage_ms_p50": dict(zip(["load", "candidates", "filter", "align_identity", "results"],
                                       [float(v) for v in np.median(
                                           np.array([r["stage_ms"] for r in results]), axis=0)])),
        "throughput": {"alignments_per_s": aligned / wall, "candidates_per_s": cands / wall,
                       "queries_per_s": queries / wall, "requests_per_s": len(reqs) / wall,
                       "passing_pairs": passing, "aligned_pairs": aligned, "candidates": cands,
                       "wall_s": wall},
        "max_batches_in_flight": stats["max_overlap"],
        "clocks": {"sm_mhz": clock["sm_mhz"], "sm_max_mhz": clock["sm_max_mhz"],
                   "reasons": clock["reasons"]},
    }


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("families"):
        run_search(args)
    elif args.workload.startswith("serving"):
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
