"""Benchmark: the large-nucleus correlator (2 flavours, n_f = 18, L = 96, 32768 x 32768 source x
sink terms in families of 32, 10 % of the families with two changed rows, 1 % of the members
forced near-singular) evaluated on the GPU through the C ABI, with the other workloads as
sub-objects of the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mhc|reference] [--workload NAME]

One step = one mhc_correlator call (every step of the hot path: block factors, cached solves,
member dot products, refactors of the guarded pairs, fixed-order reduction) for one
propagator set.  The plan (Sec. 3: graph + dominating set) is built once before timing, as the
paper amortises it over gauge configurations.  Between timed steps L2 is flushed by writing a
256 MiB buffer (outside the timed events); the block factors of one call (9.7 GB) exceed L2 as
well.  Under torchrun every rank evaluates its own independent correlator (its own
propagators: another gauge configuration), so the work per GPU is fixed ("weak" scaling) and
no collective is on the data path; rank 0 prints one JSON line with the whole-job pairs/s over
the slowest rank.

Sub-objects of the line (rank 0, N = 1 unless --headline-only):
  one_sided  the same workload planned with opts.one_sided = 1 (Sec. 3 as printed: source
             families only), time and fraction of the FP64 peak;
  row_difference  the same workload with opts.row_difference = 1 (one-row members that fail
             the lemma guard are updated from the difference of their row and the nearest
             shared row before a refactor), time and fraction of the FP64 peak;
  configs    the deuteron-like (512 x 512, n = 3) and He-4-like (4096 x 4096, n = 6) forward
             calls, the 64-correlator batch (one CUDA graph vs 64 sequential calls) and the
             adjoint on the He-4-like shapes (backward vs forward time).

--impl reference times the oracle (plain CPU FP64, fresh LU per pair) on the host cores on a
bounded sample of seeded pairs of the same workload, with the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "src×snk det pairs/sec (cplx FP64), % roofline; batched & adjoint vs plain GPU"
UNIT = "pairs/s"
# FP64 peak from unit counts and clocks: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop
NOMINAL_FP64_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum of every kernel of one forward call, from one
# ncu capture of the current kernels.  The large nucleus holds 9.7 GB of block factors, too much
# for a multi-metric capture, so its 1/8-per-side copy (--workload large_small: 1/64 of the pairs
# and of the (family, sink family) blocks) was captured and the sum scaled by 64: 165.9 MB read
# + 99.5 MB written per call of the copy (kfac_kernel, kfac_group_kernel, three fwd_kernel
# launches, reduce_kernel).
TRAFFIC = {
    "large": {"bytes": 269.78e6 * 64,
              "source": "ncu dram__bytes_read + dram__bytes_write of every kernel of one call of the "
                        "1/8-per-side copy (--workload large_small), x 64"},
    "he4": {"bytes": 108.71e6,
            "source": "ncu dram__bytes_read + dram__bytes_write of every kernel of one call"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mhc", choices=["mhc", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "he4", "deuteron", "large_noforce", "large_small"],
                    help="large (the benchmark line), he4, deuteron, or the n = 18 variants without "
                         "forced members / at 1/8 scale per side (for profiler captures)")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the selected workload only (no sub-objects, no CPU baseline)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the adjoint of the selected workload alone and print its sub-object "
                         "(for profiler captures)")
    ap.add_argument("--batch", action="store_true",
                    help="time the 64-correlator batch alone and print its sub-object (for profiler "
                         "captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--row-difference", action="store_true",
                    help="plan with opts.row_difference = 1 (recorded in config)")
    ap.add_argument("--scale", type=float, default=1.0, help=argparse.SUPPRESS)  # tests: shrink the workload
    ap.add_argument("--cpu-pairs", type=int, default=100000,
                    help="seeded (i, j) pairs the oracle evaluates for cpu_baseline / --impl reference")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="only measure the FP64 (DFMA) peak: >= 1 s of independent chains on every SM, "
                         "SM clocks sampled meanwhile")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int, name: str = "large", scale: float = 1.0):
    """The rank's own replica on its own propagators (seed); scale < 1 shrinks the family
    counts (tests)."""
    from paper_1411_3691_gb300 import workloads as wl
    if name == "he4":
        return wl.helium4(scale=scale, seed=1000 + 17 * rank)
    if name == "deuteron":
        return wl.deuteron(scale=scale, seed=17 * rank)
    if name == "large":
        return wl.large_nucleus(scale=scale, seed=3000 + 17 * rank)
    if name == "large_small":
        return wl.large_nucleus(scale=scale / 8, seed=3000 + 17 * rank)
    if name == "large_noforce":
        fams = [32] * max(1, int(round(1024 * scale)))
        return wl.make_workload("large_noforce_n18_L96", [18, 18], [96, 96], fams, fams, diag=3.0,
                                seed=3000 + 17 * rank, two_row_frac=0.1, forced_frac=0.0, twins=8)
    raise ValueError(f"unknown workload {name}")


def forward_launches(plan, w, st) -> int:
    """Kernel launches of one forward call: the block factors of a two-sided plan (one
    launch, two when a flavour has n > 6), fwd_kernel once per group of families that share
    a y-cache layout (the rank of each flavour; one launch when all share one, at most
    four), and the reduction."""
    keys = {tuple(max(1, int(r)) if n > 0 else 0 for r, n in zip(row, w.n_f))
            for row in plan.families()["rank"]}
    fwd = 1 if len(keys) < 2 else min(len(keys), 4)
    kfac = (1 + (max(w.n_f) > 6)) if st["two_sided_blocks"] > 0 else 0
    return kfac + fwd + 1


def max_over_ranks(x: float, pg, device) -> float:
    """The slowest rank's time: every rank gets the maximum (all-reduce MAX)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, pairs_per_rank: int, ms_per_step: float) -> float:
    """Pairs per second of the whole job: every rank evaluates its own correlator of
    pairs_per_rank pairs per step, the job's step lasting as long as its slowest rank."""
    return world * pairs_per_rank / (ms_per_step * 1e-3)


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_pair_rate(w, n_pairs: int, seed: int = 31):
    """The oracle (fresh partial-pivot LU per pair per flavour) on n_pairs seeded random
    (i, j) pairs of the workload on all host cores, and the sampled pairs' share of C
    (sum of w_i w_j prod_f det); returns (pairs/s, seconds, threads)."""
    import numpy as np

    import oracle
    threads = cores()
    rng = np.random.default_rng(seed)
    ii = rng.integers(0, len(w.w_src), n_pairs)
    jj = rng.integers(0, len(w.w_snk), n_pairs)
    t0 = time.perf_counter()
    d = oracle.pair_dets(w.S, w.n_f, w.labels_src, w.labels_snk, ii, jj, threads=threads)
    _ = float(np.sum(w.w_src[ii] * w.w_snk[jj] * np.prod(d, axis=1)).real)
    dt = time.perf_counter() - t0
    return n_pairs / dt, dt, threads


def cpu_baseline(w, n_pairs: int):
    rate, dt, threads = oracle_pair_rate(w, n_pairs)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_pairs} seeded random (i, j) pairs of the {len(w.w_src)} x {len(w.w_snk)} "
                      f"workload (fresh partial-pivot LU per pair per flavour, w_i w_j prod det summed), "
                      f"{dt:.2f} s on {threads} threads; rate extrapolated to all {w.pairs} pairs "
                      f"({w.pairs / rate:.0f} s)"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3][k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def workload_config(w, st=None):
    cfg = {"workload": w.name, "flavours": len(w.n_f), "n_f": w.n_f[0], "L": w.L_f[0],
           "n_src": len(w.w_src), "n_snk": len(w.w_snk), "pairs_per_gpu": w.pairs}
    if st is not None:
        cfg.update({"families": st["families"], "sink_families": st["sink_families"],
                    "two_row_family_flavours": st["rank2_family_flavours"]})
    forced = w.meta.get("src", {}).get("forced") if w.meta else None
    if forced:
        cfg["forced_near_singular_member_flavours"] = len(forced)
    return cfg


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(0, args.workload, args.scale)
    rates, secs = [], 0.0
    threads = cores()
    for s in range(args.warmup + args.steps):
        r, dt, threads = oracle_pair_rate(w, args.cpu_pairs, seed=31 + s)
        if s >= args.warmup:
            rates.append(r)
            secs += dt
    value = sum(rates) / len(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / len(rates) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"per step {args.cpu_pairs} seeded random (i, j) pairs of the "
                                       f"{len(w.w_src)} x {len(w.w_snk)} workload (fresh partial-pivot LU "
                                       f"per pair per flavour), rate extrapolated to all {w.pairs} pairs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_forward(plan, S, out, flush, stream, steps: int, warmup: int = 2):
    """Average CUDA-event time (ms) of one mhc_correlator call, L2 flushed between calls."""
    import torch
    for _ in range(warmup):
        plan.correlator(S, out=out)
    torch.cuda.synchronize()
    plan.status()
    tot = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.correlator(S, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    plan.status()
    return tot / steps


def run_gpu(args):
    import torch

    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.adjoint or args.batch:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        peak = mhc.mhc_fp64_peak(250000) / 1e12
        stream = torch.cuda.current_stream()
        if args.adjoint:
            r = time_adjoint(mhc, workload(rank, args.workload), flush, stream, peak, steps=args.steps)
        else:
            r = time_batch(mhc, flush, stream, peak, reps=args.steps)
        print(json.dumps({"adjoint" if args.adjoint else "batch": r}), flush=True)
        return
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    w = workload(rank, args.workload)
    extras = not args.headline_only and world == 1 and rank == 0
    hopts = mhc.default_opts()
    hopts.row_difference = 1 if args.row_difference else 0
    plan = mhc.Plan.from_workload(w, hopts)
    st = plan.stats()
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # FP64 peak on this GPU (DFMA chains on every SM), taken before the warm-up so that the
    # timed steps follow the warm-up directly
    peak_flops = mhc.mhc_fp64_peak(250000)

    # warm-up (the first call uploads the plan)
    for _ in range(max(args.warmup, 3)):
        plan.correlator(S, out=out)
    torch.cuda.synchronize()
    plan.status()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            plan.correlator(S, out=out)
            ends[k].record(stream)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.summary()
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.steps)]
    total_ms = sum(step_ms)
    plan.status()
    st = plan.stats()
    total_ms = max_over_ranks(total_ms, pg, "cuda")
    pairs = w.pairs
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, pairs, ms_per_step)

    # roofline (FP64 ALU bound): algorithmic flops of one call -- the planned update scheme
    # plus the refactor path as the device counted it -- over the whole step's device time
    # (every launch of the call), against the FP64 peak measured above
    refactor_pairs = (st["refactor_parent"] + st["refactor_child"]) / max(args.steps, 1)
    rowdiff_pairs = st["row_difference"] / max(args.steps, 1)
    refactor_flops = st["refactor_flops"] / max(args.steps, 1)
    flops = st["flops_per_call"] + refactor_flops
    achieved = flops / (ms_per_step * 1e-3) / 1e12
    peak = peak_flops / 1e12

    # end to end through the public API: pinned host propagators -> device, correlator,
    # result -> host, every step
    hS = [torch.from_numpy(s).pin_memory() for s in w.S]
    hout = torch.empty(2, dtype=torch.float64).pin_memory()
    dS = [torch.empty_like(s, device="cuda") for s in hS]
    for _ in range(2):
        for d, h in zip(dS, hS):
            d.copy_(h, non_blocking=True)
        plan.correlator(dS, out=out)
        hout.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(e2e_steps):
        for d, h in zip(dS, hS):
            d.copy_(h, non_blocking=True)
        plan.correlator(dS, out=out)
        hout.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, pg, "cuda")
    h2d = sum(h.numel() * h.element_size() for h in hS)
    plan.status()
    C = [float(out[0].item()), float(out[1].item())]

    launches = forward_launches(plan, w, st)
    one_sided = rowdiff = configs = None
    if extras:
        one_sided = time_one_sided(mhc, w, S, out, flush, stream, ms_per_step, peak)
        rowdiff = time_row_difference(mhc, w, S, out, flush, stream, ms_per_step, peak)
    plan.close()
    if extras:
        configs = {
            "deuteron": time_config(mhc, workload(0, "deuteron"), flush, stream, peak, steps=20),
            "he4": time_config(mhc, workload(0, "he4"), flush, stream, peak, steps=20),
            "batch": time_batch(mhc, flush, stream, peak),
            "adjoint_he4": time_adjoint(mhc, workload(0, "he4"), flush, stream, peak),
            "mixed_rows": time_grouping(mhc, flush, stream, peak),
        }

    if rank == 0:
        traffic = None if args.row_difference else TRAFFIC.get(args.workload)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w, st), **{
                "parallelism": f"{world} independent correlators (one per GPU)",
                "row_difference": bool(args.row_difference),
                "l2": "flushed between timed steps (256 MiB write outside the events); the call's "
                      "block factors exceed L2"}),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": traffic["bytes"] if traffic else None,
                         "traffic_source": traffic["source"] if traffic else None,
                         "peak_source": "FP64 DFMA chains on all SMs, measured in this run "
                                        f"(nominal {NOMINAL_FP64_TFLOPS:.3f} from unit counts and clocks)",
                         "flops_per_step": flops,
                         "flops_planned": st["flops_per_call"], "flops_refactor": refactor_flops,
                         "time_base": "whole step (every launch of one call)"},
            "e2e": {"value": whole_job_rate(world, pairs, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 16, "steps": e2e_steps},
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
            "refactors_per_step": refactor_pairs,
            "row_difference_per_step": rowdiff_pairs,
            "one_sided": one_sided,
            "row_difference": rowdiff,
            "configs": configs,
            "C": C,
        }
        if extras and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_pairs)
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def time_one_sided(mhc, w, S, out, flush, stream, two_ms, peak):
    """The same workload with opts.one_sided = 1: source families only, the shared rows
    factorised per (family, sink, flavour) -- the execution order of Sec. 3 as printed."""
    opts = mhc.default_opts()
    opts.one_sided = 1
    plan = mhc.Plan.from_workload(w, opts)
    ms = time_forward(plan, S, out, flush, stream, steps=3, warmup=2)
    st = plan.stats()
    flops = st["flops_per_call"] + st["refactor_flops"] / 3
    plan.close()
    return {"ms_per_step": ms, "pairs_per_s": w.pairs / (ms * 1e-3), "tflops": flops / (ms * 1e-3) / 1e12,
            "frac_of_fp64_peak": flops / (ms * 1e-3) / 1e12 / peak, "flops_per_step": flops,
            "two_sided_speedup": ms / two_ms}


def time_row_difference(mhc, w, S, out, flush, stream, ref_ms, peak, steps=5):
    """The same workload with opts.row_difference = 1: one-row members that fail the lemma
    guard take the row-difference update (det [A; b] = det [A; b - a_r]) and are refactored
    only if it fails its own guard."""
    opts = mhc.default_opts()
    opts.row_difference = 1
    plan = mhc.Plan.from_workload(w, opts)
    ms = time_forward(plan, S, out, flush, stream, steps=steps, warmup=2)
    st = plan.stats()
    flops = st["flops_per_call"] + st["refactor_flops"] / steps
    plan.close()
    return {"ms_per_step": ms, "pairs_per_s": w.pairs / (ms * 1e-3), "tflops": flops / (ms * 1e-3) / 1e12,
            "frac_of_fp64_peak": flops / (ms * 1e-3) / 1e12 / peak, "flops_per_step": flops,
            "refactors_per_step": (st["refactor_parent"] + st["refactor_child"]) / steps,
            "row_difference_per_step": st["row_difference"] / steps,
            "speedup_vs_refactor": ref_ms / ms}


def time_config(mhc, w, flush, stream, peak, steps=20, opts=None):
    """Forward of another workload: CUDA-event time per call and fraction of the FP64 peak."""
    import torch
    plan = mhc.Plan.from_workload(w, opts)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    ms = time_forward(plan, S, out, flush, stream, steps=steps)
    st = plan.stats()
    flops = st["flops_per_call"] + st["refactor_flops"] / steps
    res = {"workload": w.name, "ms_per_step": ms, "pairs_per_s": w.pairs / (ms * 1e-3),
           "tflops": flops / (ms * 1e-3) / 1e12, "frac_of_fp64_peak": flops / (ms * 1e-3) / 1e12 / peak,
           "flops_per_step": flops, "gpu_launches_per_step": forward_launches(plan, w, st)}
    plan.close()
    return res


def time_grouping(mhc, flush, stream, peak):
    """Families whose members change rows of their own (2 flavours, n_f = 12, L = 60, 4096 x
    4096 terms, source families of 32): the work families split by the plan's flop count
    (the default) against first fit, both timed."""
    from paper_1411_3691_gb300 import workloads as wl
    w = wl.make_workload("mixed_rows_n12_L60_4096x4096", [12, 12], [60, 60], [32] * 128, [16] * 256, seed=7,
                         mixed_rows=True)
    ff = mhc.default_opts()
    ff.first_fit = 1
    cost = time_config(mhc, w, flush, stream, peak)
    first = time_config(mhc, w, flush, stream, peak, opts=ff)
    return {"cost_grouping": cost, "first_fit": first,
            "flops_ratio": cost["flops_per_step"] / first["flops_per_step"],
            "speedup": first["ms_per_step"] / cost["ms_per_step"]}


def time_adjoint(mhc, w, flush, stream, peak, steps=10):
    """Backward (dS_f, dw_src, dw_snk for L = Re C) of the He-4-like workload, CUDA events,
    against its own forward call."""
    import torch
    plan = mhc.Plan.from_workload(w)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    fwd_ms = time_forward(plan, S, out, flush, stream, steps=steps)
    g = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    dS = [torch.empty_like(s) for s in S]
    dws = torch.empty(plan.n_src, dtype=torch.float64, device="cuda")
    dwk = torch.empty(plan.n_snk, dtype=torch.float64, device="cuda")
    for _ in range(2):
        mhc.mhc_correlator_backward(plan.handle, S, g, None, None, dS, dws, dwk)
    torch.cuda.synchronize()
    tot = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mhc.mhc_correlator_backward(plan.handle, S, g, None, None, dS, dws, dwk)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / steps
    plan.status()
    st = plan.stats()
    bflops = st["backward_flops_per_call"]
    res = {"workload": w.name, "ms_per_step": ms, "forward_ms_per_step": fwd_ms, "ratio_vs_forward": ms / fwd_ms,
           "pairs_per_s": w.pairs / (ms * 1e-3), "tflops": bflops / (ms * 1e-3) / 1e12,
           "frac_of_fp64_peak": bflops / (ms * 1e-3) / 1e12 / peak, "flops_per_step": bflops,
           "outputs": f"dS_f ({len(w.n_f)} x {w.L_f[0]} x {w.L_f[0]} complex), dw_src [{len(w.w_src)}], "
                      f"dw_snk [{len(w.w_snk)}]; L = Re C",
           # block factors and B^-1 (two-sided plans), the adjoint kernel, one dS finalize per
           # flavour, the two weight finalizes
           "gpu_launches_per_step": (3 if st["two_sided_blocks"] > 0 else 1) + len(S) + 2}
    plan.close()
    return res


def time_batch(mhc, flush, stream, peak, count=64, reps=10):
    """64 independent correlators of mixed n_f in one persistent launch under a CUDA graph,
    against 64 sequential mhc_correlator calls on the same plans and propagators."""
    import torch
    from paper_1411_3691_gb300 import workloads as wl
    items = wl.batch(count)
    plans = [mhc.Plan.from_workload(w) for w in items]
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    pairs = sum(w.pairs for w in items)
    # the autotuner's cache in a file of this run (the first create times every class, the
    # second finds each class's tile in the cache)
    cache = tempfile.NamedTemporaryFile(suffix=".jsonl", delete=False)
    cache.close()
    os.unlink(cache.name)
    saved = os.environ.get("MHC_TUNE_CACHE")
    os.environ["MHC_TUNE_CACHE"] = cache.name
    t0 = time.perf_counter()
    first = mhc.mhc_batch_create([p.handle for p in plans])
    create_s = time.perf_counter() - t0
    tiles, _, tune_ms = mhc.mhc_batch_shape(first)
    mhc.mhc_batch_destroy(first)
    t0 = time.perf_counter()
    batch = mhc.mhc_batch_create([p.handle for p in plans])
    create2_s = time.perf_counter() - t0
    tiles2, cached, _ = mhc.mhc_batch_shape(batch)
    if saved is None:
        del os.environ["MHC_TUNE_CACHE"]
    else:
        os.environ["MHC_TUNE_CACHE"] = saved
    if os.path.exists(cache.name):
        os.unlink(cache.name)
    T, n_items = mhc.mhc_batch_info(batch)
    outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in items]
    mhc.mhc_batch_correlator(batch, S, outs)
    for p, Sk, o in zip(plans, S, outs):
        p.correlator(Sk, out=o)
    torch.cuda.synchronize()

    def timed(fn):
        tot = 0.0
        for r in range(reps):
            flush.fill_(float(r))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    batch_ms = timed(lambda: mhc.mhc_batch_correlator(batch, S, outs))
    seq_ms = timed(lambda: [p.correlator(Sk, out=o) for p, Sk, o in zip(plans, S, outs)])
    flops = sum(p.stats()["flops_per_call"] for p in plans)
    for p in plans:
        p.status()
    mhc.mhc_batch_destroy(batch)
    for p in plans:
        p.close()
    return {"workload": f"{count} correlators: n_f ~ U{{3,6,9,12,18}} per flavour, L = 12 ceil(n/3) + 12, "
                        "terms per side log-U[256, 16384], family sizes U[1, 32] (seeds 2000 + b)",
            "pairs": pairs, "ms": batch_ms, "pairs_per_s": pairs / (batch_ms * 1e-3),
            "tflops": flops / (batch_ms * 1e-3) / 1e12, "frac_of_fp64_peak": flops / (batch_ms * 1e-3) / 1e12 / peak,
            "sequential_ms": seq_ms, "sequential_pairs_per_s": pairs / (seq_ms * 1e-3),
            "speedup_vs_sequential": seq_ms / batch_ms, "reps": reps, "tile": T, "work_items": n_items,
            "tiles_by_n_class": {"n<=8": tiles[0], "n<=18": tiles[1], "n<=32": tiles[2]},
            "tuning_ms_by_n_class": {"n<=8": tune_ms[0], "n<=18": tune_ms[1], "n<=32": tune_ms[2]},
            "batch_create_s": create_s, "batch_create_cached_s": create2_s,
            "second_create_from_cache": [int(c) for c, t in zip(cached, tiles2) if t], "graph": True}


def run_fp64_peak(args):
    """The roofline denominator on its own: DFMA chains on every SM for about 1.2 s, with the
    SM clocks and throttle reasons sampled while it runs."""
    import torch
    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    mhc.mhc_fp64_peak(20000)                    # warm-up
    torch.cuda.synchronize()
    iters = 1_250_000
    t0 = time.perf_counter()
    with Clocks(local) as clk:
        flops = mhc.mhc_fp64_peak(iters)
    secs = time.perf_counter() - t0
    c = clk.summary()
    nominal = NOMINAL_FP64_TFLOPS * (c["sm_mhz"] / 2070.0 if c.get("sm_mhz") else 1.0)
    print(json.dumps({"metric": "FP64 DFMA peak", "value": flops / 1e12, "unit": "TFLOP/s",
                      "seconds": secs, "dfma_per_s": flops / 2, "clocks": c,
                      "nominal_at_median_clock": nominal,
                      "kernel": "8 independent DFMA chains per thread, 2 x 256 threads per SM"}), flush=True)


def main():
    args = parse()
    if args.fp64_peak:
        run_fp64_peak(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
