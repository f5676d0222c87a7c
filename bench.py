"""Benchmark: the He-4-like correlator (2 flavours, n_f = 6, L = 48, 4096 x 4096 source x sink
terms in families of 16) evaluated on the GPU through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mhc|reference]

One step = one mhc_correlator call (every step of the hot path: shared-row factorisation,
cached solves, member dot products, refactors, fixed-order reduction) for one propagator
set.  The plan (Sec. 3: graph + dominating set) is built once before timing, as the paper
amortises it over gauge configurations.  Between timed steps L2 is flushed by writing a
256 MiB buffer (outside the timed events).  Under torchrun every rank evaluates its own
independent correlator (its own propagators: another gauge configuration), so the work per
GPU is fixed ("weak" scaling) and no collective is on the data path; rank 0 prints one
JSON line with the whole-job pairs/s over the slowest rank.

--impl reference times the oracle (plain CPU FP64, fresh LU per pair) on the host cores on
a bounded sample of the same workload, with the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
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
# dram__bytes_read.sum + dram__bytes_write.sum per forward launch, from one ncu capture of
# this workload (profiles/fwd_kernel_he4.md); None until captured for the current kernel.
FWD_TRAFFIC_BYTES = 68.89e6  # 68.34 MB read + 0.55 MB write (fwd_kernel<8>, 2.040 ms launch)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mhc", choices=["mhc", "reference"])
    ap.add_argument("--cpu-sample-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-sequential comparison")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-vs-forward comparison")
    ap.add_argument("--workload", default="he4", choices=["he4", "large", "large_noforce", "large_small"],
                    help="he4 (the benchmark line) or the n = 18 nucleus variants; the latter time "
                         "the forward only (no adjoint, batch or CPU baseline)")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="only measure the FP64 (DFMA) peak: >= 1 s of independent chains on every SM, "
                         "SM clocks sampled meanwhile")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int, scale: float = 1.0, name: str = "he4"):
    """The rank's own replica on its own propagators (seed).  he4: the He-4-like workload
    of the benchmark line; large, large_noforce, large_small: the 32768 x 32768 n = 18
    nucleus (10 % two-row families, 1 % forced near-singular members), the same without
    the forced members, and a 1/8-scale copy of the first (for profiler captures)."""
    from paper_1411_3691_gb300 import workloads as wl
    if name == "he4":
        return wl.helium4(scale=scale, seed=1000 + 17 * rank)
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


def cpu_oracle_rate(w, seconds: float):
    """Oracle pairs/s on the host cores over a bounded sample of source terms (all sinks)."""
    import oracle
    threads = cores()
    n_snk = len(w.w_snk)
    # calibrate on a small block, then size the sample for about `seconds`
    t0 = time.perf_counter()
    oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=threads,
                      src_range=(0, min(len(w.w_src), 4 * threads)))
    dt = max(time.perf_counter() - t0, 1e-3)
    rate0 = min(len(w.w_src), 4 * threads) * n_snk / dt
    n_src = int(min(len(w.w_src), max(threads, rate0 * seconds / n_snk)))
    t0 = time.perf_counter()
    C, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk,
                                 threads=threads, src_range=(0, n_src))
    dt = time.perf_counter() - t0
    return {"value": n_src * n_snk / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n_src} of {len(w.w_src)} source terms x all {n_snk} sinks "
                      f"({n_src * n_snk} pairs, fresh partial-pivot LU per pair per flavour), "
                      f"{dt:.2f} s on {threads} threads"}


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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(0)
    steps = []
    per = max(args.cpu_sample_seconds / max(args.steps + args.warmup, 1), 0.5)
    for s in range(args.warmup + args.steps):
        r = cpu_oracle_rate(w, per)
        if s >= args.warmup:
            steps.append(r)
    value = sum(r["value"] for r in steps) / len(steps)
    cb = dict(steps[-1])
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "flavours": 2, "n_f": 6, "L": 48, "n_src": len(w.w_src),
                       "n_snk": len(w.w_snk)},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    w = workload(rank, name=args.workload)
    if args.workload != "he4":  # the nucleus variants time the forward only
        args.no_adjoint = args.no_batch = args.no_cpu_baseline = True
    plan = mhc.Plan.from_workload(w)
    st = plan.stats()
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # FP64 peak on this GPU (DFMA chains on every SM), taken before the warm-up so that the
    # timed steps follow the warm-up directly
    peak_flops = mhc.mhc_fp64_peak(250000)

    # warm-up (first call uploads the plan)
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
    pairs = len(w.w_src) * len(w.w_snk)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, pairs, ms_per_step)

    # roofline of the forward kernel (FP64 ALU bound): algorithmic flops per launch over the
    # step's device time, against the FP64 peak measured above
    # refactors are not counted (they run partly as shared factorisations of a group of
    # pairs, below a fresh LU each): the FLOP figure is a lower bound of the work done
    refactor_pairs = (st["refactor_parent"] + st["refactor_child"]) / max(args.steps, 1)
    flops = st["flops_per_call"]
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        for d, h in zip(dS, hS):
            d.copy_(h, non_blocking=True)
        plan.correlator(dS, out=out)
        hout.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, pg, "cuda")
    h2d = sum(h.numel() * h.element_size() for h in hS)

    adjoint = None if args.no_adjoint else time_adjoint(mhc, plan, S, flush, stream, ms_per_step, pairs)
    batched = None if (args.no_batch or rank != 0) else time_batch(mhc, flush, stream)

    if batched:
        batched["frac_of_fp64_peak"] = batched["tflops"] / (peak_flops / 1e12)
    if adjoint:
        adjoint["frac_of_fp64_peak"] = adjoint["tflops"] / (peak_flops / 1e12)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "flavours": len(w.n_f), "n_f": w.n_f[0], "L": w.L_f[0],
                       "n_src": len(w.w_src),
                       "n_snk": len(w.w_snk), "pairs_per_gpu": pairs, "families": st["families"],
                       "parallelism": f"{world} independent correlators (one per GPU)",
                       "l2": "flushed between timed steps (256 MiB write outside the events)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": FWD_TRAFFIC_BYTES if args.workload == "he4" else None,
                         "peak_source": "FP64 DFMA chains on all SMs, measured in this run "
                                        f"(nominal {NOMINAL_FP64_TFLOPS:.3f} from unit counts and clocks)",
                         "flops_per_step": flops},
            "e2e": {"value": whole_job_rate(world, pairs, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 16},
            "gpu_launches": forward_launches(plan, w, st) * args.steps,
            "clocks": clocks,
            "refactors_per_step": refactor_pairs,
            "adjoint": adjoint,
            "batched": batched,
            "C": [float(out[0].item()), float(out[1].item())],
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_rate(w, args.cpu_sample_seconds)
        print(json.dumps(line), flush=True)
    plan.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def time_adjoint(mhc, plan, S, flush, stream, fwd_ms, pairs, steps=5):
    """Backward (dS_f, dw_src, dw_snk for L = Re C) of the same workload, CUDA events."""
    import torch
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
    bflops = plan.stats()["backward_flops_per_call"]
    return {"ms_per_step": ms, "ratio_vs_forward": ms / fwd_ms, "pairs_per_s": pairs / (ms * 1e-3),
            "tflops": bflops / (ms * 1e-3) / 1e12, "flops_per_step": bflops,
            "outputs": "dS_f (2 x 48 x 48 complex), dw_src [4096], dw_snk [4096]; L = Re C",
            # block factors and B^-1 (two-sided plans), the adjoint kernel, one dS finalize per
            # flavour, the two weight finalizes
            "gpu_launches_per_step": (3 if plan.stats()["two_sided_blocks"] > 0 else 1) + len(S) + 2}


def time_batch(mhc, flush, stream, count=64, reps=3):
    """64 independent correlators of mixed n_f in one persistent launch under a CUDA graph,
    against 64 sequential mhc_correlator calls on the same plans and propagators."""
    import torch
    from paper_1411_3691_gb300 import workloads as wl
    items = wl.batch(count)
    plans = [mhc.Plan.from_workload(w) for w in items]
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    pairs = sum(w.pairs for w in items)
    batch = mhc.mhc_batch_create([p.handle for p in plans])
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
            "tflops": flops / (batch_ms * 1e-3) / 1e12,
            "sequential_ms": seq_ms, "sequential_pairs_per_s": pairs / (seq_ms * 1e-3),
            "speedup_vs_sequential": seq_ms / batch_ms, "tile": T, "work_items": n_items,
            "graph": True}


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
