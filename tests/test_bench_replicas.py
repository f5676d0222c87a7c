"""The N > 1 path of the benchmark on CPU: two gloo ranks, each evaluating its own replica.

Under torchrun every rank evaluates an independent correlator (its own propagators, as
another gauge configuration would give), no collective touches the data path, and the job's
step time is the slowest rank's.  Here the ranks evaluate their replicas with the oracle (the
host stands in for the GPU), then take the same max-over-ranks and whole-job rate that the
benchmark takes.
"""
import json
import os
import socket
import sys
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SCALE = 4 / 256          # 4 families x 16 members on each side: 64 x 64 pairs per replica


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = bench.workload(rank, "he4", scale=SCALE)
    t0 = time.perf_counter()
    C, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
    ms = (time.perf_counter() - t0) * 1e3
    if rank == 1:
        ms += 50.0                       # rank 1 is the slow one
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    pairs = len(w.w_src) * len(w.w_snk)
    rec = {"rank": rank, "ms": ms, "job_ms": job_ms, "pairs": pairs, "C": [C.real, C.imag],
           "S0": float(np.abs(w.S[0]).sum()), "rate": bench.whole_job_rate(world, pairs, job_ms)}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(rec, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    recs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # every rank sees the slowest rank's time
    slowest = max(r["ms"] for r in recs)
    assert all(r["job_ms"] == slowest for r in recs)
    assert slowest >= 50.0
    # the replicas are independent problems of the same shape (weak scaling)
    assert recs[0]["pairs"] == recs[1]["pairs"] == 64 * 64
    assert recs[0]["S0"] != recs[1]["S0"]
    assert recs[0]["C"] != recs[1]["C"]
    # whole-job rate: all ranks' pairs over the slowest rank's step
    for r in recs:
        assert r["rate"] == pytest.approx(2 * 64 * 64 / (slowest * 1e-3), rel=1e-12)


def test_single_rank_defaults():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(1, 4096 * 4096, 2.0) == pytest.approx(4096 * 4096 / 2e-3)


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    """Under torchrun only rank 0 runs and prints the reference arm; the others return."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(monkeypatch, capsys):
    """The reference arm (the oracle on the host cores) prints one JSON line with the
    contract's keys, on the benchmark's metric and workload."""
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                                      "--cpu-pairs", "2000", "--scale", str(4 / 1024)])
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pairs/s"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == "large_n18_L96_32768x32768"
    assert d["config"]["n_f"] == 18 and d["config"]["L"] == 96


def test_forward_launch_count():
    """The bench's launch count: block factors (two launches when a flavour has n > 6),
    one forward launch per group of families with the same flavour ranks (at most four),
    and the reduction; built from the plan on the host."""
    from paper_1411_3691_gb300 import mhc
    from paper_1411_3691_gb300 import workloads as wl
    he = bench.workload(0, "he4", scale=SCALE)
    plan = mhc.Plan.from_workload(he)
    assert bench.forward_launches(plan, he, plan.stats()) == 3
    plan.close()
    w = wl.make_workload("tworow", [12, 10], [60, 48], [9, 7, 5, 6, 8, 4], [8, 6, 7, 5, 30], seed=23,
                         two_row_frac=0.5)
    plan = mhc.Plan.from_workload(w)
    ranks = plan.families()["rank"]
    groups = {tuple(int(r) for r in row) for row in ranks}
    assert len(groups) >= 2
    assert bench.forward_launches(plan, w, plan.stats()) == 2 + min(len(groups), 4) + 1
    plan.close()
