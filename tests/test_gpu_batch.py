"""Batched persistent launch (mhc_batch_create / mhc_batch_correlator) against the oracle
and against one mhc_correlator call per correlator: |C_b - C_ref| <= 1e-11 * sum |terms|."""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_3691_gb300 import workloads as wl
from parity_util import check_pairs, family_mask, oracle_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc
    return mhc


def test_batch_matches_oracle_and_plain(M):
    items = [wl.batch_item(b, max_terms=700) for b in range(7)]
    plans = [M.Plan.from_workload(w) for w in items]
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    batch = M.mhc_batch_create([p.handle for p in plans])
    T, n_items = M.mhc_batch_info(batch)
    assert T in (32, 64, 128) and n_items > 0
    outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in items]
    M.mhc_batch_correlator(batch, S, outs)
    torch.cuda.synchronize()
    first = [o.cpu().numpy().copy() for o in outs]
    for k, w in enumerate(items):
        ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
        got = complex(*first[k])
        assert abs(got - ref) <= 1e-11 * scale, (k, w.n_f, got, ref)
        plain = complex(*plans[k].correlator(S[k]).cpu().numpy())
        assert abs(got - plain) <= 1e-11 * scale
    # graph replay: bitwise identical
    for o in outs:
        o.zero_()
    M.mhc_batch_correlator(batch, S, outs)
    torch.cuda.synchronize()
    for k in range(len(items)):
        assert outs[k].cpu().numpy().tobytes() == first[k].tobytes()
    # new propagator pointers: the batch recaptures and stays correct
    S2 = [[s.clone() * 0.5 for s in Sk] for Sk in S]
    M.mhc_batch_correlator(batch, S2, outs)
    torch.cuda.synchronize()
    for k, w in enumerate(items):
        F = len(w.n_f)
        ref = complex(*first[k]) * 0.5 ** sum(w.n_f)
        _, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
        assert abs(complex(*outs[k].cpu().numpy()) - ref) <= 1e-11 * scale * 0.5 ** sum(w.n_f) * 10
    for p in plans:
        M.mhc_get_status(p.handle)
    M.mhc_batch_destroy(batch)


def test_tuning_cache_second_create(M, tmp_path, monkeypatch):
    """A second mhc_batch_create with the same plans takes every class's tile from the
    tuning cache (no timing), chooses the same tiles, and gives bitwise the same results."""
    monkeypatch.setenv("MHC_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    items = [wl.batch_item(b, max_terms=900) for b in range(12)]
    plans = [M.Plan.from_workload(w) for w in items]
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    res = []
    for rep in range(2):
        batch = M.mhc_batch_create([p.handle for p in plans])
        tiles, cached, ms = M.mhc_batch_shape(batch)
        used = [c for c in range(3) if tiles[c]]
        assert len(used) >= 2
        assert all(tiles[c] in (32, 64, 128) for c in used)
        if rep == 0:
            assert all(cached[c] == 0 and max(ms[c]) > 0 for c in used)
        else:
            assert all(cached[c] == 1 for c in used) and tiles == res[0][0]
        outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in items]
        M.mhc_batch_correlator(batch, S, outs)
        torch.cuda.synchronize()
        res.append((tiles, [o.cpu().numpy().tobytes() for o in outs]))
        M.mhc_batch_destroy(batch)
    assert res[0][1] == res[1][1]
    for k, w in enumerate(items[:4]):
        ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
        got = complex(*np.frombuffer(res[1][1][k], dtype=np.float64))
        assert abs(got - ref) <= 1e-11 * scale
    for p in plans:
        M.mhc_get_status(p.handle)
        p.close()


def test_full_batch_64_correlators(M):
    """The 64-correlator batch of the benchmark in its launch configuration (autotuned
    shape, per-class persistent kernels, CUDA graph), every correlator against the oracle
    at |dC| <= 1e-11 sum |w w prod det|:
      * a correlator the oracle evaluates in seconds: its full C;
      * any other: C with the source weights of all but 32 random families set to zero (the
        planner ignores weight values, so the families, work items and launch are those of
        the full plan) against the oracle's sum over those families x all sinks;
    and for every correlator 10^4 seeded pairs through the per-pair probe at 1e-12 relative
    (the conditioning bound where no FP64 method can reach that)."""
    items = wl.batch(64)
    budget = 5e6 * 2 * 9 ** 3          # pairs x sum_f n_f^3 of a full oracle evaluation
    keeps, plans = [], []
    for k, w in enumerate(items):
        if w.pairs * sum(n ** 3 for n in w.n_f) <= budget:
            keeps.append(None)
            ws = w.w_src
        else:
            ws, keep = family_mask(w, 32, seed=640 + k)
            keeps.append(keep)
        plans.append(M.Plan(w.n_f, w.L_f, w.labels_src, ws, w.labels_snk, w.w_snk))
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    batch = M.mhc_batch_create([p.handle for p in plans])
    outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in items]
    M.mhc_batch_correlator(batch, S, outs)
    torch.cuda.synchronize()
    got = [complex(*o.cpu().numpy()) for o in outs]
    rng = np.random.default_rng(64)
    n_full = n_masked = 0
    for k, w in enumerate(items):
        if keeps[k] is None:
            ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk,
                                           threads=16)
            n_full += 1
        else:
            ref, scale = oracle_subset(w, keeps[k])
            n_masked += 1
        assert abs(got[k] - ref) <= 1e-11 * scale, (k, w.n_f, got[k], ref, abs(got[k] - ref) / scale)
        ii = rng.integers(0, len(w.w_src), 10000)
        jj = rng.integers(0, len(w.w_snk), 10000)
        check_pairs(M, w, plans[k], S[k], ii, jj)
        assert M.mhc_get_status_code(plans[k].handle) == M.MHC_OK
    assert n_full >= 30 and n_masked >= 20
    M.mhc_batch_destroy(batch)
    for p in plans:
        p.close()


def test_one_plan_many_configurations(M):
    """One plan given four times with four propagator sets (gauge configurations): every
    entry matches its own mhc_correlator call and the oracle."""
    w = wl.helium4(scale=6 / 256)
    plan = M.Plan.from_workload(w)
    rng = np.random.default_rng(99)
    sets = [[wl.make_S(rng, s.shape[0], 2.0) for s in w.S] for _ in range(4)]
    S = [[torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in Sk] for Sk in sets]
    batch = M.mhc_batch_create([plan.handle] * 4)
    outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in range(4)]
    M.mhc_batch_correlator(batch, S, outs)
    torch.cuda.synchronize()
    got = [complex(*o.cpu().numpy()) for o in outs]
    for k in range(4):
        ref, scale = oracle.correlator(sets[k], w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
        assert abs(got[k] - ref) <= 1e-11 * scale, (k, got[k], ref)
        plain = complex(*plan.correlator(S[k]).cpu().numpy())
        assert abs(got[k] - plain) <= 1e-11 * scale
    assert len({round(g.real, 6) for g in got}) == 4      # four different configurations
    M.mhc_get_status(plan.handle)
    M.mhc_batch_destroy(batch)
