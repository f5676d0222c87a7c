"""Batched persistent launch (mhc_batch_create / mhc_batch_correlator) against the oracle
and against one mhc_correlator call per correlator: |C_b - C_ref| <= 1e-11 * sum |terms|."""
import numpy as np
import pytest
import torch

import oracle
from paper_1411_3691_gb300 import workloads as wl

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


def test_full_batch_64_correlators(M):
    """The 64-correlator batch of the benchmark, in its launch configuration (autotuned tile,
    per-class persistent kernels, CUDA graph).  Correlators of at most 5e6 pairs and n_f <= 9:
    C against the oracle.  Every correlator: C against one mhc_correlator call of the same
    plan, within 1e-10 of a scale sum |w w prod det| that the oracle estimates from 2000
    seeded pairs (exact for the small ones); and 200 seeded pairs through the per-pair probe
    against the oracle's determinants."""
    items = wl.batch(64)
    plans = [M.Plan.from_workload(w) for w in items]
    S = [[torch.from_numpy(s).cuda() for s in w.S] for w in items]
    batch = M.mhc_batch_create([p.handle for p in plans])
    outs = [torch.empty(2, dtype=torch.float64, device="cuda") for _ in items]
    M.mhc_batch_correlator(batch, S, outs)
    torch.cuda.synchronize()
    got = [complex(*o.cpu().numpy()) for o in outs]
    rng = np.random.default_rng(64)
    n_oracle = 0
    for k, w in enumerate(items):
        plain = complex(*plans[k].correlator(S[k]).cpu().numpy())
        ns, nk = len(w.w_src), len(w.w_snk)
        if w.pairs <= 5_000_000 and max(w.n_f) <= 9:
            ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk,
                                           threads=16)
            assert abs(got[k] - ref) <= 1e-11 * scale, (k, w.n_f, got[k], ref)
            n_oracle += 1
        else:
            ii = rng.integers(0, ns, 2000)
            jj = rng.integers(0, nk, 2000)
            d = oracle.pair_dets(w.S, w.n_f, w.labels_src, w.labels_snk, ii, jj)
            terms = np.abs(w.w_src[ii] * w.w_snk[jj] * np.prod(d, axis=1))
            scale = float(np.mean(terms)) * w.pairs
        assert abs(got[k] - plain) <= 1e-10 * scale, (k, w.n_f, got[k], plain)
        ii = rng.integers(0, ns, 200)
        jj = rng.integers(0, nk, 200)
        gd = plans[k].pair_dets(S[k], torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()).cpu().numpy()
        rd = oracle.pair_dets(w.S, w.n_f, w.labels_src, w.labels_snk, ii, jj)
        for f, n in enumerate(w.n_f):
            err = np.abs(gd[:, f] - rd[:, f])
            assert np.all(err <= 1e-9 * np.abs(rd[:, f]) + 1e-300), (k, f, float(np.max(err / np.abs(rd[:, f]))))
        M.mhc_get_status(plans[k].handle)
    assert n_oracle >= 8
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
