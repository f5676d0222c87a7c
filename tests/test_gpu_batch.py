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
