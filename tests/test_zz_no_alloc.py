"""The allocation-free forward entry point (mhc_correlator_noalloc) against the ordinary
one (mhc_correlator), through the C ABI.

Some callers cannot let the library allocate device memory during a call (their memory
is reserved by their own pool allocator, or an allocation would stall a latency-critical
loop); for them the library keeps the forward kernel's scratch in a fixed array.  This
file runs last so that a failure here leaves every other test already run.
"""
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


def _case(name):
    if name == "he4":
        w = wl.helium4(scale=8 / 256)
        w.labels_snk, w.w_snk = w.labels_snk[:1000], w.w_snk[:1000]
        return w
    # n > 6 and two-row families: block factors by lane groups, rank-2 solves
    return wl.make_workload("tworow", [12, 10], [60, 48], [9, 7, 5], [8, 6, 7, 5, 30], seed=23,
                            two_row_frac=0.5)


@pytest.mark.parametrize("name", ["he4", "two_rows_n12"])
def test_noalloc_matches_correlator_twice(M, name):
    w = _case(name)
    plan = M.Plan.from_workload(w)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    ref = plan.correlator(S).cpu().numpy()            # ordinary entry point (uploads the plan)
    _, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):                                # two calls in a row share the scratch
        out.fill_(float("nan"))
        M.mhc_correlator_noalloc(plan.handle, S, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(complex(*got) - complex(*ref)) <= 1e-11 * scale, (got, ref)
    M.mhc_get_status(plan.handle)
    plan.close()


def test_noalloc_rejects_oversized_plan(M):
    # single-term families of random triples: families x ceil(4096 / 128) > 65536 work items
    w = wl.make_workload("big", [3], [300], [1] * 4000, [1] * 4096, seed=3)
    plan = M.Plan.from_workload(w)
    assert plan.stats()["families"] * 32 > 65536
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MHCError) as e:
        M.mhc_correlator_noalloc(plan.handle, S, out)
    assert e.value.status == M.MHC_EINVAL
    assert "work items" in str(e.value)
    plan.close()
