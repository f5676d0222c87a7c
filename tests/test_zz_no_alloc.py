"""The allocation-free forward entry point (mhc_correlator_noalloc) against the ordinary
one (mhc_correlator), through the C ABI.

Some callers cannot let the library allocate device memory during a call: a process whose
device memory is reserved up front by its own pool allocator (a cudaMalloc could fail or
fragment the pool), or a latency-critical loop where an allocation would stall the device.
For them the library keeps the forward kernel's per-work-item scratch in a fixed array in
its own device memory.  The two entry points run the same kernels in the same fixed order,
so their results agree bitwise.  This file runs last so that a failure here leaves every
other test already run.
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
    if name == "small":
        return wl.deuteron(scale=4 / 64)
    # n > 6 and two-row families: block factors by lane groups, rank-2 solves
    return wl.make_workload("tworow", [12, 10], [60, 48], [9, 7, 5], [8, 6, 7, 5, 30], seed=23,
                            two_row_frac=0.5)


def _noalloc(M, plan, S, out):
    out.fill_(float("nan"))
    M.mhc_correlator_noalloc(plan.handle, S, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


@pytest.mark.parametrize("name", ["he4", "two_rows_n12"])
def test_noalloc_matches_correlator_twice(M, name):
    w = _case(name)
    plan = M.Plan.from_workload(w)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    ref = plan.correlator(S).cpu().numpy()            # ordinary entry point (uploads the plan)
    C, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(complex(*ref) - C) <= 1e-11 * scale
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):                                # two calls in a row share the scratch
        got = _noalloc(M, plan, S, out)
        assert got.tobytes() == ref.tobytes(), (got, ref)
    M.mhc_get_status(plan.handle)
    plan.close()


def test_noalloc_allocates_nothing(M):
    """Free device memory is the same before and after a call (after the first call on the
    device has looked up the scratch's address)."""
    w = _case("he4")
    plan = M.Plan.from_workload(w)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    plan.correlator(S)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    _noalloc(M, plan, S, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    M.mhc_correlator_noalloc(plan.handle, S, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    M.mhc_get_status(plan.handle)
    plan.close()


def test_noalloc_plans_in_turn(M):
    """Plan A (more work items), then plan B, then A again through the shared scratch: each
    result bitwise equal to the plan's mhc_correlator call (no slot of an earlier, larger
    plan leaks into a later call)."""
    wa, wb = _case("he4"), _case("small")
    pa, pb = M.Plan.from_workload(wa), M.Plan.from_workload(wb)
    Sa = [torch.from_numpy(s).cuda() for s in wa.S]
    Sb = [torch.from_numpy(s).cuda() for s in wb.S]
    ra, rb = pa.correlator(Sa).cpu().numpy(), pb.correlator(Sb).cpu().numpy()
    assert pa.stats()["families"] * ((len(wa.w_snk) + 127) // 128) > \
        pb.stats()["families"] * ((len(wb.w_snk) + 127) // 128)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for plan, S, ref in ((pa, Sa, ra), (pb, Sb, rb), (pa, Sa, ra)):
        assert _noalloc(M, plan, S, out).tobytes() == ref.tobytes()
    for p in (pa, pb):
        M.mhc_get_status(p.handle)
        p.close()


def test_noalloc_rejects_plan_not_on_device(M):
    """A plan whose tables were never uploaded to the current device is rejected (the
    entry point does not upload, since uploading allocates)."""
    w = _case("small")
    plan = M.Plan.from_workload(w)
    S = [torch.from_numpy(s).cuda() for s in w.S]
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MHCError) as e:
        M.mhc_correlator_noalloc(plan.handle, S, out)
    assert e.value.status == M.MHC_EINVAL
    assert "not on the current device" in str(e.value)
    plan.close()


def test_noalloc_rejects_oversized_plan(M):
    # single-term families of random triples: families x ceil(4096 / 128) > 65536 work items
    w = wl.make_workload("big", [3], [300], [1] * 4000, [1] * 4096, seed=3)
    plan = M.Plan.from_workload(w)
    assert plan.stats()["families"] * 32 > 65536
    S = [torch.from_numpy(s).cuda() for s in w.S]
    plan.correlator(S)                                # uploads the plan
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MHCError) as e:
        M.mhc_correlator_noalloc(plan.handle, S, out)
    assert e.value.status == M.MHC_EINVAL
    assert "work items" in str(e.value)
    M.mhc_get_status(plan.handle)
    plan.close()
