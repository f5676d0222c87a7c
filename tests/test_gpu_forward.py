"""GPU parity of the forward correlator and the per-pair probe against the oracle.

Tolerances (from the arithmetic; stated per test):
  * C: |C_gpu - C_oracle| <= 1e-11 * sum_ij |w_i w_j prod det|.
  * per pair and flavour: |d_gpu - d_ref| <= 1e-12 |d_ref|, or, for an ill-conditioned
    block, <= 4 n u kappa_inf(G) |d_ref| with d_ref in double-double and u = 2^-53.
"""
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


def dev_S(w):
    return [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in w.S]


def gpu_C(M, w, opts=None, plan=None, S=None):
    plan = plan or M.Plan.from_workload(w, opts)
    S = S or dev_S(w)
    out = plan.correlator(S)
    torch.cuda.synchronize()
    return complex(out[0].item(), out[1].item()), plan, S


def small_cases():
    he = wl.helium4(scale=6 / 256)
    he.labels_snk, he.w_snk = he.labels_snk[:300], he.w_snk[:300]          # ragged sink tile
    lg = wl.large_nucleus(scale=4 / 1024)
    lg.labels_snk, lg.w_snk = lg.labels_snk[:70], lg.w_snk[:70]
    rep = wl.make_workload("repeat", [4, 3], [10, 9], [6, 3, 5], [4, 4, 3], seed=44)
    rng = np.random.default_rng(3)
    for t in rng.choice(rep.labels_src.shape[0], 4, replace=False):
        rep.labels_src[t, 1] = rep.labels_src[t, 0]                         # repeated label: det 0
    diag = wl.make_workload("diag", [3, 3], [8, 8], [4, 4, 4], [6, 6], seed=45)
    d = [np.diag(np.diag(s)) for s in diag.S]
    diag.S = [np.ascontiguousarray(x) for x in d]
    perm_snk = np.concatenate([diag.labels_src[:, :3][:, ::-1], diag.labels_src[:, 3:]], axis=1)
    diag.labels_snk = np.concatenate([diag.labels_snk, perm_snk]).astype(np.int32)
    diag.w_snk = np.concatenate([diag.w_snk, np.ones(perm_snk.shape[0])])
    return {
        "deuteron_full": wl.deuteron(),
        "he4_ragged": he,
        "large_rank2_forced": lg,
        "mixed_nf0": wl.make_workload("mixed", [3, 0, 7], [24, 5, 30], [5, 1, 3, 8, 2], [7, 9, 3], seed=9,
                                      two_row_frac=0.3),
        "n9_n12": wl.make_workload("n9n12", [9, 12], [36, 48], [5, 7, 3], [40, 33], seed=10, two_row_frac=0.2),
        "n1": wl.make_workload("n1", [1, 1], [6, 7], [3, 2, 4], [5, 4], seed=11),
        "repeated_labels": rep,
        "diagonal_S": diag,
        "n32": wl.make_workload("n32", [32], [64], [3, 2], [40], seed=12),
        "two_rows_both_sides": wl.make_workload("tworow", [12, 10], [60, 48], [9, 7, 5], [8, 6, 7, 5, 30],
                                                seed=23, two_row_frac=0.5),
        "eight_flavours": wl.make_workload("f8", [2, 3, 1, 4, 2, 3, 1, 2], [12, 16, 8, 20, 12, 16, 8, 12],
                                           [5, 4], [6, 3], seed=51),
        "single_terms": wl.make_workload("one", [3, 2], [10, 8], [1], [1], seed=53),
        # members changing rows of their own: families split and merged by the flop count
        "mixed_rows": wl.make_workload("mr", [12, 18], [60, 96], [9, 12, 7, 16], [5, 6, 4, 20], diag=3.0,
                                       seed=97, mixed_rows=True),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", list(CASES))
def test_forward_matches_oracle(M, name):
    w = CASES[name]
    C, plan, S = gpu_C(M, w)
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (name, C, ref, abs(C - ref) / scale)
    code = M.mhc_get_status_code(plan.handle)
    assert code == M.MHC_OK
    plan.close()


def test_forward_deterministic(M):
    w = CASES["large_rank2_forced"]
    plan = M.Plan.from_workload(w)
    S = dev_S(w)
    a = plan.correlator(S).cpu().numpy()
    b = plan.correlator(S).cpu().numpy()
    assert a.tobytes() == b.tobytes()


def test_weights_override(M):
    w = CASES["he4_ragged"]
    plan = M.Plan.from_workload(w)
    S = dev_S(w)
    rng = np.random.default_rng(5)
    ws, wk = rng.normal(size=w.w_src.shape), rng.normal(size=w.w_snk.shape)
    out = plan.correlator(S, torch.from_numpy(ws).cuda(), torch.from_numpy(wk).cuda())
    C = complex(*out.cpu().numpy())
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, ws, w.labels_snk, wk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale


@pytest.mark.parametrize("row_difference", [0, 1])
def test_pair_dets(M, row_difference):
    """Every pair of the forced workload through the probe against the oracle.  The forced
    near-singular members (a changed row set to the near-twin of a shared row) left the
    lemma update for every sink: by a refactor (default), or with row_difference = 1 by the
    row-difference update (one- and two-row families) unless its own guard failed too."""
    w = CASES["large_rank2_forced"]
    opts = M.default_opts()
    opts.row_difference = row_difference
    plan = M.Plan.from_workload(w, opts)
    S = dev_S(w)
    ii, jj = np.meshgrid(np.arange(len(w.w_src)), np.arange(len(w.w_snk)), indexing="ij")
    path, n_ill = check_pairs(M, w, plan, S, ii.ravel(), jj.ravel())
    forced = w.meta["src"]["forced"]
    assert len(forced) > 0
    P = path.reshape(len(w.w_src), len(w.w_snk))
    for t, f in forced:
        assert np.all(((P[t] >> f) | (P[t] >> (8 + f))) & 1), (t, f)
    if row_difference:
        assert np.any(P >> 8)  # some forced members were one-row members
    else:
        assert not np.any(P >> 8)


@pytest.mark.parametrize("row_difference", [0, 1])
def test_refactor_counters(M, row_difference):
    w = CASES["large_rank2_forced"]
    opts = M.default_opts()
    opts.row_difference = row_difference
    C, plan, S = gpu_C(M, w, opts)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    st = plan.stats()
    forced = w.meta["src"]["forced"]
    assert st["refactor_child"] + st["row_difference"] >= len(forced) * len(w.w_snk)
    if row_difference:
        assert st["row_difference"] > 0
    else:
        assert st["row_difference"] == 0
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)


def test_nonfinite_status(M):
    w = wl.deuteron(scale=2 / 64)
    S = dev_S(w)
    S[0][w.labels_src[0, 0], :] = float("nan")
    C, plan, S = gpu_C(M, w, S=S)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_ENONFINITE


def test_full_helium4(M):
    """The 4096 x 4096 He-4-like workload at full size against the threaded oracle."""
    w = wl.helium4()
    C, plan, S = gpu_C(M, w)
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=16)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK


_LARGE = {}


def _large_and_reference():
    """The large nucleus, and the oracle's C over 32 random source families x all sinks
    (computed once for the parametrised test below)."""
    if not _LARGE:
        w = wl.large_nucleus()
        ws, keep = family_mask(w, 32, seed=33)
        _LARGE.update(w=w, ws=ws, keep=keep, ref=oracle_subset(w, keep))
    return _LARGE


@pytest.mark.parametrize("row_difference", [0, 1])
def test_full_large_nucleus_sampled(M, row_difference):
    """32768 x 32768, n = 18, in the plan and launch configuration the benchmark times:
    10^5 seeded pairs through the probe against the oracle (1e-12 relative, or the
    conditioning bound for the forced near-singular members, which must have left the
    lemma update: refactored, or with row_difference = 1 the one-row ones by the
    row-difference update), and C of the full plan with the source weights of all but 32
    random families set to zero against the oracle's sum over those families x all 32768
    sinks."""
    L = _large_and_reference()
    w = L["w"]
    opts = M.default_opts()
    opts.row_difference = row_difference
    plan = M.Plan.from_workload(w, opts)
    S = dev_S(w)
    rng = np.random.default_rng(31)
    ii = rng.integers(0, len(w.w_src), 100000)
    jj = rng.integers(0, len(w.w_snk), 100000)
    path, n_ill = check_pairs(M, w, plan, S, ii, jj)
    forced = set(map(tuple, w.meta["src"]["forced"]))
    for p in range(len(ii)):
        for f in range(2):
            if (int(ii[p]), f) in forced:
                assert ((path[p] >> f) | (path[p] >> (8 + f))) & 1, (ii[p], jj[p], f)
    ws, keep = L["ws"], L["keep"]
    assert len(keep) == 32 * 32
    out = plan.correlator(S, torch.from_numpy(ws).cuda())
    C = complex(*out.cpu().numpy())
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    st = plan.stats()
    if row_difference:
        assert st["row_difference"] > 0                # the forced members' row differences
    else:
        assert st["refactor_child"] > 0 and st["row_difference"] == 0
    ref, scale = L["ref"]
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)
    plan.close()


def test_families_of_64(M):
    """The largest family the planner forms (opts.max_family = 64) on both sides."""
    w = wl.make_workload("fam64", [4, 4], [40, 40], [64, 10], [64, 5], seed=52)
    opts = M.default_opts()
    opts.max_family = 64
    C, plan, S = gpu_C(M, w, opts)
    assert plan.stats()["families"] == 2
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK


def test_complex_weights(M):
    """mhc_correlator_cw against the oracle through bilinearity: four real-weight oracle
    sums combined as C = C(a, c) - C(b, d) + i (C(a, d) + C(b, c))."""
    w = CASES["two_rows_both_sides"]
    plan = M.Plan.from_workload(w)
    S = dev_S(w)
    rng = np.random.default_rng(17)
    a, b = rng.normal(size=len(w.w_src)), rng.normal(size=len(w.w_src))
    c, d = rng.normal(size=len(w.w_snk)), rng.normal(size=len(w.w_snk))
    ws = torch.from_numpy(a + 1j * b).cuda()
    wk = torch.from_numpy(c + 1j * d).cuda()
    out = M.mhc_correlator_cw(plan.handle, S, ws, wk)
    got = complex(*out.cpu().numpy())
    parts, scale = {}, 0.0
    for kx, x in (("a", a), ("b", b)):
        for ky, y in (("c", c), ("d", d)):
            parts[kx + ky], sc = oracle.correlator(w.S, w.n_f, w.labels_src, x, w.labels_snk, y, threads=8)
            scale += sc
    ref = parts["ac"] - parts["bd"] + 1j * (parts["ad"] + parts["bc"])
    assert abs(got - ref) <= 1e-11 * scale, (got, ref)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK


@pytest.mark.parametrize("one_sided", [0, 1])
def test_three_row_families(M, one_sided):
    """Rank-3 families (opts.rank3, n_f >= 14): C against the oracle, with sink families
    (the rank-3 blocks take the one-sided path) and without, and every pair's determinants
    through the probe."""
    w = wl.make_workload("r3", [14, 14], [56, 56], [6, 5, 4, 7], [5, 6, 4, 20], seed=67, two_row_frac=0.2,
                         three_row_frac=0.5)
    opts = M.default_opts()
    opts.rank3 = 1
    opts.one_sided = one_sided
    C, plan, S = gpu_C(M, w, opts)
    assert plan.stats()["rank3_family_flavours"] > 0
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    ii, jj = np.meshgrid(np.arange(len(w.w_src)), np.arange(len(w.w_snk)), indexing="ij")
    check_pairs(M, w, plan, S, ii.ravel(), jj.ravel())


@pytest.mark.parametrize("three_row_frac", [0.0, 0.3])
def test_forced_members_in_multi_row_families(M, three_row_frac):
    """Members near-singular against families with two (three) changed rows: whole warps of
    their pairs fail the guard and are refactored as groups that share the member's rows and
    the sink family's shared columns (Sec. 2.1's fallback to a fresh factorisation); C against
    the oracle, and the refactors counted."""
    w = wl.make_workload("forced_multirow", [14, 12], [64, 56], [32, 32, 32], [32, 32, 32, 7], seed=71,
                         two_row_frac=0.5, three_row_frac=three_row_frac, forced_frac=0.2, twins=8)
    info = w.meta["src"]
    forced = info["forced"]
    assert any(len(info["rows"][info["family_of"][t]][f]) >= 2 for t, f in forced)
    opts = M.default_opts()
    opts.rank3 = 1 if three_row_frac else 0
    C, plan, S = gpu_C(M, w, opts)
    st = plan.stats()
    assert st["rank2_family_flavours"] > 0
    if three_row_frac:
        assert st["rank3_family_flavours"] > 0
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    st = plan.stats()
    assert st["refactor_child"] + st["row_difference"] >= len(forced) * len(w.w_snk) // 2
    plan.close()


def test_forced_members_against_two_column_sink_families(M):
    """Near-singular members (a row set to the near-twin of a shared row) against sink
    families that change two columns: the pairs of one member and one such sink family agree
    in all but their last two columns and are refactored together (the shared elimination of
    the first n - 2 columns once, then each sink's two columns and the last 2 x 2 step).  C
    against the oracle, the refactors counted, and the refactor flops below a fresh LU per
    refactored pair and flavour."""
    a = wl.make_workload("f2c", [18, 12], [96, 60], [32, 32, 32], [32, 32, 32, 7], diag=3.0, seed=81,
                         two_row_frac=0.0, forced_frac=0.2, twins=8)
    b = wl.make_workload("f2c", [18, 12], [96, 60], [32, 32, 32], [32, 32, 32, 7], diag=3.0, seed=81,
                         two_row_frac=1.0, forced_frac=0.2, twins=8)
    assert all(np.array_equal(x, y) for x, y in zip(a.S, b.S))
    w = wl.Workload("f2c", a.n_f, a.S, a.labels_src, a.w_src, b.labels_snk, b.w_snk, a.meta)
    plan = M.Plan.from_workload(w)
    sinks = plan.sinks()
    assert sinks["two_sided"].sum() >= 3
    C, plan, S = gpu_C(M, w, plan=plan)
    st = plan.stats()
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    st = plan.stats()
    forced = w.meta["src"]["forced"]
    assert len(forced) > 0
    n_ref = st["refactor_parent"] + st["refactor_child"]
    assert n_ref >= len(forced) * len(w.w_snk) // 2
    fresh18 = 18 * 19 / 2 + 6 * 17 + 3 * 18 * 17 + 8 * 17 * 18 * 35 / 6 + 6 * 17
    assert 0 < st["refactor_flops"] < 0.5 * n_ref * fresh18
    plan.close()


def _rank_k_workload(k):
    """Source families that change k rows of their first flavour (rank k needs n_f >= 4k + 2:
    n_f = 18 for k = 4, 22 for k = 5), two-row families in the other flavour."""
    if k == 4:
        return wl.make_workload("r4", [18, 12], [96, 60], [5, 4, 4, 3, 6], [5, 6, 4, 20], diag=3.0, seed=93,
                                two_row_frac=0.3, more_rows=[{4: 0.7}, {}])
    return wl.make_workload("r5", [22, 10], [110, 40], [5, 4, 3, 6], [4, 5, 3, 12], diag=3.0, seed=94,
                            more_rows=[{4: 0.3, 5: 0.6}, {}])


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("one_sided", [0, 1])
def test_rank_k_families(M, k, one_sided):
    """The general rank-k update (k null vectors of the shared rows, a k x k determinant per
    member by a small LU), k = 4 and 5: C against the oracle with and without sink families,
    and every pair's determinants through the probe."""
    w = _rank_k_workload(k)
    opts = M.default_opts()
    opts.max_rank = k
    opts.one_sided = one_sided
    C, plan, S = gpu_C(M, w, opts)
    assert plan.stats()["rank4plus_family_flavours"] > 0
    assert int(plan.families()["rank"].max()) == k
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    ii, jj = np.meshgrid(np.arange(len(w.w_src)), np.arange(len(w.w_snk)), indexing="ij")
    check_pairs(M, w, plan, S, ii.ravel(), jj.ravel())
    plan.close()


def test_two_row_sources_against_warp_wide_sink_families(M):
    """Two-row source families against one-column sink families of exactly 32 sinks, so
    that each warp's sinks share one sink family: the members' dots with the block's first
    null vector are formed once per warp.  C against the oracle."""
    a = wl.make_workload("r2w", [12, 10], [60, 48], [7, 5, 6, 9], [32, 32, 32], seed=48, two_row_frac=0.7)
    b = wl.make_workload("r2w", [12, 10], [60, 48], [7, 5, 6, 9], [32, 32, 32], seed=48, two_row_frac=0.0)
    assert all(np.array_equal(x, y) for x, y in zip(a.S, b.S))
    w = wl.Workload("r2w", a.n_f, a.S, a.labels_src, a.w_src, b.labels_snk, b.w_snk)
    C, plan, S = gpu_C(M, w)
    assert plan.stats()["rank2_family_flavours"] > 0
    assert np.all(plan.sinks()["two_sided"] == 1)
    ref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=8)
    assert abs(C - ref) <= 1e-11 * scale, (C, ref, abs(C - ref) / scale)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    plan.close()
