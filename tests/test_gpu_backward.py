"""GPU parity of the adjoint (mhc_correlator_backward) against the oracle's Jacobi-formula
gradient and against central differences of the GPU forward.

Conventions: with g = dL/dRe C + i dL/dIm C, the library returns dS_f = g conj(dC/dS_f) and
dw = Re(conj(g) dC/dw) (PyTorch's gradient of a real loss).  Tolerances:
  * vs the oracle, per entry: |d_gpu - d_ref| <= 1e-10 * scale_entry + 1e-12 * max scale,
    scale_entry = sum of |contributions| to that entry (the oracle returns it);
  * central differences with h = 1e-6: C is affine in every single S entry (each entry
    appears at most once in a distinct-label G) and linear in every weight, so the
    difference quotient is exact up to rounding: |g - g_FD| <= 1e-9 * sum_ij |w w prod det|.
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


def dev_S(w):
    return [torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in w.S]


def gpu_backward(M, plan, S, g):
    g_out = torch.tensor(g, dtype=torch.float64, device="cuda")
    dS = [torch.empty_like(s) for s in S]
    dws = torch.empty(plan.n_src, dtype=torch.float64, device="cuda")
    dwk = torch.empty(plan.n_snk, dtype=torch.float64, device="cuda")
    M.mhc_correlator_backward(plan.handle, S, g_out, None, None, dS, dws, dwk)
    torch.cuda.synchronize()
    return [d.cpu().numpy() for d in dS], dws.cpu().numpy(), dwk.cpu().numpy()


def check_vs_oracle(M, w, opts=None, threads=8):
    if opts is None:
        opts = M.default_opts()
        opts.rank2 = 1 if w.name in ("tc", "r2", "mr") else 0
    plan = M.Plan.from_workload(w, opts)
    if w.name == "r2":
        assert plan.stats()["rank2_family_flavours"] > 0
    S = dev_S(w)
    ref = oracle.correlator_grad(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=threads)
    worst = 0.0
    for g in ((1.0, 0.0), (0.0, 1.0), (0.6, -0.8)):
        gc = complex(*g)
        dS, dws, dwk = gpu_backward(M, plan, S, g)
        for f in range(len(w.S)):
            if w.n_f[f] == 0:
                continue
            want = gc * np.conj(ref["dS"][f])
            sc = ref["dS_scale"][f]
            tol = 1e-10 * sc + 1e-12 * sc.max()
            err = np.abs(dS[f] - want)
            assert np.all(err <= tol), (f, g, float(np.max(err / (sc + 1e-300))))
            worst = max(worst, float(np.max(err / np.maximum(tol, 1e-300))))
        for got, D, sc in ((dws, ref["dw_src"], ref["dw_src_scale"]), (dwk, ref["dw_snk"], ref["dw_snk_scale"])):
            want = (np.conj(gc) * D).real
            tol = 1e-10 * sc + 1e-12 * sc.max()
            assert np.all(np.abs(got - want) <= tol)
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    plan.close()
    return worst


CASES = {
    "deuteron": lambda: wl.deuteron(scale=6 / 64),
    "he4_small": lambda: _cut(wl.helium4(scale=3 / 256), 150),
    "mixed_nf0": lambda: wl.make_workload("mixed", [3, 0, 7], [24, 5, 30], [5, 1, 3, 8, 2], [7, 9, 3], seed=9),
    "n1": lambda: wl.make_workload("n1", [1, 1], [6, 7], [3, 2, 4], [5, 4], seed=11),
    "n9_n12": lambda: wl.make_workload("n9n12", [9, 12], [36, 48], [5, 4], [20, 13], seed=10),
    "diagonal_S": lambda: _diag(),
    "repeated_labels": lambda: _repeat(),
    "two_column_sink_families": lambda: _two_col_sinks(),
    "two_row_families": lambda: wl.make_workload("r2", [12, 10], [60, 48], [6, 5, 4, 7], [5, 6, 4, 3],
                                                 seed=41, two_row_frac=0.5),
    "two_row_sources_one_column_sinks": lambda: _two_row_sources(),
    "eight_flavours": lambda: wl.make_workload("f8", [2, 3, 1, 4, 2, 3, 1, 2], [12, 16, 8, 20, 12, 16, 8, 12],
                                               [5, 4], [6, 3], seed=51),
    "n32": lambda: wl.make_workload("n32", [32], [64], [3, 2], [6, 4], seed=12),
    "single_terms": lambda: wl.make_workload("one", [3, 2], [10, 8], [1], [1], seed=53),
    "mixed_rows": lambda: wl.make_workload("mr", [12, 10], [60, 48], [9, 7, 8], [5, 6, 4], seed=97,
                                           mixed_rows=True),
    "two_row_families_n18": lambda: wl.make_workload("r2", [18, 18], [96, 96], [8, 6], [7, 5], diag=3.0,
                                                     seed=43, two_row_frac=0.5),
}


def _two_row_sources():
    """Two-row source families against sink families that change one column, so the
    adjoint takes the two-sided rank-2 x rank-1 blocks (kapply2)."""
    a = wl.make_workload("r2", [12, 10], [60, 48], [7, 5, 6], [9, 6, 8, 5], seed=47, two_row_frac=0.6)
    b = wl.make_workload("r2", [12, 10], [60, 48], [7, 5, 6], [9, 6, 8, 5], seed=47, two_row_frac=0.0)
    assert all(np.array_equal(x, y) for x, y in zip(a.S, b.S))
    return wl.Workload("r2", a.n_f, a.S, a.labels_src, a.w_src, b.labels_snk, b.w_snk)


def _two_col_sinks():
    """One-row source families against sink families that change two columns (n_f >= 10),
    so the adjoint takes the two-column blocks of the two-sided update."""
    a = wl.make_workload("tc", [12, 10], [60, 48], [7, 5, 4], [9, 6, 8, 5], seed=31, two_row_frac=0.0)
    b = wl.make_workload("tc", [12, 10], [60, 48], [7, 5, 4], [9, 6, 8, 5], seed=31, two_row_frac=0.6)
    assert all(np.array_equal(x, y) for x, y in zip(a.S, b.S))
    return wl.Workload("tc", a.n_f, a.S, a.labels_src, a.w_src, b.labels_snk, b.w_snk)


def _cut(w, n):
    w.labels_snk, w.w_snk = w.labels_snk[:n], w.w_snk[:n]
    return w


def _diag():
    w = wl.make_workload("diag", [3, 3], [8, 8], [4, 4, 4], [6, 6], seed=45)
    w.S = [np.ascontiguousarray(np.diag(np.diag(s))) for s in w.S]
    perm = np.concatenate([w.labels_src[:, :3][:, ::-1], w.labels_src[:, 3:]], axis=1)
    w.labels_snk = np.concatenate([w.labels_snk, perm]).astype(np.int32)
    w.w_snk = np.concatenate([w.w_snk, np.ones(perm.shape[0])])
    return w


def _repeat():
    w = wl.make_workload("repeat", [4, 3], [10, 9], [6, 3, 5], [4, 4, 3], seed=44)
    rng = np.random.default_rng(3)
    for t in rng.choice(w.labels_src.shape[0], 4, replace=False):
        w.labels_src[t, 1] = w.labels_src[t, 0]
    return w


@pytest.mark.parametrize("name", list(CASES))
def test_backward_matches_oracle(M, name):
    check_vs_oracle(M, CASES[name]())


def test_backward_deterministic(M):
    w = CASES["he4_small"]()
    opts = M.default_opts()
    opts.rank2 = 0
    plan = M.Plan.from_workload(w, opts)
    S = dev_S(w)
    a = gpu_backward(M, plan, S, (0.3, 0.7))
    b = gpu_backward(M, plan, S, (0.3, 0.7))
    for x, y in zip(a[0] + [a[1], a[2]], b[0] + [b[1], b[2]]):
        assert x.tobytes() == y.tobytes()


def test_autograd_function(M):
    w = CASES["deuteron"]()
    plan = M.Plan.from_workload(w)
    S = [s.requires_grad_(True) for s in dev_S(w)]
    ws = torch.from_numpy(w.w_src).cuda().requires_grad_(True)
    wk = torch.from_numpy(w.w_snk).cuda().requires_grad_(True)
    C = M.correlator(plan, S, ws, wk)
    loss = 0.7 * C.real - 1.3 * C.imag
    loss.backward()
    ref = oracle.correlator_grad(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
    g = complex(0.7, -1.3)
    Cref, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
    for f in range(2):
        assert np.max(np.abs(S[f].grad.cpu().numpy() - g * np.conj(ref["dS"][f]))) <= 1e-10 * scale
    assert np.max(np.abs(ws.grad.cpu().numpy() - (np.conj(g) * ref["dw_src"]).real)) <= 1e-10 * scale
    assert np.max(np.abs(wk.grad.cpu().numpy() - (np.conj(g) * ref["dw_snk"]).real)) <= 1e-10 * scale


def test_full_helium4_fd_and_oracle(M):
    """4096 x 4096, n = 6: backward of Re C and Im C against central differences of the GPU
    forward on 200 random touched S entries (real and imaginary directions) and 200
    weights, and the full problem's gradient (every dS_f entry, every weight, three loss
    directions) against the oracle's Jacobi-formula gradient (cofactors from signed minors)."""
    w = wl.helium4()
    opts = M.default_opts()
    opts.rank2 = 0
    plan = M.Plan.from_workload(w, opts)
    S = dev_S(w)
    _, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, threads=16)
    dS_r, dws_r, dwk_r = gpu_backward(M, plan, S, (1.0, 0.0))   # L = Re C
    dS_i, dws_i, dwk_i = gpu_backward(M, plan, S, (0.0, 1.0))   # L = Im C
    rng = np.random.default_rng(77)
    h = 1e-6
    out = torch.empty(2, dtype=torch.float64, device="cuda")

    def C_of(Sx, ws=None, wk=None):
        plan.correlator(Sx, ws, wk, out=out)
        return complex(*out.cpu().numpy())

    # entries touched by some pair: rows and columns present in the label lists
    for k in range(100):
        f = int(rng.integers(2))
        a = int(w.labels_src[rng.integers(len(w.w_src)), 6 * f + rng.integers(6)])
        b = int(w.labels_snk[rng.integers(len(w.w_snk)), 6 * f + rng.integers(6)])
        for direction in (1.0, 1j):
            Sp = [s.clone() for s in S]
            Sm = [s.clone() for s in S]
            Sp[f][a, b] += h * direction
            Sm[f][a, b] -= h * direction
            fd = (C_of(Sp) - C_of(Sm)) / (2 * h)   # dC along this direction
            # torch gradient of L = Re C is conj(dC/dS); pairing with the direction:
            # dRe C = Re(dC/dS * dir) = Re(conj(grad_r) * dir)
            g_r = dS_r[f][a, b]
            g_i = dS_i[f][a, b]
            assert abs(fd.real - (np.conj(g_r) * direction).real) <= 1e-9 * scale
            assert abs(fd.imag - (np.conj(g_i) * direction).real) <= 1e-9 * scale
    for side in ("src", "snk"):
        n = len(w.w_src) if side == "src" else len(w.w_snk)
        for idx in rng.choice(n, 100, replace=False):
            base = torch.from_numpy(w.w_src if side == "src" else w.w_snk).cuda()
            wp, wm = base.clone(), base.clone()
            wp[idx] += h
            wm[idx] -= h
            if side == "src":
                fd = (C_of(S, wp, None) - C_of(S, wm, None)) / (2 * h)
                gr, gi = dws_r[idx], dws_i[idx]
            else:
                fd = (C_of(S, None, wp) - C_of(S, None, wm)) / (2 * h)
                gr, gi = dwk_r[idx], dwk_i[idx]
            assert abs(fd.real - gr) <= 1e-9 * scale and abs(fd.imag - gi) <= 1e-9 * scale
    plan.close()
    # Jacobi gradient of the oracle on the whole problem (same plan options)
    check_vs_oracle(M, w, opts, threads=16)


def test_two_row_family_with_repeated_shared_label(M):
    """Two-row families whose shared rows hold a repeated label: the shared rows are
    rank-deficient, so every member's determinant and every member-row cofactor is 0 and
    only the repeated rows' cofactors survive (from signed minors).  The gradient against
    the oracle's Jacobi gradient, and a clean status.  (Repeated labels under one-row
    families: the repeated_labels case.)"""
    w = CASES["two_row_families"]()
    info = w.meta["src"]
    hit = 0
    for p in range(len(info["family_sizes"])):
        rows = info["rows"][p][0]
        if len(rows) != 2 or 0 in rows or 1 in rows:
            continue
        terms = np.nonzero(info["family_of"] == p)[0]
        w.labels_src[terms, 1] = w.labels_src[terms, 0]   # shared rows 0 and 1 repeat in flavour 0
        hit += 1
        if hit == 2:
            break
    assert hit >= 1
    opts = M.default_opts()
    opts.rank2 = 1
    plan = M.Plan.from_workload(w, opts)
    assert plan.stats()["rank2_family_flavours"] > 0
    plan.close()
    check_vs_oracle(M, w, opts)


def test_two_row_family_with_near_singular_shared_rows(M):
    """Two-row families whose shared rows are nearly dependent: in two families whose shared
    rows hold a twin origin o_t, another shared row of every member becomes twin(o_t) (a copy
    of row o_t plus 1e-13 noise), so the shared-row factorisation fails the pivot guard for
    every sink and the null vectors are recomputed with complete pivoting.  The gradient
    against the oracle's Jacobi gradient (the other families keep flavour 1's scale regular:
    a flavour-1 entry whose every contribution carries a 1e-13 determinant would be compared
    at a scale below its FP64 error)."""
    w = wl.make_workload("r2", [12, 10], [60, 48], [6, 5, 4, 7, 5], [5, 6, 4, 3], seed=41,
                         two_row_frac=1.0, twins=8)
    info = w.meta["src"]
    origin = w.meta["twin_origin"][0]
    L0, changed = 60, 0
    for p, size in enumerate(info["family_sizes"]):
        terms = np.nonzero(info["family_of"] == p)[0]
        rows = info["rows"][p][0]
        parent = w.labels_src[terms[0], :12]
        shared = [s for s in range(12) if s not in rows]
        hit = [(s, origin.index(int(parent[s]))) for s in shared if int(parent[s]) in origin]
        if not hit:
            continue
        s0, t = hit[0]
        s1 = next(s for s in shared if s != s0)
        w.labels_src[terms, s1] = L0 - 8 + t
        changed += 1
        if changed == 2:       # the other families keep a regular scale for flavour 1
            break
    assert changed == 2
    opts = M.default_opts()
    opts.rank2 = 1
    check_vs_oracle(M, w, opts)


def test_backward_families_of_64(M):
    w = wl.make_workload("fam64", [4, 4], [40, 40], [64, 10], [64, 5], seed=52)
    opts = M.default_opts()
    opts.max_family = 64
    opts.rank2 = 0
    check_vs_oracle(M, w, opts)


def test_three_row_families(M):
    """Rank-3 families (opts.rank3, n_f >= 14): the adjoint against the oracle's Jacobi
    gradient, with and without sink families."""
    w = wl.make_workload("r3", [14, 10], [56, 40], [6, 5, 4], [4, 3], seed=61, two_row_frac=0.3,
                         three_row_frac=0.6)
    for one_sided in (0, 1):
        opts = M.default_opts()
        opts.rank3 = 1
        opts.one_sided = one_sided
        plan = M.Plan.from_workload(w, opts)
        assert plan.stats()["rank3_family_flavours"] > 0
        plan.close()
        check_vs_oracle(M, w, opts)


@pytest.mark.parametrize("k", [4, 5])
def test_rank_k_families(M, k):
    """The adjoint of rank-k families (k = 4, 5: member-row cofactors sd Z adj(D), the
    shared rows' from the right inverse of the shared rows; adj(D) from (k-1) x (k-1)
    minors) against the oracle's Jacobi gradient, with and without sink families."""
    if k == 4:
        w = wl.make_workload("r4", [18, 12], [96, 60], [5, 4, 3, 4], [4, 3, 5], diag=3.0, seed=95,
                             two_row_frac=0.3, more_rows=[{4: 0.7}, {}])
    else:
        w = wl.make_workload("r5", [22, 10], [110, 40], [5, 4, 3], [3, 4, 2], diag=3.0, seed=96,
                             more_rows=[{4: 0.3, 5: 0.6}, {}])
    for one_sided in (0, 1):
        opts = M.default_opts()
        opts.max_rank = k
        opts.one_sided = one_sided
        plan = M.Plan.from_workload(w, opts)
        assert int(plan.families()["rank"].max()) == k
        plan.close()
        check_vs_oracle(M, w, opts)
