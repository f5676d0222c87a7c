"""Pins of the oracle: checks against facts fixed by the paper and by mathematics, not by
the oracle itself.  Each check raises AssertionError on a mismatch.  They are run by
tests/test_oracle_pins.py against the oracle, and by tests/test_oracle_mutants.py
against oracle builds with a planted mistake (each such build must fail at least one).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

import oracle
from paper_1411_3691_gb300 import workloads as wl


def rand_c(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


def perm_sign(p) -> int:
    p = list(p)
    inv = sum(1 for a in range(len(p)) for b in range(a + 1, len(p)) if p[a] > p[b])
    return -1 if inv % 2 else 1


def leibniz(G) -> complex:
    """det as the signed permutation sum (the epsilon-tensor form of Sec. 1)."""
    n = G.shape[0]
    tot = 0j
    for p in itertools.permutations(range(n)):
        t = complex(perm_sign(p))
        for m in range(n):
            t *= complex(G[m, p[m]])
        tot += t
    return tot


# ---- exact complex-rational arithmetic (for exact determinants of float inputs) ----
def _cf(z):
    return (Fraction(float(np.real(z))), Fraction(float(np.imag(z))))


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def _csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def _cdiv(a, b):
    d = b[0] * b[0] + b[1] * b[1]
    return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)


def exact_det(G):
    """Exact determinant of the exact binary values of G (Gaussian elimination over Q[i])."""
    n = G.shape[0]
    A = [[_cf(G[m, q]) for q in range(n)] for m in range(n)]
    det = (Fraction(1), Fraction(0))
    for k in range(n):
        p = next((i for i in range(k, n) if A[i][k] != (0, 0)), None)
        if p is None:
            return (Fraction(0), Fraction(0))
        if p != k:
            A[k], A[p] = A[p], A[k]
            det = (-det[0], -det[1])
        det = _cmul(det, A[k][k])
        for i in range(k + 1, n):
            l = _cdiv(A[i][k], A[k][k])
            for q in range(k + 1, n):
                A[i][q] = _csub(A[i][q], _cmul(l, A[k][q]))
    return det


def _close(a, b, tol, scale):
    assert abs(a - b) <= tol * scale, f"|{a} - {b}| = {abs(a - b):.3e} > {tol:.1e} * {scale:.3e}"


# ------------------------------------------------------------------------------------------
def check_leibniz():
    """LU det equals the signed permutation sum for n <= 5 (Sec. 1)."""
    rng = np.random.default_rng(11)
    for n in range(1, 6):
        for _ in range(4):
            G = rand_c(rng, (n, n))
            ref = leibniz(G)
            scale = sum(math.prod(abs(G[m, p[m]]) for m in range(n))
                        for p in itertools.permutations(range(n)))
            _close(oracle.det(G), ref, 1e-14, scale)


def check_double_permutation_sum():
    """The alpha/beta double sum over orderings with epsilon^alpha epsilon^beta (Sec. 1)
    equals n! det G^{(ij)}; the correlator uses det (the n! is dropped)."""
    rng = np.random.default_rng(12)
    L = 7
    S = rand_c(rng, (L, L))
    for n in range(1, 5):
        a = rng.choice(L, size=n, replace=False)
        b = rng.choice(L, size=n, replace=False)
        tot = 0j
        for al in itertools.permutations(range(n)):
            for be in itertools.permutations(range(n)):
                t = complex(perm_sign(al) * perm_sign(be))
                for m in range(n):
                    t *= S[a[al[m]], b[be[m]]]
                tot += t
        d = oracle.pair_dets([S], [n], a[None, :], b[None, :], [0], [0])[0, 0]
        _close(tot / math.factorial(n), d, 1e-13, 1.0 + abs(d) + abs(tot) / math.factorial(n))


def check_exact_rational():
    """fp64 det within its error bound of the exact determinant of the same inputs; the
    double-double det within 1e-24 relative (well-conditioned) and within kappa * 2^-100
    (ill-conditioned)."""
    rng = np.random.default_rng(13)
    for n in (2, 3, 5, 7):
        for _ in range(3):
            G = (rng.integers(-8, 9, size=(n, n)) + 1j * rng.integers(-8, 9, size=(n, n))) / 8.0
            G += 3.0 * np.eye(n)
            ex = exact_det(G)
            exc = complex(float(ex[0]), float(ex[1]))
            kap = oracle.cond_inf(G)
            _close(oracle.det(G), exc, 8 * n * 2.0**-53 * kap, abs(exc))
            hi_re, lo_re, hi_im, lo_im = oracle.det_dd(G)
            err = abs((Fraction(hi_re) + Fraction(lo_re) - ex[0])) + abs((Fraction(hi_im) + Fraction(lo_im) - ex[1]))
            assert float(err) <= 1e-24 * abs(exc), (n, float(err), abs(exc))
    # ill-conditioned: two rows equal up to 2^-40
    n = 5
    G = rand_c(rng, (n, n))
    G[3] = G[1] + 2.0**-40 * rand_c(rng, n)
    ex = exact_det(G)
    exc = complex(float(ex[0]), float(ex[1]))
    kap = oracle.cond_inf(G)
    assert kap > 1e9
    hi_re, lo_re, hi_im, lo_im = oracle.det_dd(G)
    err = abs((Fraction(hi_re) + Fraction(lo_re) - ex[0])) + abs((Fraction(hi_im) + Fraction(lo_im) - ex[1]))
    assert float(err) <= 8 * n * 2.0**-100 * kap * abs(exc)
    _close(oracle.det(G), exc, 8 * n * 2.0**-53 * kap, abs(exc))


def check_gather_orientation():
    """G^{(ij)}[m][q] = S[a_i^m][a_j^q]: rows from the source term, columns from the sink
    term (Sec. 1); compared with LAPACK's det of the same gathered block."""
    rng = np.random.default_rng(14)
    L, n = 9, 4
    S = rand_c(rng, (L, L))
    for _ in range(5):
        a = rng.choice(L, size=n, replace=False)
        b = rng.choice(L, size=n, replace=False)
        d = oracle.pair_dets([S], [n], a[None, :], b[None, :], [0], [0])[0, 0]
        ref = np.linalg.det(S[np.ix_(a, b)])
        _close(d, ref, 1e-13, abs(ref) + 1.0)


def check_swap_and_repeat():
    """Swapping two labels of a term flips the sign; a repeated label gives exactly 0
    (the wavefunction tensor vanishes on equal indices, Sec. 1)."""
    rng = np.random.default_rng(15)
    L, n = 12, 5
    S = rand_c(rng, (L, L)) + 2 * np.eye(L)
    a = rng.choice(L, size=n, replace=False).astype(np.int32)
    b = rng.choice(L, size=n, replace=False).astype(np.int32)
    a2 = a.copy()
    a2[[1, 3]] = a2[[3, 1]]
    b2 = b.copy()
    b2[[0, 4]] = b2[[4, 0]]
    rep = a.copy()
    rep[2] = rep[0]
    src = np.stack([a, a2, rep, a])
    snk = np.stack([b, b, b, b2])
    d = oracle.pair_dets([S], [n], src, snk, [0, 1, 2, 3], [0, 1, 2, 3])[:, 0]
    _close(d[1], -d[0], 1e-14, abs(d[0]))
    _close(d[3], -d[0], 1e-14, abs(d[0]))
    assert d[2] == 0.0


def check_block_diagonal():
    """det G = prod_f det G_f for the flavour-block-diagonal G (end of Sec. 1)."""
    rng = np.random.default_rng(16)
    n_f = [3, 2, 4]
    L_f = [8, 6, 9]
    S = [rand_c(rng, (L, L)) for L in L_f]
    src = np.concatenate([rng.choice(L, size=n, replace=False) for n, L in zip(n_f, L_f)])[None, :]
    snk = np.concatenate([rng.choice(L, size=n, replace=False) for n, L in zip(n_f, L_f)])[None, :]
    d = oracle.pair_dets(S, n_f, src, snk, [0], [0])[0]
    N = sum(n_f)
    big = np.zeros((N, N), dtype=complex)
    off = 0
    for f, n in enumerate(n_f):
        big[off:off + n, off:off + n] = S[f][np.ix_(src[0, off:off + n], snk[0, off:off + n])]
        off += n
    ref = np.linalg.det(big)
    _close(np.prod(d), ref, 1e-13, abs(ref))


def check_lemma():
    """det(G + u v^T) = (1 + v^T G^{-1} u) det G (Sec. 2.1) with u = e_r, and the rank-2
    form det(G + U V^T) = det(I + V^T G^{-1} U) det G, for a child whose changed row
    comes from the same propagator."""
    rng = np.random.default_rng(17)
    L, n = 20, 6
    S = rand_c(rng, (L, L)) + 2 * np.eye(L)
    perm = rng.permutation(L)
    a = perm[:n].astype(np.int32)
    b = rng.choice(L, size=n, replace=False).astype(np.int32)
    G = S[np.ix_(a, b)]
    dG = oracle.det(G)
    for r in range(n):
        c = a.copy()
        c[r] = perm[n + r]
        v = S[c[r], b] - G[r]
        x = np.linalg.solve(G, np.eye(n)[:, r])
        direct = oracle.pair_dets([S], [n], c[None, :], b[None, :], [0], [0])[0, 0]
        _close(direct, (1 + v @ x) * dG, 1e-12, abs(direct) + abs(dG))
    r1, r2 = 1, 4
    c = a.copy()
    c[r1], c[r2] = perm[n], perm[n + 1]
    U = np.eye(n)[:, [r1, r2]]
    V = np.stack([S[c[r1], b] - G[r1], S[c[r2], b] - G[r2]], axis=1)
    M = np.eye(2) + V.T @ np.linalg.solve(G, U)
    direct = oracle.pair_dets([S], [n], c[None, :], b[None, :], [0], [0])[0, 0]
    _close(direct, np.linalg.det(M) * dG, 1e-12, abs(direct) + abs(dG))


def check_diag_closed_form():
    """S_f = diag(d_f): det G = sgn(pi) prod_m d[a^m] when the sink tuple is a permutation
    pi of the source tuple, else 0; the whole correlator in closed form."""
    rng = np.random.default_rng(18)
    L, n = 6, 3
    d = [rand_c(rng, L), rand_c(rng, L)]
    S = [np.diag(x) for x in d]
    base = list(itertools.combinations(range(L), n))[:6]
    terms = []
    for t in base:
        for p in list(itertools.permutations(t))[:3]:
            terms.append(p)
    terms = terms[:14]
    rows = []
    for k, tu in enumerate(terms):
        tv = terms[(5 * k + 3) % len(terms)]
        rows.append(list(tu) + list(tv))
    src = np.array(rows, dtype=np.int32)
    snk = np.array(rows[::-1], dtype=np.int32)
    ws = rng.normal(size=len(src))
    wk = rng.normal(size=len(snk))

    def det_diag(dd, a, b):
        if sorted(a) != sorted(b) or len(set(a)) < len(a):
            return 0.0
        pos = [list(b).index(x) for x in a]
        return perm_sign(pos) * math.prod(dd[x] for x in a)

    ref = 0j
    scale = 0.0
    for i in range(len(src)):
        for j in range(len(snk)):
            v = ws[i] * wk[j]
            for f in range(2):
                v *= det_diag(d[f], src[i, f * n:(f + 1) * n], snk[j, f * n:(f + 1) * n])
            ref += v
            scale += abs(v)
    C, sc = oracle.correlator(S, [n, n], src, ws, snk, wk)
    assert scale > 0
    _close(C, ref, 1e-14, scale)
    _close(sc, scale, 1e-14, scale)


def cauchy_binet_problem(rng, F, Lp, n):
    """All sorted n-subsets of [Lp] (product sets across flavours) as terms with
    w = prod_f det(P_f[:, a^f]) (source) and prod_f det(Q_f[:, b^f]) (sink)."""
    subs = list(itertools.combinations(range(Lp), n))
    P = [rng.normal(size=(n, Lp)) for _ in range(F)]
    Q = [rng.normal(size=(n, Lp)) for _ in range(F)]
    S = [rand_c(rng, (Lp, Lp)) for _ in range(F)]
    combos = list(itertools.product(range(len(subs)), repeat=F))
    labels = np.array([[x for f in range(F) for x in subs[c[f]]] for c in combos], dtype=np.int32)
    ws = np.array([math.prod(np.linalg.det(P[f][:, list(subs[c[f]])]) for f in range(F)) for c in combos])
    wk = np.array([math.prod(np.linalg.det(Q[f][:, list(subs[c[f]])]) for f in range(F)) for c in combos])
    M = [P[f] @ S[f] @ Q[f].T for f in range(F)]
    C = math.prod(np.linalg.det(m) for m in M)
    return S, labels, ws, wk, P, Q, M, C


def check_cauchy_binet():
    """Sum over all sorted subsets: C = prod_f det(P_f S_f Q_f^T) (Cauchy-Binet twice)."""
    rng = np.random.default_rng(19)
    for F, Lp, n in ((1, 9, 3), (2, 6, 2)):
        S, lab, ws, wk, P, Q, M, Cref = cauchy_binet_problem(rng, F, Lp, n)
        C, sc = oracle.correlator(S, [n] * F, lab, ws, lab, wk)
        _close(C, Cref, 1e-12, sc)


def check_cauchy_binet_grad():
    """dC/dS_f = (prod_{f'!=f} det M_f') det M_f P_f^T M_f^{-T} Q_f and
    dC/dw_i = prod_f det((S_f Q_f^T)[a_i^f, :]) for the Cauchy-Binet problem."""
    rng = np.random.default_rng(20)
    F, Lp, n = 2, 5, 2
    S, lab, ws, wk, P, Q, M, Cref = cauchy_binet_problem(rng, F, Lp, n)
    g = oracle.correlator_grad(S, [n] * F, lab, ws, lab, wk)
    dets = [np.linalg.det(m) for m in M]
    for f in range(F):
        others = math.prod(dets[k] for k in range(F) if k != f)
        ref = others * dets[f] * P[f].T @ np.linalg.inv(M[f]).T @ Q[f]
        sc = max(float(np.max(g["dS_scale"][f])), 1e-300)
        assert np.max(np.abs(g["dS"][f] - ref)) <= 1e-12 * sc
    SQ = [S[f] @ Q[f].T for f in range(F)]
    ref_w = np.array([math.prod(np.linalg.det(SQ[f][lab[i, f * n:(f + 1) * n], :]) for f in range(F))
                      for i in range(lab.shape[0])])
    assert np.max(np.abs(g["dw_src"] - ref_w)) <= 1e-12 * max(float(np.max(g["dw_src_scale"])), 1e-300)
    PS = [P[f] @ S[f] for f in range(F)]
    ref_k = np.array([math.prod(np.linalg.det(PS[f][:, lab[j, f * n:(f + 1) * n]]) for f in range(F))
                      for j in range(lab.shape[0])])
    assert np.max(np.abs(g["dw_snk"] - ref_k)) <= 1e-12 * max(float(np.max(g["dw_snk_scale"])), 1e-300)


def check_n1_bilinear():
    """n_f = 1: C = sum_ij w_i w_j prod_f S_f[a_i][b_j], a bilinear form."""
    rng = np.random.default_rng(21)
    L = 7
    S = [rand_c(rng, (L, L)), rand_c(rng, (L, L))]
    src = rng.integers(0, L, size=(15, 2)).astype(np.int32)
    snk = rng.integers(0, L, size=(11, 2)).astype(np.int32)
    ws, wk = rng.normal(size=15), rng.normal(size=11)
    K = S[0][np.ix_(src[:, 0], snk[:, 0])] * S[1][np.ix_(src[:, 1], snk[:, 1])]
    ref = ws @ K @ wk
    C, sc = oracle.correlator(S, [1, 1], src, ws, snk, wk)
    _close(C, ref, 1e-14, sc)


def check_grad_fd():
    """Oracle gradient against central differences (h = 1e-6).  Each S entry enters a
    distinct-label G at most once, so C is affine in it, and C is linear in each weight:
    the difference quotient has no truncation error, only rounding."""
    w = wl.make_workload("fd", [3, 2], [9, 7], [3, 2, 4], [2, 3, 2], seed=7)
    g = oracle.correlator_grad(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
    C0, scale = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
    rng = np.random.default_rng(22)
    h = 1e-6
    for f in range(2):
        L = w.S[f].shape[0]
        touched = np.argwhere(g["dS_scale"][f] > 0)
        pick = touched[rng.choice(len(touched), size=min(8, len(touched)), replace=False)]
        for a, b in pick:
            for direction in (1.0, 1j):
                Sp = [s.copy() for s in w.S]
                Sm = [s.copy() for s in w.S]
                Sp[f][a, b] += h * direction
                Sm[f][a, b] -= h * direction
                Cp, _ = oracle.correlator(Sp, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
                Cm, _ = oracle.correlator(Sm, w.n_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk)
                fd = (Cp - Cm) / (2 * h)          # = dC/dS * direction (C holomorphic)
                _close(fd, g["dS"][f][a, b] * direction, 1e-9, scale)
    for i in rng.choice(len(w.w_src), size=3, replace=False):
        wp, wm = w.w_src.copy(), w.w_src.copy()
        wp[i] += h
        wm[i] -= h
        Cp, _ = oracle.correlator(w.S, w.n_f, w.labels_src, wp, w.labels_snk, w.w_snk)
        Cm, _ = oracle.correlator(w.S, w.n_f, w.labels_src, wm, w.labels_snk, w.w_snk)
        _close((Cp - Cm) / (2 * h), g["dw_src"][i], 1e-9, scale)
    for j in rng.choice(len(w.w_snk), size=3, replace=False):
        wp, wm = w.w_snk.copy(), w.w_snk.copy()
        wp[j] += h
        wm[j] -= h
        Cp, _ = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, wp)
        Cm, _ = oracle.correlator(w.S, w.n_f, w.labels_src, w.w_src, w.labels_snk, wm)
        _close((Cp - Cm) / (2 * h), g["dw_snk"][j], 1e-9, scale)


def check_compensated_sum():
    """Neumaier summation: 1e16 + 1 - 1e16 in term order gives exactly 1."""
    S = [np.array([[1.0 + 0j]])]
    src = np.zeros((3, 1), dtype=np.int32)
    snk = np.zeros((1, 1), dtype=np.int32)
    C, sc = oracle.correlator(S, [1], src, np.array([1e16, 1.0, -1e16]), snk, np.array([1.0]))
    assert C == 1.0 + 0j, C


def check_brute_force():
    """Tiny problem (repeated labels included): LAPACK det per pair, summed in Python."""
    rng = np.random.default_rng(23)
    n_f, L_f = [3, 2], [6, 5]
    S = [rand_c(rng, (L, L)) for L in L_f]
    src = np.concatenate([rng.integers(0, L, size=(9, n)) for n, L in zip(n_f, L_f)], axis=1).astype(np.int32)
    snk = np.concatenate([rng.integers(0, L, size=(7, n)) for n, L in zip(n_f, L_f)], axis=1).astype(np.int32)
    ws, wk = rng.normal(size=9), rng.normal(size=7)
    ref = 0j
    scale = 0.0
    for i in range(9):
        for j in range(7):
            v = ws[i] * wk[j]
            off = 0
            for f, n in enumerate(n_f):
                v *= np.linalg.det(S[f][np.ix_(src[i, off:off + n], snk[j, off:off + n])])
                off += n
            ref += v
            scale += abs(v)
    C, sc = oracle.correlator(S, n_f, src, ws, snk, wk)
    _close(C, ref, 1e-13, scale)
    _close(sc, scale, 1e-12, scale)


def check_cond():
    """kappa_inf against LAPACK's inverse."""
    rng = np.random.default_rng(24)
    for n in (2, 4, 6):
        G = rand_c(rng, (n, n))
        ref = np.linalg.norm(G, np.inf) * np.linalg.norm(np.linalg.inv(G), np.inf)
        _close(oracle.cond_inf(G), ref, 1e-10, ref)


ALL_CHECKS = [check_leibniz, check_double_permutation_sum, check_exact_rational,
              check_gather_orientation, check_swap_and_repeat, check_block_diagonal,
              check_lemma, check_diag_closed_form, check_cauchy_binet, check_cauchy_binet_grad,
              check_n1_bilinear, check_grad_fd, check_compensated_sum, check_brute_force,
              check_cond]
