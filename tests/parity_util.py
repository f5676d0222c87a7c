"""Parity helpers shared by the GPU tests (test support; not a test file).

Tolerances (from the arithmetic):
  * C: |C_gpu - C_oracle| <= 1e-11 * sum_ij |w_i w_j prod det| (the oracle returns the sum).
  * per pair and flavour: |d_gpu - d_ref| <= 1e-12 |d_ref|; for a block too ill-conditioned for
    that bound to be reachable by any FP64 method (the forced near-singular members),
    |d_gpu - d_dd| <= 4 n u kappa_inf(G) |d_dd| with d_dd the determinant in double-double and
    u = 2^-53 (a backward-stable LU's forward error bound).
"""
import numpy as np

import oracle

U = 2.0 ** -53


def check_pairs(M, w, plan, S, ii, jj, threads=16):
    """Per-pair determinants of the probe (mhc_pair_dets) against the oracle's fresh LUs.
    Returns (path bits per pair, number of blocks checked against the conditioning bound)."""
    import torch
    ii = np.asarray(ii, dtype=np.int64)
    jj = np.asarray(jj, dtype=np.int64)
    it = torch.from_numpy(ii).cuda()
    jt = torch.from_numpy(jj).cuda()
    path = torch.zeros(len(ii), dtype=torch.int32, device="cuda")
    got = plan.pair_dets(S, it, jt, path).cpu().numpy()
    path = path.cpu().numpy()
    assert M.mhc_get_status_code(plan.handle) == M.MHC_OK
    ref = oracle.pair_dets(w.S, w.n_f, w.labels_src, w.labels_snk, ii, jj, threads=threads)
    off = np.cumsum([0] + list(w.n_f))
    err = np.abs(got - ref)
    bad = err > 1e-12 * np.abs(ref)
    for f, n in enumerate(w.n_f):
        if n == 0:
            bad[:, f] = False
    n_ill = 0
    for p, f in zip(*np.nonzero(bad)):
        n = w.n_f[f]
        G = w.S[f][np.ix_(w.labels_src[ii[p], off[f]:off[f] + n], w.labels_snk[jj[p], off[f]:off[f] + n])]
        kap = oracle.cond_inf(G)
        hr, lr, hi, li = oracle.det_dd(G)
        dd = complex(hr + lr, hi + li)
        n_ill += 1
        assert abs(got[p, f] - dd) <= 4 * n * U * kap * abs(dd) + 1e-300, (p, f, got[p, f], dd, kap)
    return path, n_ill


def family_mask(w, n_fam, seed):
    """Source weights with every term outside n_fam random families of the workload's
    generator set to zero, and the kept term indices.  The planner does not look at weight
    values, so a plan built with these weights has the same families, work items and launch
    configuration as the full plan, while its correlator is the sum over the kept terms only."""
    fam_of = np.asarray(w.meta["src"]["family_of"])
    n_all = int(fam_of.max()) + 1
    rng = np.random.default_rng(seed)
    keep_fams = rng.choice(n_all, size=min(n_fam, n_all), replace=False)
    keep = np.nonzero(np.isin(fam_of, keep_fams))[0]
    ws = np.zeros_like(w.w_src)
    ws[keep] = w.w_src[keep]
    return ws, keep


def oracle_subset(w, keep, threads=16):
    """The oracle's C and scale over the kept source terms x all sinks."""
    return oracle.correlator(w.S, w.n_f, w.labels_src[keep], w.w_src[keep], w.labels_snk, w.w_snk,
                             threads=threads)
