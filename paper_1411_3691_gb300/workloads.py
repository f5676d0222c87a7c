"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and builds term lists; it holds none of the
method's arithmetic (no determinant, no update, no sum).  Both the GPU library's tests
and the oracle's tests take their inputs from here.

The paper's own wavefunctions (Sec. 4: alpha-particle wavefunctions with 1, 1944 and
5718 terms of 6x6 per-flavour blocks) are not available; these generators stand in
for their shape: two flavours, per-flavour label tuples of n distinct labels out of an
alphabet of L spin-colour-site labels, and terms that come in families sharing all but
one label per flavour (Sec. 3: the dominating sets printed in Sec. 4 give families of
about 8 to 11 terms).

Recipe (every workload):
  * S_f: re, im i.i.d. N(0, 1/2), plus diag * I.
  * A side (source or sink) is a list of families.  Per (family, flavour): a parent
    tuple of n distinct labels drawn without replacement from the ordinary labels and
    sorted; a changed row r ~ U{0..n-1} (two distinct rows for a two-row family).
    Member k > 0 replaces the label at r with a label not in the parent, drawn without
    replacement while the pool lasts and with replacement afterwards; the member keeps
    the parent's label positions.  Term (p, k) uses member k of family p in every
    flavour.
  * w ~ N(0, 1).
  * Seeds: numpy PCG64 streams from SeedSequence(seed).spawn(4): S, source, sink, shape.
  * Near-singular stress (large-nucleus workload): the top 8 labels of each flavour are
    "twins": S_f[L-8+t, :] = S_f[o_t, :] + 1e-13 (N(0,1/2) + i N(0,1/2)) for 8 distinct
    ordinary labels o_t; ordinary tuples never use twins; a forced member (1% of
    (member, flavour)) whose parent holds some o_t at a row s != r gets twin(o_t) at r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    n_f: list
    S: list                      # complex128 [L_f, L_f] per flavour
    labels_src: np.ndarray       # int32 [N_s, sum n_f]
    w_src: np.ndarray            # float64 [N_s]
    labels_snk: np.ndarray       # int32 [N_k, sum n_f]
    w_snk: np.ndarray            # float64 [N_k]
    meta: dict = field(default_factory=dict)

    @property
    def L_f(self):
        return [int(s.shape[0]) for s in self.S]

    @property
    def pairs(self) -> int:
        return int(self.w_src.shape[0]) * int(self.w_snk.shape[0])


def make_S(rng, L: int, diag: float) -> np.ndarray:
    re = rng.normal(0.0, math.sqrt(0.5), size=(L, L))
    im = rng.normal(0.0, math.sqrt(0.5), size=(L, L))
    S = re + 1j * im
    S += diag * np.eye(L)
    return np.ascontiguousarray(S, dtype=np.complex128)


def add_twins(rng, S: np.ndarray, n_twins: int = 8, noise: float = 1e-13):
    """Reserve the top n_twins labels as near-copies of n_twins ordinary rows."""
    L = S.shape[0]
    origin = rng.choice(L - n_twins, size=n_twins, replace=False)
    for t, o in enumerate(origin):
        e = rng.normal(0.0, math.sqrt(0.5), size=L) + 1j * rng.normal(0.0, math.sqrt(0.5), size=L)
        S[L - n_twins + t, :] = S[o, :] + noise * e
    return [int(o) for o in origin]


def make_side(rng, n_f, L_f, family_sizes, two_row_frac=0.0, forced_frac=0.0,
              n_ordinary=None, twin_origin=None, three_row_frac=0.0, more_rows=None, mixed_rows=False):
    """Term list of one side; returns (labels int32 [N, sum n_f], info dict).  more_rows:
    {k: fraction} (every flavour) or a list of such dicts (one per flavour) for families
    whose members change k >= 4 rows of a flavour (drawn only when given, so the other
    workloads keep their random streams).  mixed_rows: every member k > 0 of a family
    changes one row of its own choosing in each flavour (the family's rows are then all
    rows its members change), instead of the family's common rows."""
    F = len(n_f)
    Tn = int(sum(n_f))
    N = int(sum(family_sizes))
    labels = np.zeros((N, Tn), dtype=np.int32)
    fam_of = np.zeros(N, dtype=np.int64)
    member_of = np.zeros(N, dtype=np.int64)
    rows = []          # per family: per flavour tuple of changed rows
    forced = []        # (term, flavour) pairs that were forced near-singular
    t0 = 0
    for p, size in enumerate(family_sizes):
        fam_rows = []
        off = 0
        for f in range(F):
            n, L = int(n_f[f]), int(L_f[f])
            if n == 0:
                fam_rows.append(())
                continue
            ordinary = L if n_ordinary is None else int(n_ordinary[f])
            parent = np.sort(rng.choice(ordinary, size=n, replace=False)).astype(np.int32)
            two = n >= 2 and rng.random() < two_row_frac
            three = three_row_frac > 0 and n >= 3 and rng.random() < three_row_frac
            big = 0
            mr = more_rows[f] if isinstance(more_rows, (list, tuple)) else more_rows
            for k in sorted(mr or {}):
                if n >= k and rng.random() < mr[k]:
                    big = k
            if big:
                rr = tuple(sorted(int(x) for x in rng.choice(n, size=big, replace=False)))
            elif three:
                rr = tuple(sorted(int(x) for x in rng.choice(n, size=3, replace=False)))
            elif two:
                rr = tuple(sorted(int(x) for x in rng.choice(n, size=2, replace=False)))
            else:
                rr = (int(rng.integers(n)),)
            fam_rows.append(rr)
            pool = np.setdiff1d(np.arange(ordinary, dtype=np.int32), parent)
            need = (size - 1) * len(rr)
            if need <= pool.size:
                new = rng.choice(pool, size=need, replace=False)
            else:  # pool exhausted: repeat labels (repeated terms are legal)
                new = np.concatenate([rng.permutation(pool),
                                      rng.choice(pool, size=need - pool.size, replace=True)])
            new = new.astype(np.int32).reshape(max(size - 1, 0), len(rr)) if size > 1 else np.zeros((0, len(rr)), np.int32)
            own = [int(rng.integers(n)) for _ in range(size - 1)] if mixed_rows else None
            if mixed_rows:
                fam_rows[-1] = tuple(sorted(set(own)))
            for k in range(size):
                tup = parent.copy()
                if k > 0 and mixed_rows:
                    tup[own[k - 1]] = new[k - 1, 0]
                elif k > 0:
                    for t, r in enumerate(rr):
                        tup[r] = new[k - 1, t]
                    if forced_frac > 0 and twin_origin is not None and rng.random() < forced_frac:
                        # a parent label o_t at a row s outside rr: set row rr[0] to its twin
                        cands = [(s, twin_origin[f].index(int(parent[s])))
                                 for s in range(n) if s not in rr and int(parent[s]) in twin_origin[f]]
                        if cands:
                            s, t = cands[int(rng.integers(len(cands)))]
                            tup[rr[0]] = L - len(twin_origin[f]) + t
                            forced.append((t0 + k, f))
                labels[t0 + k, off:off + n] = tup
            off += n
        rows.append(fam_rows)
        fam_of[t0:t0 + size] = p
        member_of[t0:t0 + size] = np.arange(size)
        t0 += size
    info = {"family_sizes": list(map(int, family_sizes)), "rows": rows, "forced": forced,
            "family_of": fam_of, "member_of": member_of}
    return labels, info


def make_workload(name, n_f, L_f, fam_src, fam_snk, diag=2.0, seed=0, two_row_frac=0.0,
                  forced_frac=0.0, twins=0, three_row_frac=0.0, more_rows=None, mixed_rows=False):
    ss = np.random.SeedSequence(seed)
    r_S, r_src, r_snk, _ = [np.random.default_rng(s) for s in ss.spawn(4)]
    S = [make_S(r_S, int(L), diag) for L in L_f]
    twin_origin = None
    n_ord = None
    if twins:
        twin_origin = [add_twins(r_S, s, twins) for s in S]
        n_ord = [int(L) - twins for L in L_f]
    ls, info_s = make_side(r_src, n_f, L_f, fam_src, two_row_frac, forced_frac, n_ord, twin_origin,
                           three_row_frac, more_rows, mixed_rows)
    lk, info_k = make_side(r_snk, n_f, L_f, fam_snk, two_row_frac, 0.0, n_ord, twin_origin, three_row_frac)
    ws = r_src.normal(size=ls.shape[0])
    wk = r_snk.normal(size=lk.shape[0])
    return Workload(name, [int(x) for x in n_f], S, ls, ws, lk, wk,
                    {"src": info_s, "snk": info_k, "seed": seed, "twin_origin": twin_origin})


# --------------------------------------------------------------------------------------
# The five workloads (sizes as stated; `scale` < 1 shrinks the family counts for tests)
# --------------------------------------------------------------------------------------
def _fams(count, size, scale):
    return [size] * max(1, int(round(count * scale)))


def deuteron(scale: float = 1.0, seed: int = 0) -> Workload:
    """2 flavours, n=3, L=24; 512 x 512 terms as 64 families x 8 (parent + 7)."""
    return make_workload("deuteron_n3_L24_512x512", [3, 3], [24, 24], _fams(64, 8, scale),
                         _fams(64, 8, scale), diag=2.0, seed=seed)


def helium4(scale: float = 1.0, seed: int = 1000) -> Workload:
    """2 flavours, n=6, L=48; 4096 x 4096 terms as 256 families x 16 (parent + 15)."""
    return make_workload("he4_n6_L48_4096x4096", [6, 6], [48, 48], _fams(256, 16, scale),
                         _fams(256, 16, scale), diag=2.0, seed=seed)


def large_nucleus(scale: float = 1.0, seed: int = 3000) -> Workload:
    """2 flavours, n=18, L=96, +3I; 32768 x 32768 terms as 1024 families x 32; 10% of
    (family, flavour) with two changed rows; 1% forced near-singular members."""
    return make_workload("large_n18_L96_32768x32768", [18, 18], [96, 96], _fams(1024, 32, scale),
                         _fams(1024, 32, scale), diag=3.0, seed=seed, two_row_frac=0.1,
                         forced_frac=0.01, twins=8)


def batch_item(b: int, max_terms: int = 16384, min_terms: int = 256) -> Workload:
    """Batch item b: n_f ~ U{3,6,9,12,18} per flavour, L_f = 12 ceil(n_f/3) + 12, term
    counts per side log-uniform in [min_terms, max_terms], family sizes U[1, 32]."""
    seed = 2000 + b
    shape_rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(4)[3])
    n_f = [int(shape_rng.choice([3, 6, 9, 12, 18])) for _ in range(2)]
    L_f = [12 * math.ceil(n / 3) + 12 for n in n_f]

    def fams():
        N = int(round(math.exp(shape_rng.uniform(math.log(min_terms), math.log(max_terms)))))
        sizes = []
        while sum(sizes) < N:
            sizes.append(int(shape_rng.integers(1, 33)))
        sizes[-1] -= sum(sizes) - N
        return [s for s in sizes if s > 0]

    fs, fk = fams(), fams()
    return make_workload(f"batch{b}", n_f, L_f, fs, fk, diag=2.0, seed=seed)


def batch(count: int = 64, max_terms: int = 16384, min_terms: int = 256):
    return [batch_item(b, max_terms, min_terms) for b in range(count)]
