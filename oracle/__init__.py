"""Oracle: a plain, slow, obviously correct CPU reference for the multi-hadron correlator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The library (``paper_1411_3691_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``mhc_oracle.c`` (fresh partial-pivot LU per pair per flavour,
Sec. 1 and Sec. 2 of the paper); this module compiles it with gcc on first use, loads it
with ctypes and marshals numpy arrays.  Threaded calls split the source terms into
blocks, run them in parallel (ctypes releases the GIL) and combine the per-block
Neumaier states with ``math.fsum``, which is exact-rounded and independent of the
order of completion.

Functions whose parity is pinned by tests/test_oracle_pins.py: det, det_dd, cond_inf,
correlator, pair_dets, correlator_grad.  None is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_mhc_oracle.so")
_lib = None
_lock = threading.Lock()

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_CFLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_mhc_oracle.so (gcc, no arch-specific flags; no
    contraction of a*b+c into fused multiply-adds, which gcc does by default on some targets,
    so that the oracle rounds the same way on every host)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    lib.oracle_det.argtypes = [ctypes.c_int, _f64p, _f64p]
    lib.oracle_det.restype = None
    lib.oracle_det_dd.argtypes = [ctypes.c_int, _f64p, _f64p]
    lib.oracle_det_dd.restype = None
    lib.oracle_cond_inf.argtypes = [ctypes.c_int, _f64p]
    lib.oracle_cond_inf.restype = ctypes.c_double
    common = [ctypes.c_int, _i32p, _i32p, ctypes.POINTER(_f64p)]
    lib.oracle_correlator.argtypes = common + [
        ctypes.c_int64, _i32p, _f64p, ctypes.c_int64, _i32p, _f64p,
        ctypes.c_int64, ctypes.c_int64, _f64p, _f64p]
    lib.oracle_correlator.restype = ctypes.c_int
    lib.oracle_pair_dets.argtypes = common + [
        _i32p, _i32p, ctypes.c_int64, _i64p, _i64p, _f64p]
    lib.oracle_pair_dets.restype = ctypes.c_int
    lib.oracle_correlator_grad.argtypes = common + [
        ctypes.c_int64, _i32p, _f64p, ctypes.c_int64, _i32p, _f64p,
        ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
    lib.oracle_correlator_grad.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def build_mutant(k: int, out_dir: str) -> str:
    """Compile the oracle with planted mistake number k (mutation test of the pins)."""
    path = os.path.join(out_dir, f"_mhc_oracle_mutant{k}.so")
    subprocess.check_call(["gcc", *_CFLAGS, f"-DORACLE_MUTANT={k}", "-o", path, _SRC, "-lm"])
    return path


class use_library:
    """Context manager: route every oracle call through the library at `path`."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        with _lock:
            _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _p(a, t):
    return a.ctypes.data_as(t)


class _Problem:
    """Marshalled, contiguous copies of one correlator's inputs."""

    def __init__(self, S, n_f, labels_src, w_src, labels_snk, w_snk):
        self.F = len(n_f)
        self.n_f = np.ascontiguousarray(n_f, dtype=np.int32)
        self.S = [np.ascontiguousarray(s, dtype=np.complex128) for s in S]
        self.L_f = np.array([s.shape[0] for s in self.S], dtype=np.int32)
        for s in self.S:
            assert s.ndim == 2 and s.shape[0] == s.shape[1]
        self.ls = np.ascontiguousarray(labels_src, dtype=np.int32)
        self.lk = np.ascontiguousarray(labels_snk, dtype=np.int32)
        self.ws = np.ascontiguousarray(w_src, dtype=np.float64)
        self.wk = np.ascontiguousarray(w_snk, dtype=np.float64)
        T = int(self.n_f.sum())
        assert self.ls.shape == (self.ws.shape[0], T) or (T == 0 and self.ls.shape[0] == self.ws.shape[0])
        assert self.lk.shape == (self.wk.shape[0], T) or (T == 0 and self.lk.shape[0] == self.wk.shape[0])
        self.n_src = self.ws.shape[0]
        self.n_snk = self.wk.shape[0]
        self.S_ptrs = (_f64p * max(self.F, 1))(*[s.view(np.float64).ctypes.data_as(_f64p) for s in self.S])

    def head(self):
        return [self.F, _p(self.n_f, _i32p), _p(self.L_f, _i32p), self.S_ptrs]


def det(G) -> complex:
    """det of one square complex matrix by fresh partial-pivot LU (Sec. 2)."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    n = G.shape[0]
    out = np.zeros(2)
    _load().oracle_det(n, _p(G.view(np.float64), _f64p), _p(out, _f64p))
    return complex(out[0], out[1])


def det_dd(G):
    """det in double-double arithmetic; returns (re_hi, re_lo, im_hi, im_lo)."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    out = np.zeros(4)
    _load().oracle_det_dd(G.shape[0], _p(G.view(np.float64), _f64p), _p(out, _f64p))
    return tuple(float(x) for x in out)


def cond_inf(G) -> float:
    """Infinity-norm condition number from the explicit inverse."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    return float(_load().oracle_cond_inf(G.shape[0], _p(G.view(np.float64), _f64p)))


def _blocks(n, nblocks):
    nblocks = max(1, min(nblocks, n))
    edges = [round(k * n / nblocks) for k in range(nblocks + 1)]
    return [(edges[k], edges[k + 1]) for k in range(nblocks) if edges[k + 1] > edges[k]]


def correlator(S, n_f, labels_src, w_src, labels_snk, w_snk, threads: int = 1, src_range=None):
    """C = sum_i sum_j w_i w_j prod_f det G_f^(ij) with fresh LUs (Sec. 1).

    Returns (C, scale) with scale = sum |w_i w_j prod det|.  ``src_range=(i0, i1)``
    restricts the source sum.  ``threads`` > 1 splits the source range into blocks.
    """
    lib = _load()
    pr = _Problem(S, n_f, labels_src, w_src, labels_snk, w_snk)
    i0, i1 = src_range if src_range is not None else (0, pr.n_src)

    def run(b):
        sums = np.zeros(4)
        scale = np.zeros(1)
        rc = lib.oracle_correlator(*pr.head(), pr.n_src, _p(pr.ls, _i32p), _p(pr.ws, _f64p),
                                   pr.n_snk, _p(pr.lk, _i32p), _p(pr.wk, _f64p), b[0], b[1],
                                   _p(sums, _f64p), _p(scale, _f64p))
        if rc != 0:
            raise ValueError("oracle_correlator: bad argument")
        return sums, scale[0]

    blocks = _blocks(i1 - i0, threads * 4 if threads > 1 else 1)
    blocks = [(i0 + a, i0 + b) for a, b in blocks] or [(i0, i0)]
    if threads > 1 and len(blocks) > 1:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(run, blocks))
    else:
        res = [run(b) for b in blocks]
    re = math.fsum([x for s, _ in res for x in (s[0], s[1])])
    im = math.fsum([x for s, _ in res for x in (s[2], s[3])])
    scale = math.fsum([sc for _, sc in res])
    return complex(re, im), scale


def pair_dets(S, n_f, labels_src, labels_snk, i_idx, j_idx, threads: int = 1):
    """Per-pair per-flavour determinants, complex array [n_pairs, F].  ``threads`` > 1
    splits the pair list into blocks evaluated in parallel (each pair is independent)."""
    lib = _load()
    n_src = np.asarray(labels_src).shape[0]
    n_snk = np.asarray(labels_snk).shape[0]
    pr = _Problem(S, n_f, labels_src, np.zeros(n_src), labels_snk, np.zeros(n_snk))
    ii = np.ascontiguousarray(i_idx, dtype=np.int64)
    jj = np.ascontiguousarray(j_idx, dtype=np.int64)
    assert ii.shape == jj.shape
    assert (ii.size == 0) or (ii.min() >= 0 and ii.max() < n_src and jj.min() >= 0 and jj.max() < n_snk)
    out = np.zeros((ii.size, pr.F, 2))

    def run(b):
        a, e = b
        rc = lib.oracle_pair_dets(*pr.head(), _p(pr.ls, _i32p), _p(pr.lk, _i32p), e - a,
                                  _p(ii[a:], _i64p), _p(jj[a:], _i64p), _p(out[a:], _f64p))
        if rc != 0:
            raise ValueError("oracle_pair_dets: bad argument")

    blocks = _blocks(ii.size, threads * 4 if threads > 1 else 1) or [(0, 0)]
    if threads > 1 and len(blocks) > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, blocks))
    else:
        for b in blocks:
            run(b)
    return out[..., 0] + 1j * out[..., 1]


def correlator_grad(S, n_f, labels_src, w_src, labels_snk, w_snk, threads: int = 1):
    """Holomorphic derivatives dC/dS_f (complex, L_f x L_f each), dC/dw_src, dC/dw_snk
    (complex), each with its absolute scale, by Jacobi's formula with cofactors taken
    from their definition (signed minors)."""
    lib = _load()
    pr = _Problem(S, n_f, labels_src, w_src, labels_snk, w_snk)
    tot = int(sum(int(L) * int(L) for L in pr.L_f))

    def run(b):
        dS = np.zeros(tot, dtype=np.complex128)
        dSs = np.zeros(tot)
        dwi = np.zeros(pr.n_src, dtype=np.complex128)
        dwis = np.zeros(pr.n_src)
        dwj = np.zeros(pr.n_snk, dtype=np.complex128)
        dwjs = np.zeros(pr.n_snk)
        rc = lib.oracle_correlator_grad(
            *pr.head(), pr.n_src, _p(pr.ls, _i32p), _p(pr.ws, _f64p), pr.n_snk, _p(pr.lk, _i32p),
            _p(pr.wk, _f64p), b[0], b[1], _p(dS.view(np.float64), _f64p), _p(dSs, _f64p),
            _p(dwi.view(np.float64), _f64p), _p(dwis, _f64p), _p(dwj.view(np.float64), _f64p),
            _p(dwjs, _f64p))
        if rc != 0:
            raise ValueError("oracle_correlator_grad: bad argument")
        return dS, dSs, dwi, dwis, dwj, dwjs

    blocks = _blocks(pr.n_src, threads * 4 if threads > 1 else 1) or [(0, 0)]
    if threads > 1 and len(blocks) > 1:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(run, blocks))
    else:
        res = [run(b) for b in blocks]
    acc = [sum(r[k] for r in res) for k in range(6)]
    dS, dSs = acc[0], acc[1]
    out_S, out_Ss, off = [], [], 0
    for L in pr.L_f:
        L = int(L)
        out_S.append(dS[off:off + L * L].reshape(L, L))
        out_Ss.append(dSs[off:off + L * L].reshape(L, L))
        off += L * L
    return {"dS": out_S, "dS_scale": out_Ss, "dw_src": acc[2], "dw_src_scale": acc[3],
            "dw_snk": acc[4], "dw_snk_scale": acc[5]}
