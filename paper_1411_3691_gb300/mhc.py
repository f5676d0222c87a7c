"""Python binding of the C ABI in include/mhc.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libmhc.so``; this module converts
numpy arrays and torch tensors to pointers, calls the entry point of the same name and
turns a non-zero status into an exception.  There is no fallback: if the library is
missing, importing the entry points raises.

Conventions: propagators S_f are complex128 CUDA tensors of shape (L_f, L_f), row-major
and contiguous; weights are float64 CUDA tensors; outputs are CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmhc.so")

MHC_OK, MHC_EINVAL, MHC_ENOMEM, MHC_ECUDA, MHC_ETIMEOUT, MHC_ENONFINITE, MHC_EUNSUPPORTED = range(7)
MHC_MAX_RANK = 6  # stride of the changed-row tables (include/mhc.h)
STATUS_NAMES = ["MHC_OK", "MHC_EINVAL", "MHC_ENOMEM", "MHC_ECUDA", "MHC_ETIMEOUT",
                "MHC_ENONFINITE", "MHC_EUNSUPPORTED"]
MHC_NMAX = 32
MHC_FMAX = 8

EXPORTED = ["mhc_last_error", "mhc_plan_opts_default", "mhc_plan", "mhc_plan_destroy",
            "mhc_plan_stats", "mhc_plan_families", "mhc_plan_sinks", "mhc_correlator", "mhc_correlator_noalloc",
            "mhc_correlator_cw",
            "mhc_correlator_backward",
            "mhc_pair_dets", "mhc_get_status", "mhc_batch_create", "mhc_batch_destroy",
            "mhc_batch_correlator", "mhc_batch_info", "mhc_batch_shape", "mhc_tune_cache_get",
            "mhc_tune_cache_put", "mhc_fp64_peak", "mhc_complex_reciprocal"]


class MHCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class PlanOpts(ctypes.Structure):
    _fields_ = [("tau_parent", ctypes.c_double), ("tau_child", ctypes.c_double),
                ("sink_tile", ctypes.c_int32), ("rank2", ctypes.c_int32),
                ("max_family", ctypes.c_int32), ("one_sided", ctypes.c_int32),
                ("rank3", ctypes.c_int32), ("max_rank", ctypes.c_int32), ("first_fit", ctypes.c_int32),
                ("row_difference", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Stats(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_snk", ctypes.c_int64), ("n_flavours", ctypes.c_int32),
                ("max_n", ctypes.c_int32), ("dominators", ctypes.c_int64), ("families", ctypes.c_int64),
                ("rank2_family_flavours", ctypes.c_int64), ("members", ctypes.c_int64),
                ("graph_edges", ctypes.c_int64), ("flops_per_call", ctypes.c_double),
                ("fresh_lu_flops_per_pair", ctypes.c_double), ("bytes_per_call", ctypes.c_double),
                ("plan_seconds", ctypes.c_double), ("refactor_parent", ctypes.c_int64),
                ("refactor_child", ctypes.c_int64), ("sink_families", ctypes.c_int64),
                ("two_sided_blocks", ctypes.c_int64), ("backward_flops_per_call", ctypes.c_double),
                ("rank3_family_flavours", ctypes.c_int64), ("refactor_flops", ctypes.c_double),
                ("rank4plus_family_flavours", ctypes.c_int64), ("row_difference", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run "
                               "python -c 'import __graft_entry__ as g; g.build()'")
        L = ctypes.CDLL(LIB_PATH)
        L.mhc_last_error.restype = ctypes.c_char_p
        L.mhc_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
        L.mhc_plan.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, _i32p, _i32p, ctypes.c_int64, _i32p,
                               _f64p, ctypes.c_int64, _i32p, _f64p, ctypes.POINTER(PlanOpts)]
        L.mhc_plan_destroy.argtypes = [_vp]
        L.mhc_plan_destroy.restype = None
        L.mhc_plan_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
        L.mhc_plan_families.argtypes = [_vp, _i64p, _i64p, _i32p, _i32p, _i32p, _i64p, _i32p, _i32p]
        L.mhc_plan_sinks.argtypes = [_vp, _i64p, _i32p, _i32p, _i32p, _i32p, _i32p]
        L.mhc_correlator.argtypes = [_vp, ctypes.POINTER(_vp), _vp, _vp, _vp, _vp]
        L.mhc_correlator_noalloc.argtypes = [_vp, ctypes.POINTER(_vp), _vp, _vp, _vp, _vp]
        L.mhc_correlator_backward.argtypes = [_vp, ctypes.POINTER(_vp), _vp, _vp, _vp,
                                              ctypes.POINTER(_vp), _vp, _vp, _vp]
        L.mhc_pair_dets.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
        L.mhc_get_status.argtypes = [_vp, _vp]
        L.mhc_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(_vp)]
        L.mhc_batch_destroy.argtypes = [_vp]
        L.mhc_batch_destroy.restype = None
        L.mhc_batch_correlator.argtypes = [_vp, ctypes.POINTER(ctypes.POINTER(_vp)), ctypes.POINTER(_vp), _vp]
        L.mhc_batch_info.argtypes = [_vp, _i32p, _i32p]
        L.mhc_batch_shape.argtypes = [_vp, _i32p, _i32p, _f64p]
        L.mhc_tune_cache_get.argtypes = [ctypes.c_char_p, _i32p]
        L.mhc_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_int32]
        L.mhc_fp64_peak.argtypes = [ctypes.c_int32, _f64p, _vp]
        L.mhc_complex_reciprocal.argtypes = [ctypes.c_int64, _vp, _vp, _vp]
        for name in EXPORTED:
            if name not in ("mhc_last_error", "mhc_plan_opts_default", "mhc_plan_destroy",
                            "mhc_batch_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status):
    if status != MHC_OK:
        raise MHCError(status, lib().mhc_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _S_ptrs(S: Sequence):
    import torch
    arr = (_vp * max(len(S), 1))()
    for f, s in enumerate(S):
        if s is None:
            arr[f] = None
            continue
        assert isinstance(s, torch.Tensor) and s.is_cuda and s.dtype == torch.complex128, \
            "S_f must be complex128 CUDA tensors"
        assert s.is_contiguous() and s.dim() == 2 and s.shape[0] == s.shape[1]
        arr[f] = s.data_ptr()
    return arr


def default_opts() -> PlanOpts:
    o = PlanOpts()
    lib().mhc_plan_opts_default(ctypes.byref(o))
    return o


# ------------------------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ------------------------------------------------------------------------------------------
def mhc_plan(n_f, L_f, labels_src, w_src, labels_snk, w_snk, opts: Optional[PlanOpts] = None):
    """Build a plan on the host; returns the opaque handle (an int)."""
    n_f = _np(n_f, np.int32)
    L_f = _np(L_f, np.int32)
    ls = _np(labels_src, np.int32)
    lk = _np(labels_snk, np.int32)
    ws = _np(w_src, np.float64)
    wk = _np(w_snk, np.float64)
    h = _vp()
    _check(lib().mhc_plan(ctypes.byref(h), len(n_f), n_f.ctypes.data_as(_i32p), L_f.ctypes.data_as(_i32p),
                          ws.shape[0], ls.ctypes.data_as(_i32p), ws.ctypes.data_as(_f64p), wk.shape[0],
                          lk.ctypes.data_as(_i32p), wk.ctypes.data_as(_f64p),
                          ctypes.byref(opts) if opts is not None else None))
    return h.value


def mhc_plan_destroy(plan):
    lib().mhc_plan_destroy(_vp(plan))


def mhc_plan_stats(plan) -> dict:
    s = Stats()
    _check(lib().mhc_plan_stats(_vp(plan), ctypes.byref(s)))
    return s.as_dict()


def mhc_plan_families(plan, F: int, Tn: int, n_src: int) -> dict:
    nW = ctypes.c_int64()
    L = lib()
    _check(L.mhc_plan_families(_vp(plan), ctypes.byref(nW), None, None, None, None, None, None, None))
    W = nW.value
    off = np.zeros(W + 1, np.int64)
    rank = np.zeros((W, F), np.int32)
    rows = np.zeros((W, F, MHC_MAX_RANK), np.int32)
    ref = np.zeros((W, Tn), np.int32)
    term = np.zeros(n_src, np.int64)
    sign = np.zeros(n_src, np.int32)
    labs = np.zeros((n_src, F, MHC_MAX_RANK), np.int32)
    _check(L.mhc_plan_families(_vp(plan), ctypes.byref(nW), off.ctypes.data_as(_i64p), rank.ctypes.data_as(_i32p),
                               rows.ctypes.data_as(_i32p), ref.ctypes.data_as(_i32p), term.ctypes.data_as(_i64p),
                               sign.ctypes.data_as(_i32p), labs.ctypes.data_as(_i32p)))
    return {"offset": off, "rank": rank, "rows": rows, "ref": ref, "term": term, "sign": sign,
            "labels": labs}


def mhc_plan_sinks(plan, Tn: int, n_snk: int) -> dict:
    nQ = ctypes.c_int64()
    L = lib()
    _check(L.mhc_plan_sinks(_vp(plan), ctypes.byref(nQ), None, None, None, None, None))
    order = np.zeros(n_snk, np.int32)
    labels = np.zeros((n_snk, Tn), np.int32)
    parity = np.zeros(n_snk, np.int32)
    family = np.zeros(n_snk, np.int32)
    two = np.zeros(nQ.value, np.int32)
    _check(L.mhc_plan_sinks(_vp(plan), ctypes.byref(nQ), order.ctypes.data_as(_i32p), labels.ctypes.data_as(_i32p),
                            parity.ctypes.data_as(_i32p), family.ctypes.data_as(_i32p), two.ctypes.data_as(_i32p)))
    return {"order": order, "labels": labels, "parity": parity, "family": family, "two_sided": two}


def mhc_correlator(plan, S, w_src=None, w_snk=None, out=None, stream=None):
    """Forward correlator; returns out (float64 CUDA tensor [2]: Re C, Im C)."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=S[0].device)
    _check(lib().mhc_correlator(_vp(plan), _S_ptrs(S), _ptr(w_src), _ptr(w_snk), _ptr(out), _stream(stream)))
    return out


def mhc_correlator_cw(plan, S, w_src, w_snk, out=None, stream=None):
    """Forward correlator with complex weights: w_src, w_snk complex128 CUDA tensors (their
    real and imaginary parts are passed as separate float64 arrays).  Returns out."""
    import torch
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=S[0].device)
    parts = [torch.view_as_real(w)[:, k].contiguous() for w in (w_src, w_snk) for k in (0, 1)]
    _check(lib().mhc_correlator_cw(_vp(plan), _S_ptrs(S), _ptr(parts[0]), _ptr(parts[1]), _ptr(parts[2]),
                                   _ptr(parts[3]), _ptr(out), _stream(stream)))
    return out


def mhc_correlator_noalloc(plan, S, out, w_src=None, w_snk=None, stream=None):
    """Forward correlator that allocates nothing during the call (for callers whose device
    memory is reserved by their own allocator, or who cannot afford an allocation in the
    loop).  `out` must be given (float64 CUDA tensor [2]).  The plan must have been used
    once by mhc_correlator on this device; see include/mhc.h for the scratch limits."""
    _check(lib().mhc_correlator_noalloc(_vp(plan), _S_ptrs(S), _ptr(w_src), _ptr(w_snk), _ptr(out),
                                        _stream(stream)))
    return out


def mhc_correlator_backward(plan, S, g_out, w_src=None, w_snk=None, dS=None, dw_src=None,
                            dw_snk=None, stream=None):
    """Adjoint; writes dS (list of complex128 tensors or None), dw_src, dw_snk."""
    arr = (_vp * max(len(S), 1))()
    if dS is not None:
        for f, t in enumerate(dS):
            arr[f] = None if t is None else t.data_ptr()
    _check(lib().mhc_correlator_backward(_vp(plan), _S_ptrs(S), _ptr(w_src), _ptr(w_snk), _ptr(g_out),
                                         arr if dS is not None else None, _ptr(dw_src), _ptr(dw_snk),
                                         _stream(stream)))


def mhc_pair_dets(plan, S, i_idx, j_idx, dets=None, path=None, stream=None):
    """Per-pair, per-flavour determinants: returns complex128 CUDA tensor [n_pairs, F]."""
    import torch
    n = int(i_idx.numel())
    F = len(S)
    if dets is None:
        dets = torch.empty((n, F), dtype=torch.complex128, device=i_idx.device)
    _check(lib().mhc_pair_dets(_vp(plan), _S_ptrs(S), n, _ptr(i_idx), _ptr(j_idx), _ptr(dets), _ptr(path),
                               _stream(stream)))
    return dets


def mhc_get_status(plan, stream=None):
    """Synchronise, read and clear the device status; raises on an error status."""
    _check(lib().mhc_get_status(_vp(plan), _stream(stream)))


def mhc_get_status_code(plan, stream=None) -> int:
    return int(lib().mhc_get_status(_vp(plan), _stream(stream)))


def mhc_batch_create(plans):
    arr = (_vp * len(plans))(*plans)
    h = _vp()
    _check(lib().mhc_batch_create(ctypes.byref(h), len(plans), arr))
    return h.value


def mhc_batch_destroy(batch):
    lib().mhc_batch_destroy(_vp(batch))


def mhc_batch_correlator(batch, S_list, outs, stream=None):
    n = len(S_list)
    inner = [_S_ptrs(S) for S in S_list]
    arr = (ctypes.POINTER(_vp) * n)(*[ctypes.cast(a, ctypes.POINTER(_vp)) for a in inner])
    o = (_vp * n)(*[t.data_ptr() for t in outs])
    _check(lib().mhc_batch_correlator(_vp(batch), arr, o, _stream(stream)))
    return outs


def mhc_batch_info(batch):
    t = ctypes.c_int32()
    n = ctypes.c_int32()
    _check(lib().mhc_batch_info(_vp(batch), ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


def mhc_batch_shape(batch):
    """Per n class (n_f <= 8, <= 18, <= 32): chosen sink tiles, whether each came from the
    tuning cache, and the timed candidates (ms at tiles 32, 64, 128)."""
    tiles = (ctypes.c_int32 * 3)()
    cached = (ctypes.c_int32 * 3)()
    ms = (ctypes.c_double * 9)()
    _check(lib().mhc_batch_shape(_vp(batch), tiles, cached, ms))
    return list(tiles), list(cached), [list(ms[3 * c:3 * c + 3]) for c in range(3)]


def mhc_tune_cache_get(key: str) -> int:
    t = ctypes.c_int32()
    _check(lib().mhc_tune_cache_get(key.encode(), ctypes.byref(t)))
    return t.value


def mhc_tune_cache_put(key: str, tile: int) -> None:
    _check(lib().mhc_tune_cache_put(key.encode(), tile))


def mhc_fp64_peak(iters: int = 200000, stream=None) -> float:
    f = ctypes.c_double()
    _check(lib().mhc_fp64_peak(iters, ctypes.byref(f), _stream(stream)))
    return f.value


def mhc_complex_reciprocal(z, out=None, stream=None):
    """1/z elementwise by the library's device reciprocal (z: complex128 CUDA tensor)."""
    import torch
    z = z.contiguous()
    if out is None:
        out = torch.empty_like(z)
    _check(lib().mhc_complex_reciprocal(z.numel(), _ptr(z), _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------------------------------
# Convenience wrapper and autograd
# ------------------------------------------------------------------------------------------
class Plan:
    """Owns one plan handle.  Inputs as numpy arrays (see mhc_plan)."""

    def __init__(self, n_f, L_f, labels_src, w_src, labels_snk, w_snk, opts: Optional[PlanOpts] = None):
        self.n_f = [int(x) for x in n_f]
        self.L_f = [int(x) for x in L_f]
        self.F = len(self.n_f)
        self.Tn = sum(self.n_f)
        self.n_src = int(np.asarray(w_src).shape[0])
        self.n_snk = int(np.asarray(w_snk).shape[0])
        self.handle = mhc_plan(n_f, L_f, labels_src, w_src, labels_snk, w_snk, opts)

    @classmethod
    def from_workload(cls, w, opts=None):
        return cls(w.n_f, w.L_f, w.labels_src, w.w_src, w.labels_snk, w.w_snk, opts)

    def stats(self):
        return mhc_plan_stats(self.handle)

    def families(self):
        return mhc_plan_families(self.handle, self.F, self.Tn, self.n_src)

    def sinks(self):
        return mhc_plan_sinks(self.handle, self.Tn, self.n_snk)

    def correlator(self, S, w_src=None, w_snk=None, out=None, stream=None):
        return mhc_correlator(self.handle, S, w_src, w_snk, out, stream)

    def pair_dets(self, S, i_idx, j_idx, path=None, stream=None):
        return mhc_pair_dets(self.handle, S, i_idx, j_idx, None, path, stream)

    def status(self, stream=None):
        mhc_get_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            mhc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class CorrelatorFn(torch.autograd.Function):
        """C(S_1..S_F, w_src, w_snk) as a complex scalar with the hand-written adjoint."""

        @staticmethod
        def forward(ctx, plan, w_src, w_snk, *S):
            out = mhc_correlator(plan.handle, list(S), w_src.contiguous(), w_snk.contiguous())
            ctx.plan = plan
            ctx.save_for_backward(w_src, w_snk, *S)
            return torch.complex(out[0], out[1])

        @staticmethod
        def backward(ctx, g):
            w_src, w_snk, *S = ctx.saved_tensors
            plan = ctx.plan
            g_out = torch.stack([g.real, g.imag]).to(torch.float64).contiguous()
            need_S = ctx.needs_input_grad[3:]
            dS = [torch.empty_like(s) if need else None for s, need in zip(S, need_S)]
            dws = torch.empty_like(w_src) if ctx.needs_input_grad[1] else None
            dwk = torch.empty_like(w_snk) if ctx.needs_input_grad[2] else None
            mhc_correlator_backward(plan.handle, list(S), g_out, w_src.contiguous(), w_snk.contiguous(),
                                    dS, dws, dwk)
            return (None, dws, dwk, *dS)

    return CorrelatorFn


_Fn = None


def correlator(plan: Plan, S, w_src, w_snk):
    """Differentiable correlator: complex128 scalar tensor; gradients flow to S_f, w_src, w_snk."""
    global _Fn
    if _Fn is None:
        _Fn = _autograd()
    return _Fn.apply(plan, w_src, w_snk, *S)
