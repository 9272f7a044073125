"""GB300 (sm_103a) solver for group-sparse regularised optimal transport.

Python binding of ``libotgs.so`` (C ABI in ``include/otgs.h``).  This module
only marshals arguments: tensors are PyTorch CUDA tensors whose device
pointers and the current CUDA stream are passed to the library, where every
step of the computation runs in the package's own CUDA kernels.  There is no
CPU fallback: when the library has not been built, every entry point raises.

Functions keep the ABI's names (``ot_gs_create``, ``ot_gs_grad``, ...); the
:class:`GroupSparseOT` class bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libotgs.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "otgs.h")

OTGS_OK, OTGS_EINVAL, OTGS_ECUDA, OTGS_ENOMEM = 0, -1, -2, -3
OTGS_ENOTCONV, OTGS_ETIMEOUT, OTGS_ELINESEARCH, OTGS_ENONFINITE = -4, -5, -6, -7
STATUS_NAMES = {0: "OTGS_OK", -1: "OTGS_EINVAL", -2: "OTGS_ECUDA", -3: "OTGS_ENOMEM",
                -4: "OTGS_ENOTCONV", -5: "OTGS_ETIMEOUT", -6: "OTGS_ELINESEARCH",
                -7: "OTGS_ENONFINITE"}


class OTGSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("r", ctypes.c_int32),
                ("lbfgs_m", ctypes.c_int32), ("use_screening", ctypes.c_int32),
                ("use_lower_bound", ctypes.c_int32), ("time_budget_ms", ctypes.c_double),
                ("ftol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("iters", ctypes.c_int64),
                ("blocks_total", ctypes.c_int64), ("blocks_in_N", ctypes.c_int64),
                ("blocks_skipped", ctypes.c_int64), ("blocks_checked", ctypes.c_int64),
                ("units_total", ctypes.c_int64), ("units_computed", ctypes.c_int64),
                ("snapshots", ctypes.c_int64), ("c_bytes", ctypes.c_double),
                ("kernels", ctypes.c_int64), ("blocks_flagged", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded ``libotgs.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "ot_gs_create": ([ctypes.POINTER(P), P, i64, P, P, P, i64, i64, i32, dbl, dbl, P], ctypes.c_int),
        "ot_gs_create_shard": ([ctypes.POINTER(P), P, i64, P, P, P, i64, i64, i32, dbl, dbl, P], ctypes.c_int),
        "ot_gs_destroy": ([P], ctypes.c_int),
        "ot_gs_set_stream": ([P, P], ctypes.c_int),
        "ot_gs_set_params": ([P, ctypes.POINTER(Params)], ctypes.c_int),
        "ot_gs_get_params": ([P, ctypes.POINTER(Params)], ctypes.c_int),
        "ot_gs_grad": ([P, P, P, P], ctypes.c_int),
        "ot_gs_grad_screened": ([P, P, P, P, P], ctypes.c_int),
        "ot_gs_snapshot": ([P, P, P, ctypes.c_int, P], ctypes.c_int),
        "ot_gs_get_screen_state": ([P, P, P, P, P, P], ctypes.c_int),
        "ot_gs_solve": ([P, dbl, i32], ctypes.c_int),
        "ot_gs_get_solution": ([P, P, P, P, P, P], ctypes.c_int),
        "ot_gs_set_state": ([P, P, P], ctypes.c_int),
        "ot_gs_get_trace": ([P, P, P, P, i32, P], ctypes.c_int),
        "ot_gs_get_stats": ([P, ctypes.POINTER(Stats)], ctypes.c_int),
        "ot_gs_state_size": ([P, P], ctypes.c_int),
        "ot_gs_get_state": ([P, P, i64], ctypes.c_int),
        "ot_gs_restore_state": ([P, P, i64], ctypes.c_int),
        "ot_gs_reset_stats": ([P], ctypes.c_int),
        "ot_gs_set_timing": ([P, ctypes.c_int], ctypes.c_int),
        "ot_gs_debug": ([P, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
        "ot_gs_get_timing": ([P, P, P], ctypes.c_int),
        "ot_gs_last_error": ([P], ctypes.c_char_p),
        "ot_gs_version": ([], ctypes.c_char_p),
        "ot_gs_plan_info": ([P, i64, i64, i32, P, P, P], ctypes.c_int),
        "ot_gs_grad_noalloc": ([P, i64, P, P, P, i64, i64, i32, dbl, dbl, P, P, P, P], ctypes.c_int),
        "ot_gs_noalloc_last_error": ([], ctypes.c_char_p),
        "ot_gs_plan": ([P, P, P, P, i64], ctypes.c_int),
        "ot_gs_barycentric": ([P, P, P, P, i32, P], ctypes.c_int),
        "ot_gs_create_batch": ([ctypes.POINTER(P), i32, P, P, P, P, P, P, P, P, dbl, dbl, P], ctypes.c_int),
        "ot_gs_batch_size": ([P, P, P, P], ctypes.c_int),
        "ot_gs_batch_grad": ([P, P, P, P, P], ctypes.c_int),
        "ot_gs_batch_solve": ([P, dbl, i32, P, dbl], ctypes.c_int),
        "ot_gs_batch_set_state": ([P, P, P], ctypes.c_int),
        "ot_gs_batch_shift": ([P, P, P, i32], ctypes.c_int),
        "ot_gs_batch_result": ([P, P, P, P, P, P, P, P, P], ctypes.c_int),
        "ot_gs_set_plan": ([P, i32, i32, i32], ctypes.c_int),
        "ot_gs_get_plan": ([P, P, P, P, P], ctypes.c_int),
        "ot_gs_autotune": ([P, P, P, i32, P, P, P, P], ctypes.c_int),
        "ot_gs_autotune_clear_cache": ([], ctypes.c_int),
        "ot_gs_plan_info_batch": ([i32, P, P, P, P, i32, i32, i32, P, P, P], ctypes.c_int),
        "ot_gs_mlp_create": ([ctypes.POINTER(P), i32, i32, i64, ctypes.c_uint64, P], ctypes.c_int),
        "ot_gs_mlp_destroy": ([P], ctypes.c_int),
        "ot_gs_mlp_num_params": ([P, P], ctypes.c_int),
        "ot_gs_mlp_set_params": ([P, P], ctypes.c_int),
        "ot_gs_mlp_get_params": ([P, P], ctypes.c_int),
        "ot_gs_mlp_forward": ([P, P, i64, P], ctypes.c_int),
        "ot_gs_mlp_grad": ([P, P, P, i64, P, P], ctypes.c_int),
        "ot_gs_mlp_adam": ([P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float], ctypes.c_int),
        "ot_gs_mlp_features": ([P, i64, i64, i64, P, P, i32, P, i32, ctypes.c_float, i32, P, P], ctypes.c_int),
        "ot_gs_mlp_last_error": ([P], ctypes.c_char_p),
        "ot_gs_mlp_features_batch": ([i32, P, P, P, P, P, P, i32, P, P, ctypes.c_float, i32, P, P], ctypes.c_int),
        "ot_gs_mlp_refine_features": ([i32, P, P, P, P, P, P, ctypes.c_float, i32, i32, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def header_symbols(path: str = HEADER):
    """Names of the functions declared in include/otgs.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_gs_\w+)\s*\(", txt)))


# ----------------------------------------------------------------- helpers
def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, numel=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _check(h, rc):
    if rc != OTGS_OK and rc not in (OTGS_ENOTCONV, OTGS_ETIMEOUT, OTGS_ELINESEARCH):
        msg = lib().ot_gs_last_error(h)
        raise OTGSError(rc, msg.decode() if msg else "")
    return rc


def rho_to_gamma_mu(gamma: float, rho: float):
    """The rho form used in the experiments (Sec. 5.2),
    gamma (1/2 (1 - rho) ||t||^2 + rho sum_l ||t_[l]||), is Eq. 3 with
    gamma' = gamma (1 - rho) and mu' = rho / (1 - rho)."""
    if not 0.0 <= rho < 1.0:
        raise ValueError("rho must be in [0, 1)")
    return gamma * (1.0 - rho), rho / (1.0 - rho)


# ---------------------------------------------------------- ABI wrappers
def ot_gs_create(C, a, b, labels, L, gamma, mu, stream=None, shard=False):
    """C: (m, n) float32 CUDA (row stride C.stride(0)); a (m,), b (n,) float64;
    labels (m,) int32 in [0, L).  shard: C and b are a column shard of a
    larger problem (ot_gs_create_shard).  Returns the raw handle (ctypes.c_void_p)."""
    import torch
    if C.dim() != 2 or C.stride(1) != 1:
        raise ValueError("C must be 2-D with unit column stride")
    m, n = C.shape
    h = ctypes.c_void_p()
    fn = lib().ot_gs_create_shard if shard else lib().ot_gs_create
    rc = fn(ctypes.byref(h), _ptr(C, torch.float32, name="C") if C.is_contiguous()
                            else ctypes.c_void_p(C.data_ptr()), C.stride(0),
                            _ptr(a, torch.float64, m, "a"), _ptr(b, torch.float64, n, "b"),
                            _ptr(labels, torch.int32, m, "labels"), m, n, int(L), float(gamma),
                            float(mu), _stream_ptr(stream))
    if rc != OTGS_OK:
        raise OTGSError(rc, lib().ot_gs_last_error(None).decode())
    return h


def ot_gs_destroy(h):
    return lib().ot_gs_destroy(h)


def ot_gs_set_stream(h, stream=None):
    return _check(h, lib().ot_gs_set_stream(h, _stream_ptr(stream)))


def ot_gs_set_params(h, params: Params):
    return _check(h, lib().ot_gs_set_params(h, ctypes.byref(params)))


def ot_gs_get_params(h) -> Params:
    p = Params()
    _check(h, lib().ot_gs_get_params(h, ctypes.byref(p)))
    return p


def ot_gs_grad(h, alpha, beta, out):
    import torch
    return _check(h, lib().ot_gs_grad(h, _ptr(alpha, torch.float64, name="alpha"),
                                      _ptr(beta, torch.float64, name="beta"),
                                      _ptr(out, torch.float64, name="out")))


def ot_gs_grad_screened(h, alpha, beta, out, skip_mask=None):
    import torch
    return _check(h, lib().ot_gs_grad_screened(
        h, _ptr(alpha, torch.float64, name="alpha"), _ptr(beta, torch.float64, name="beta"),
        _ptr(out, torch.float64, name="out"), _ptr(skip_mask, torch.int32, name="skip_mask")))


def ot_gs_snapshot(h, alpha, beta, build_N, out=None):
    import torch
    return _check(h, lib().ot_gs_snapshot(h, _ptr(alpha, torch.float64, name="alpha"),
                                          _ptr(beta, torch.float64, name="beta"), int(build_N),
                                          _ptr(out, torch.float64, name="out")))


def ot_gs_get_screen_state(h, zt=None, ot=None, alpha_s=None, beta_s=None, N_mask=None):
    import torch
    return _check(h, lib().ot_gs_get_screen_state(
        h, _ptr(zt, torch.float32, name="zt"), _ptr(ot, torch.float32, name="ot"),
        _ptr(alpha_s, torch.float64, name="alpha_s"), _ptr(beta_s, torch.float64, name="beta_s"),
        _ptr(N_mask, torch.int32, name="N_mask")))


def ot_gs_solve(h, tol, maxit):
    return _check(h, lib().ot_gs_solve(h, float(tol), int(maxit)))


def ot_gs_get_solution(h, alpha, beta):
    import torch
    D, gi, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(h, lib().ot_gs_get_solution(h, _ptr(alpha, torch.float64, name="alpha"),
                                       _ptr(beta, torch.float64, name="beta"), ctypes.byref(D),
                                       ctypes.byref(gi), ctypes.byref(it)))
    return D.value, gi.value, it.value


def ot_gs_get_trace(h):
    """Objective trace of the last solve: (D, t_ms, evals) numpy arrays, entry
    0 the start point and entry k the k-th accepted iteration; t_ms is device
    time since the solve was launched."""
    cnt = ctypes.c_int32()
    _check(h, lib().ot_gs_get_trace(h, None, None, None, 0, ctypes.byref(cnt)))
    k = cnt.value
    D, t, ev = np.empty(k), np.empty(k), np.empty(k, dtype=np.int64)
    if k:
        _check(h, lib().ot_gs_get_trace(h, D.ctypes.data_as(ctypes.c_void_p), t.ctypes.data_as(ctypes.c_void_p),
                                        ev.ctypes.data_as(ctypes.c_void_p), k, ctypes.byref(cnt)))
    return D, t, ev


def ot_gs_set_state(h, alpha, beta):
    import torch
    return _check(h, lib().ot_gs_set_state(h, _ptr(alpha, torch.float64, name="alpha"),
                                           _ptr(beta, torch.float64, name="beta")))


def ot_gs_state_size(h) -> int:
    n = ctypes.c_int64()
    _check(h, lib().ot_gs_state_size(h, ctypes.byref(n)))
    return n.value


def ot_gs_get_state(h, buf):
    """Copies the solver state into buf (a CUDA uint8 tensor of at least
    ot_gs_state_size(h) bytes)."""
    import torch
    _ptr(buf, torch.uint8, name="buf")
    return _check(h, lib().ot_gs_get_state(h, ctypes.c_void_p(buf.data_ptr()), buf.numel()))


def ot_gs_restore_state(h, buf):
    import torch
    _ptr(buf, torch.uint8, name="buf")
    return _check(h, lib().ot_gs_restore_state(h, ctypes.c_void_p(buf.data_ptr()), buf.numel()))


def ot_gs_get_stats(h) -> dict:
    s = Stats()
    _check(h, lib().ot_gs_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def ot_gs_reset_stats(h):
    return _check(h, lib().ot_gs_reset_stats(h))


OTGS_DEBUG_STALL = 2
OTGS_DEBUG_NAN_EVAL = 3
OTGS_DEBUG_SCREEN_ROUTE = 4


def ot_gs_debug(h, what: int, value: int):
    """Test hooks of later evaluations (see include/otgs.h)."""
    return _check(h, lib().ot_gs_debug(h, ctypes.c_int(what), ctypes.c_int64(value)))


def ot_gs_set_timing(h, enable: bool):
    return _check(h, lib().ot_gs_set_timing(h, int(bool(enable))))


def ot_gs_get_timing(h):
    """(launches, total_ms) of the evaluation kernel since the last call."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(h, lib().ot_gs_get_timing(h, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def ot_gs_last_error(h=None) -> str:
    return lib().ot_gs_last_error(h).decode()


def ot_gs_version() -> str:
    return lib().ot_gs_version().decode()


def ot_gs_plan_info(labels, n, L):
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    np_, ni, rl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib().ot_gs_plan_info(lab.ctypes.data_as(ctypes.c_void_p), len(lab), int(n), int(L),
                               ctypes.byref(np_), ctypes.byref(ni), ctypes.byref(rl))
    if rc != OTGS_OK:
        raise OTGSError(rc, "invalid plan input")
    return dict(n_panels=np_.value, n_items=ni.value, n_stages=rl.value)


def ot_gs_grad_noalloc(C, a, b, labels_host, L, gamma, mu, alpha, beta, out, stream=None):
    """Dense evaluation without a handle and without any device allocation
    (for callers that cannot allocate); labels_host is a host int32 array of
    non-decreasing labels.  Raises OTGSError on a non-zero status."""
    import torch
    if not isinstance(C, torch.Tensor) or not C.is_cuda or C.dtype != torch.float32:
        raise TypeError("C must be a float32 CUDA tensor")
    if C.dim() != 2 or C.stride(1) != 1:
        raise ValueError("C must be 2-D with unit column stride")
    m, n = C.shape
    lab = np.ascontiguousarray(labels_host, dtype=np.int32)
    if lab.shape != (m,):
        raise ValueError("labels_host must have m entries")
    rc = lib().ot_gs_grad_noalloc(ctypes.c_void_p(C.data_ptr()), C.stride(0),
                                  _ptr(a, torch.float64, m, "a"), _ptr(b, torch.float64, n, "b"),
                                  lab.ctypes.data_as(ctypes.c_void_p), m, n, int(L), float(gamma),
                                  float(mu), _ptr(alpha, torch.float64, m, "alpha"),
                                  _ptr(beta, torch.float64, n, "beta"),
                                  _ptr(out, torch.float64, 1 + m + n, "out"), _stream_ptr(stream))
    if rc != OTGS_OK:
        raise OTGSError(rc, lib().ot_gs_noalloc_last_error().decode())
    return rc


def _host_array(vals, ctype):
    arr = (ctype * len(vals))(*vals)
    return arr, ctypes.cast(arr, ctypes.c_void_p)


def ot_gs_create_batch(Cs, As, Bs, labels, Ls, gamma, mu, stream=None):
    """Batch of independent problems: lists of CUDA tensors C_k (m_k, n_k)
    float32 (unit column stride), a_k, b_k float64, labels_k int32, and class
    counts L_k.  Returns the raw handle."""
    import torch
    k = len(Cs)
    if not (len(As) == len(Bs) == len(labels) == len(Ls) == k) or k == 0:
        raise ValueError("need equally long, non-empty lists")
    cp, lp, ap, bp, lab, ms, ns = [], [], [], [], [], [], []
    for q in range(k):
        C = Cs[q]
        if C.dim() != 2 or C.stride(1) != 1 or C.dtype != torch.float32 or not C.is_cuda:
            raise ValueError(f"C[{q}] must be a 2-D float32 CUDA tensor with unit column stride")
        m, n = C.shape
        cp.append(C.data_ptr())
        lp.append(C.stride(0))
        ap.append(_ptr(As[q], torch.float64, m, f"a[{q}]").value)
        bp.append(_ptr(Bs[q], torch.float64, n, f"b[{q}]").value)
        lab.append(_ptr(labels[q], torch.int32, m, f"labels[{q}]").value)
        ms.append(m)
        ns.append(n)
    keep = [_host_array(cp, ctypes.c_void_p), _host_array(lp, ctypes.c_int64), _host_array(ap, ctypes.c_void_p),
            _host_array(bp, ctypes.c_void_p), _host_array(lab, ctypes.c_void_p), _host_array(ms, ctypes.c_int64),
            _host_array(ns, ctypes.c_int64), _host_array([int(x) for x in Ls], ctypes.c_int32)]
    h = ctypes.c_void_p()
    rc = lib().ot_gs_create_batch(ctypes.byref(h), k, *[p for _, p in keep], float(gamma), float(mu),
                                  _stream_ptr(stream))
    if rc != OTGS_OK:
        raise OTGSError(rc, lib().ot_gs_last_error(None).decode())
    return h


def ot_gs_batch_size(h):
    k, m, n = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(h, lib().ot_gs_batch_size(h, ctypes.byref(k), ctypes.byref(m), ctypes.byref(n)))
    return k.value, m.value, n.value


def ot_gs_batch_grad(h, alpha, beta, D, grad=None):
    import torch
    return _check(h, lib().ot_gs_batch_grad(h, _ptr(alpha, torch.float64, name="alpha"),
                                            _ptr(beta, torch.float64, name="beta"),
                                            _ptr(D, torch.float64, name="D"),
                                            _ptr(grad, torch.float64, name="grad")))


def ot_gs_batch_solve(h, tol, maxit, target_D=None, target_rtol=0.0):
    tgt = None
    if target_D is not None:
        tgt = np.ascontiguousarray(target_D, dtype=np.float64)
    return _check(h, lib().ot_gs_batch_solve(h, float(tol), int(maxit),
                                             None if tgt is None else tgt.ctypes.data_as(ctypes.c_void_p),
                                             float(target_rtol)))


def ot_gs_batch_set_state(h, alpha, beta):
    import torch
    return _check(h, lib().ot_gs_batch_set_state(h, _ptr(alpha, torch.float64, name="alpha"),
                                                 _ptr(beta, torch.float64, name="beta")))


def ot_gs_batch_shift(h, alpha, beta, iters=40):
    import torch
    return _check(h, lib().ot_gs_batch_shift(h, _ptr(alpha, torch.float64, name="alpha"),
                                             _ptr(beta, torch.float64, name="beta"), int(iters)))


def ot_gs_batch_result(h, nprob, alpha=None, beta=None):
    """Per-problem results of the last batch solve as numpy arrays (and the
    iterate into alpha, beta when given)."""
    import torch
    D, gi, t = np.empty(nprob), np.empty(nprob), np.empty(nprob)
    it, stt = np.empty(nprob, dtype=np.int32), np.empty(nprob, dtype=np.int32)
    ev = np.empty(nprob, dtype=np.int64)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(h, lib().ot_gs_batch_result(h, _ptr(alpha, torch.float64, name="alpha"),
                                       _ptr(beta, torch.float64, name="beta"), vp(D), vp(gi), vp(it), vp(stt),
                                       vp(ev), vp(t)))
    return dict(D=D, grad_inf=gi, iters=it, status=stt, evals=ev, t_ms=t)


def ot_gs_set_plan(h, panel_rows=0, split_rows=0, stage_fill=0):
    return _check(h, lib().ot_gs_set_plan(h, int(panel_rows), int(split_rows), int(stage_fill)))


def ot_gs_get_plan(h):
    pr, sr, sf, ni = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(h, lib().ot_gs_get_plan(h, ctypes.byref(pr), ctypes.byref(sr), ctypes.byref(sf), ctypes.byref(ni)))
    return dict(panel_rows=pr.value, split_rows=sr.value, stage_fill=sf.value, n_items=ni.value)


def ot_gs_autotune(h, alpha, beta, evals=5):
    import torch
    pr, sr, sf, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(h, lib().ot_gs_autotune(h, _ptr(alpha, torch.float64, name="alpha"),
                                   _ptr(beta, torch.float64, name="beta"), int(evals), ctypes.byref(pr),
                                   ctypes.byref(sr), ctypes.byref(sf), ctypes.byref(ms)))
    return dict(panel_rows=pr.value, split_rows=sr.value, stage_fill=sf.value, best_ms=ms.value)


def ot_gs_autotune_clear_cache():
    return lib().ot_gs_autotune_clear_cache()


def ot_gs_plan_info_batch(labels_list, ns, Ls, panel_rows=0, split_rows=0, stage_fill=0):
    """Host-only plan of a batch: counts of panels, work items and stages."""
    k = len(labels_list)
    labs = [np.ascontiguousarray(x, dtype=np.int32) for x in labels_list]
    lp = _host_array([x.ctypes.data for x in labs], ctypes.c_void_p)
    mp = _host_array([len(x) for x in labs], ctypes.c_int64)
    npp = _host_array([int(x) for x in ns], ctypes.c_int64)
    Lp = _host_array([int(x) for x in Ls], ctypes.c_int32)
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib().ot_gs_plan_info_batch(k, lp[1], mp[1], npp[1], Lp[1], int(panel_rows), int(split_rows),
                                     int(stage_fill), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc != OTGS_OK:
        raise OTGSError(rc, "invalid plan input")
    return dict(n_panels=a.value, n_items=b.value, n_stages=c.value)


# ------------------------------------------------------------ convenience
class GroupSparseOT:
    """One problem on the current CUDA device.  Keeps references to the
    borrowed input tensors for the handle's lifetime."""

    def __init__(self, C, a, b, labels, L, gamma, mu, stream=None, shard=False):
        import torch
        self._keep = (C, a, b, labels)
        self.m, self.n = C.shape
        self.L = int(L)
        self.device = C.device
        self.h = ot_gs_create(C, a, b, labels, L, gamma, mu, stream, shard=shard)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            ot_gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> Params:
        return ot_gs_get_params(self.h)

    def set_params(self, **kw):
        p = ot_gs_get_params(self.h)
        for k, v in kw.items():
            setattr(p, k, v)
        ot_gs_set_params(self.h, p)

    def grad(self, alpha, beta, out=None):
        import torch
        if out is None:
            out = torch.empty(1 + self.m + self.n, dtype=torch.float64, device=self.device)
        ot_gs_grad(self.h, alpha, beta, out)
        return out

    def grad_screened(self, alpha, beta, out=None, skip_mask=None):
        import torch
        if out is None:
            out = torch.empty(1 + self.m + self.n, dtype=torch.float64, device=self.device)
        ot_gs_grad_screened(self.h, alpha, beta, out, skip_mask)
        return out

    def snapshot(self, alpha, beta, build_N=False, out=None):
        ot_gs_snapshot(self.h, alpha, beta, build_N, out)
        return out

    def solve(self, tol=1e-8, maxit=1000):
        return ot_gs_solve(self.h, tol, maxit)

    def solution(self):
        import torch
        al = torch.empty(self.m, dtype=torch.float64, device=self.device)
        be = torch.empty(self.n, dtype=torch.float64, device=self.device)
        D, ginf, it = ot_gs_get_solution(self.h, al, be)
        return dict(alpha=al, beta=be, D=D, grad_inf=ginf, iters=it)

    def set_state(self, alpha, beta):
        ot_gs_set_state(self.h, alpha, beta)

    def trace(self):
        return ot_gs_get_trace(self.h)

    def save_state(self):
        """The solver's full state (a CUDA uint8 tensor) for restore_state."""
        import torch
        buf = torch.empty(ot_gs_state_size(self.h), dtype=torch.uint8, device=self.device)
        ot_gs_get_state(self.h, buf)
        return buf

    def restore_state(self, buf):
        """Loads a saved state; the next solve continues it (maxit counts the
        whole solve's iterations)."""
        ot_gs_restore_state(self.h, buf)

    def plan(self, alpha, beta, out=None):
        """Transport plan t = grad psi at (alpha, beta): (m, n) FP32 (Sec. 2.3)."""
        import torch
        if out is None:
            out = torch.empty(self.m, self.n, dtype=torch.float32, device=self.device)
        _check(self.h, lib().ot_gs_plan(self.h, _ptr(alpha, torch.float64, self.m, "alpha"),
                                        _ptr(beta, torch.float64, self.n, "beta"),
                                        ctypes.c_void_p(out.data_ptr()), out.stride(0)))
        return out

    def barycentric(self, alpha, beta, XS):
        """n T^T X_S (Sec. 2.1): (n, d) FP32 images of the target samples."""
        import torch
        d = XS.shape[1]
        out = torch.empty(self.n, d, dtype=torch.float32, device=self.device)
        _check(self.h, lib().ot_gs_barycentric(self.h, _ptr(alpha, torch.float64, self.m, "alpha"),
                                               _ptr(beta, torch.float64, self.n, "beta"),
                                               _ptr(XS, torch.float32, self.m * d, "XS"), d,
                                               _ptr(out, torch.float32, self.n * d, "out")))
        return out

    def stats(self):
        return ot_gs_get_stats(self.h)


class GroupSparseOTBatch:
    """Independent problems solved together (one evaluation kernel for all,
    one L-BFGS state per problem).  Vectors use the concatenated layout:
    problem k's alpha at rows row_off[k]:row_off[k]+m_k, its beta at
    col_off[k]:col_off[k]+n_k."""

    def __init__(self, Cs, As, Bs, labels, Ls, gamma, mu, stream=None):
        self._keep = (list(Cs), list(As), list(Bs), list(labels))
        self.ms = [int(C.shape[0]) for C in Cs]
        self.ns = [int(C.shape[1]) for C in Cs]
        self.nprob = len(Cs)
        self.row_off = np.concatenate([[0], np.cumsum(self.ms)]).astype(np.int64)
        self.col_off = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        self.m, self.n = int(self.row_off[-1]), int(self.col_off[-1])
        self.device = Cs[0].device
        self.h = ot_gs_create_batch(Cs, As, Bs, labels, Ls, gamma, mu, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            ot_gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        p = ot_gs_get_params(self.h)
        for k, v in kw.items():
            setattr(p, k, v)
        ot_gs_set_params(self.h, p)

    def grad(self, alpha, beta, with_grad=True):
        import torch
        D = torch.empty(self.nprob, dtype=torch.float64, device=self.device)
        g = torch.empty(self.m + self.n, dtype=torch.float64, device=self.device) if with_grad else None
        ot_gs_batch_grad(self.h, alpha, beta, D, g)
        return D, g

    def solve(self, tol=1e-8, maxit=1000, target_D=None, target_rtol=0.0):
        return ot_gs_batch_solve(self.h, tol, maxit, target_D, target_rtol)

    def set_state(self, alpha, beta):
        ot_gs_batch_set_state(self.h, alpha, beta)

    def shift(self, alpha, beta, iters=40):
        """Best common shift of each problem's alpha, in place (see ot_gs_batch_shift)."""
        ot_gs_batch_shift(self.h, alpha, beta, iters)
        return alpha

    def result(self, with_iterate=True):
        import torch
        al = be = None
        if with_iterate:
            al = torch.empty(self.m, dtype=torch.float64, device=self.device)
            be = torch.empty(self.n, dtype=torch.float64, device=self.device)
        r = ot_gs_batch_result(self.h, self.nprob, al, be)
        if with_iterate:
            r["alpha"], r["beta"] = al, be
        return r

    def set_plan(self, panel_rows=0, split_rows=0, stage_fill=0):
        ot_gs_set_plan(self.h, panel_rows, split_rows, stage_fill)

    def plan(self):
        return ot_gs_get_plan(self.h)

    def autotune(self, alpha, beta, evals=5):
        return ot_gs_autotune(self.h, alpha, beta, evals)

    def split(self, vec, k, part):
        """Problem k's alpha (part 'alpha') or beta (part 'beta') of a
        concatenated vector; for a gradient vector the beta part starts at m."""
        if part == "alpha":
            return vec[self.row_off[k]:self.row_off[k + 1]]
        base = self.m if vec.numel() == self.m + self.n else 0
        return vec[base + self.col_off[k]:base + self.col_off[k + 1]]


# ------------------------------------------------------------ warm start
class MLPError(OTGSError):
    pass


def _mlp_check(h, rc):
    if rc != OTGS_OK:
        msg = lib().ot_gs_mlp_last_error(h)
        raise MLPError(rc, msg.decode() if msg else "")
    return rc


def mlp_features(C, XS, XT, labels, L, gamma, in_dim, out=None, stream=None):
    """Input features of one problem (device tensors): (m + n, in_dim) FP32,
    source rows then target columns (see ot_gs_mlp_features)."""
    import torch
    m, n = C.shape
    d = XS.shape[1]
    if C.stride(1) != 1 or C.dtype != torch.float32:
        raise ValueError("C must be float32 with unit column stride")
    if out is None:
        out = torch.empty(m + n, in_dim, dtype=torch.float32, device=C.device)
    rc = lib().ot_gs_mlp_features(ctypes.c_void_p(C.data_ptr()), C.stride(0), m, n,
                                  _ptr(XS, torch.float32, m * d, "XS"), _ptr(XT, torch.float32, n * d, "XT"),
                                  d, _ptr(labels, torch.int32, m, "labels"), int(L), float(gamma), int(in_dim),
                                  _ptr(out, torch.float32, (m + n) * in_dim, "out"), _stream_ptr(stream))
    _mlp_check(None, rc)
    return out


def mlp_features_batch(Cs, XSs, XTs, labels, Ls, gamma, in_dim, out=None, stream=None):
    """Features of many problems in one launch: rows of all source samples
    (concatenated), then of all target samples."""
    import torch
    k = len(Cs)
    d = XSs[0].shape[1]
    ms = [int(C.shape[0]) for C in Cs]
    ns = [int(C.shape[1]) for C in Cs]
    f32, i32 = torch.float32, torch.int32
    for q in range(k):  # (inline checks: this runs for every problem of a batch)
        C, xs, xt, lb = Cs[q], XSs[q], XTs[q], labels[q]
        if C.dtype != f32 or C.stride(1) != 1 or not C.is_cuda:
            raise ValueError(f"C[{q}] must be a CUDA float32 tensor with unit column stride")
        if xs.dtype != f32 or not xs.is_cuda or not xs.is_contiguous() or xs.numel() != ms[q] * d:
            raise ValueError(f"XS[{q}] must be a contiguous CUDA float32 tensor of {ms[q] * d} elements")
        if xt.dtype != f32 or not xt.is_cuda or not xt.is_contiguous() or xt.numel() != ns[q] * d:
            raise ValueError(f"XT[{q}] must be a contiguous CUDA float32 tensor of {ns[q] * d} elements")
        if lb.dtype != i32 or not lb.is_cuda or not lb.is_contiguous() or lb.numel() != ms[q]:
            raise ValueError(f"labels[{q}] must be a contiguous CUDA int32 tensor of {ms[q]} elements")
    if out is None:
        out = torch.empty(sum(ms) + sum(ns), in_dim, dtype=torch.float32, device=Cs[0].device)
    arrs = [_host_array([C.data_ptr() for C in Cs], ctypes.c_void_p),
            _host_array([C.stride(0) for C in Cs], ctypes.c_int64), _host_array(ms, ctypes.c_int64),
            _host_array(ns, ctypes.c_int64), _host_array([x.data_ptr() for x in XSs], ctypes.c_void_p),
            _host_array([x.data_ptr() for x in XTs], ctypes.c_void_p)]
    lp = _host_array([x.data_ptr() for x in labels], ctypes.c_void_p)
    Lp = _host_array([int(x) for x in Ls], ctypes.c_int32)
    rc = lib().ot_gs_mlp_features_batch(k, *[a[1] for a in arrs], d, lp[1], Lp[1], float(gamma), int(in_dim),
                                        _ptr(out, torch.float32, out.numel(), "out"), _stream_ptr(stream))
    _mlp_check(None, rc)
    return out


def mlp_refine_features(Cs, alpha_hat, beta_hat, gamma, col0, out, stream=None):
    """Second-pass inputs (see ot_gs_mlp_refine_features): columns [col0,
    col0 + 4) of out, the features of the problems Cs in the batch layout,
    from a first prediction alpha_hat (sum m) and beta_hat (sum n), FP32."""
    import torch
    ms = [int(C.shape[0]) for C in Cs]
    ns = [int(C.shape[1]) for C in Cs]
    for q, C in enumerate(Cs):
        if C.dtype != torch.float32 or C.stride(1) != 1 or not C.is_cuda:
            raise ValueError(f"C[{q}] must be a CUDA float32 tensor with unit column stride")
    M, N = sum(ms), sum(ns)
    if out.dim() != 2 or out.shape[0] != M + N:
        raise ValueError(f"out must have {M + N} rows")
    arrs = [_host_array([C.data_ptr() for C in Cs], ctypes.c_void_p),
            _host_array([C.stride(0) for C in Cs], ctypes.c_int64), _host_array(ms, ctypes.c_int64),
            _host_array(ns, ctypes.c_int64)]
    rc = lib().ot_gs_mlp_refine_features(len(Cs), *[a[1] for a in arrs],
                                         _ptr(alpha_hat, torch.float32, M, "alpha_hat"),
                                         _ptr(beta_hat, torch.float32, N, "beta_hat"), float(gamma), int(col0),
                                         int(out.shape[1]), _ptr(out, torch.float32, out.numel(), "out"),
                                         _stream_ptr(stream))
    _mlp_check(None, rc)
    return out


class WarmStartMLP:
    """The warm-start network on the current CUDA device (C ABI handle)."""

    def __init__(self, in_dim, width=256, max_batch=8192, seed=0, stream=None):
        import torch
        self.in_dim, self.width, self.max_batch = int(in_dim), int(width), int(max_batch)
        h = ctypes.c_void_p()
        rc = lib().ot_gs_mlp_create(ctypes.byref(h), self.in_dim, self.width, self.max_batch, int(seed),
                                    _stream_ptr(stream))
        _mlp_check(None, rc)
        self.h = h
        n = ctypes.c_int64()
        _mlp_check(h, lib().ot_gs_mlp_num_params(h, ctypes.byref(n)))
        self.num_params = n.value
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ot_gs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import torch
        p = torch.empty(self.num_params, dtype=torch.float32, device=self.device)
        _mlp_check(self.h, lib().ot_gs_mlp_get_params(self.h, _ptr(p, torch.float32, self.num_params, "p")))
        return p

    def set_params(self, p):
        import torch
        _mlp_check(self.h, lib().ot_gs_mlp_set_params(self.h, _ptr(p, torch.float32, self.num_params, "p")))

    def forward(self, X, out=None):
        """Predictions for the rows of X (in chunks of max_batch)."""
        import torch
        B = X.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float32, device=X.device)
        for s in range(0, B, self.max_batch):
            e = min(B, s + self.max_batch)
            xs, ys = X[s:e], out[s:e]
            _mlp_check(self.h, lib().ot_gs_mlp_forward(self.h, _ptr(xs, torch.float32, (e - s) * self.in_dim, "X"),
                                                       e - s, _ptr(ys, torch.float32, e - s, "y")))
        return out

    def grad(self, X, t, want_grad=False):
        import torch
        B = X.shape[0]
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        g = torch.empty(self.num_params, dtype=torch.float32, device=X.device) if want_grad else None
        _mlp_check(self.h, lib().ot_gs_mlp_grad(self.h, _ptr(X, torch.float32, B * self.in_dim, "X"),
                                                _ptr(t, torch.float32, B, "t"), B, _ptr(loss, torch.float32, 1, "loss"),
                                                _ptr(g, torch.float32, self.num_params, "grad")))
        return loss, g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _mlp_check(self.h, lib().ot_gs_mlp_adam(self.h, float(lr), float(beta1), float(beta2), float(eps)))

    def train_step(self, X, t, lr):
        loss, _ = self.grad(X, t)
        self.adam(lr)
        return loss
