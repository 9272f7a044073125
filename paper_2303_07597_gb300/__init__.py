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
                ("use_lower_bound", ctypes.c_int32), ("time_budget_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("iters", ctypes.c_int64),
                ("blocks_total", ctypes.c_int64), ("blocks_in_N", ctypes.c_int64),
                ("blocks_skipped", ctypes.c_int64), ("blocks_checked", ctypes.c_int64),
                ("units_total", ctypes.c_int64), ("units_computed", ctypes.c_int64),
                ("snapshots", ctypes.c_int64), ("c_bytes", ctypes.c_double)]

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
        "ot_gs_reset_stats": ([P], ctypes.c_int),
        "ot_gs_set_timing": ([P, ctypes.c_int], ctypes.c_int),
        "ot_gs_get_timing": ([P, P, P], ctypes.c_int),
        "ot_gs_last_error": ([P], ctypes.c_char_p),
        "ot_gs_version": ([], ctypes.c_char_p),
        "ot_gs_plan_info": ([P, i64, i64, i32, P, P, P], ctypes.c_int),
        "ot_gs_grad_noalloc": ([P, i64, P, P, P, i64, i64, i32, dbl, dbl, P, P, P, P], ctypes.c_int),
        "ot_gs_noalloc_last_error": ([], ctypes.c_char_p),
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
def ot_gs_create(C, a, b, labels, L, gamma, mu, stream=None):
    """C: (m, n) float32 CUDA (row stride C.stride(0)); a (m,), b (n,) float64;
    labels (m,) int32 in [0, L).  Returns the raw handle (ctypes.c_void_p)."""
    import torch
    if C.dim() != 2 or C.stride(1) != 1:
        raise ValueError("C must be 2-D with unit column stride")
    m, n = C.shape
    h = ctypes.c_void_p()
    rc = lib().ot_gs_create(ctypes.byref(h), _ptr(C, torch.float32, name="C") if C.is_contiguous()
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


def ot_gs_get_stats(h) -> dict:
    s = Stats()
    _check(h, lib().ot_gs_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def ot_gs_reset_stats(h):
    return _check(h, lib().ot_gs_reset_stats(h))


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


# ------------------------------------------------------------ convenience
class GroupSparseOT:
    """One problem on the current CUDA device.  Keeps references to the
    borrowed input tensors for the handle's lifetime."""

    def __init__(self, C, a, b, labels, L, gamma, mu, stream=None):
        import torch
        self._keep = (C, a, b, labels)
        self.m, self.n = C.shape
        self.L = int(L)
        self.device = C.device
        self.h = ot_gs_create(C, a, b, labels, L, gamma, mu, stream)

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

    def stats(self):
        return ot_gs_get_stats(self.h)
