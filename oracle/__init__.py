"""FP64 CPU oracle for group-sparse regularised optimal transport.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never calls it; the library product fails loudly when
its CUDA extension is missing instead of falling back here.

The arithmetic lives in ``otgs_oracle.c`` (plain C, FP64, single thread),
compiled with gcc into ``_build/liborc.so`` on first use.  This module only
marshals numpy arrays.  Functions and the paper passages they follow:

* :meth:`Oracle.dual`      D and grad D, dense (Eq. 4, Eq. 5)
* :meth:`Oracle.plan`      plan recovery t_j = grad psi(...) (Sec. 2.3)
* :meth:`Oracle.primal`    primal objective (Eq. 2, Eq. 3)
* :meth:`Oracle.bounds`    upper / lower bounds (Eq. 6, Eq. 7)
* :meth:`Oracle.gradpsi`   screened evaluation (Alg. 2)
* :meth:`Oracle.solve`     L-BFGS, dense or screened (Alg. 1)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "otgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -4: "maxit", -6: "line search"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (ISO C11, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-frounding-math", "-fPIC",
                               "-shared", "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [i64, i64, i32, P, P, P, P, dbl, dbl]
        lib.orc_destroy.argtypes = [P]
        lib.orc_theta.restype = dbl
        lib.orc_theta.argtypes = [P]
        lib.orc_dual.argtypes = [P, P, P, P, P, P, P, P]
        lib.orc_plan.argtypes = [P, P, P, P]
        lib.orc_primal.restype = dbl
        lib.orc_primal.argtypes = [P, P]
        lib.orc_bounds.argtypes = [P, P, P, P, P, P, P, P, P]
        lib.orc_gradpsi.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_gpu_screen.argtypes = [P, P, P, P, P, P, P, i64, P, i64, P, P, P]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_solve.argtypes = [P, P, P, dbl, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int, P]
        _lib = lib
        return lib


def _p(x: np.ndarray | None):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _f64(x, k=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if k is not None and x.shape != (k,):
        raise ValueError(f"expected shape ({k},), got {x.shape}")
    return x


def rho_to_gamma_mu(gamma: float, rho: float):
    """The experiments' rho form (Sec. 5.2), gamma(1/2 (1-rho)||t||^2 +
    rho sum_l ||t_[l]||), equals Eq. 3 with gamma' = gamma (1 - rho) and
    mu' = rho / (1 - rho)."""
    if not (0.0 <= rho < 1.0):
        raise ValueError("rho must be in [0, 1)")
    return gamma * (1.0 - rho), rho / (1.0 - rho)


class Oracle:
    """One problem instance (copies C, labels, a, b)."""

    def __init__(self, C, labels, a, b, L, gamma, mu):
        lib = _load()
        self.C = np.ascontiguousarray(C, dtype=np.float32)
        self.m, self.n = self.C.shape
        self.labels = np.ascontiguousarray(labels, dtype=np.int32)
        self.a = _f64(a, self.m)
        self.b = _f64(b, self.n)
        self.L = int(L)
        self.gamma, self.mu = float(gamma), float(mu)
        h = lib.orc_create(self.m, self.n, self.L, _p(self.C), _p(self.labels), _p(self.a),
                           _p(self.b), self.gamma, self.mu)
        if not h:
            raise ValueError("invalid oracle problem")
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.theta = lib.orc_theta(self._h)
        self.sizes = np.bincount(self.labels, minlength=self.L)

    @classmethod
    def from_problem(cls, p, gamma, mu):
        return cls(p.C, p.labels, p.a, p.b, p.L, gamma, mu)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_destroy(h)
            self._h = None

    def dual(self, alpha, beta, want_norms=False):
        """Returns (D, dD/dalpha, dD/dbeta[, z, o]) -- Eq. 4, Eq. 5."""
        alpha, beta = _f64(alpha, self.m), _f64(beta, self.n)
        D = np.zeros(1)
        ga, gb = np.empty(self.m), np.empty(self.n)
        z = o = None
        if want_norms:
            z, o = np.empty((self.L, self.n)), np.empty((self.L, self.n))
        self._lib.orc_dual(self._h, _p(alpha), _p(beta), _p(D), _p(ga), _p(gb), _p(z), _p(o))
        if want_norms:
            return float(D[0]), ga, gb, z, o
        return float(D[0]), ga, gb

    def plan(self, alpha, beta):
        alpha, beta = _f64(alpha, self.m), _f64(beta, self.n)
        T = np.empty((self.m, self.n))
        self._lib.orc_plan(self._h, _p(alpha), _p(beta), _p(T))
        return T

    def primal(self, T):
        T = np.ascontiguousarray(T, dtype=np.float64)
        assert T.shape == (self.m, self.n)
        return float(self._lib.orc_primal(self._h, _p(T)))

    def bounds(self, alpha, beta, alpha_s, beta_s, zt, ot):
        """(zbar, zlow), each L x n -- Eq. 6, Eq. 7."""
        args = [_f64(alpha, self.m), _f64(beta, self.n), _f64(alpha_s, self.m),
                _f64(beta_s, self.n)]
        zt = np.ascontiguousarray(zt, dtype=np.float64)
        ot = np.ascontiguousarray(ot, dtype=np.float64)
        zup, zlow = np.empty((self.L, self.n)), np.empty((self.L, self.n))
        self._lib.orc_bounds(self._h, *[_p(x) for x in args], _p(zt), _p(ot), _p(zup), _p(zlow))
        return zup, zlow

    def gradpsi(self, alpha, beta, alpha_s, beta_s, zt, inN):
        """Screened evaluation (Alg. 2).  Returns (D, ga, gb, skipped, counts)."""
        args = [_f64(alpha, self.m), _f64(beta, self.n), _f64(alpha_s, self.m),
                _f64(beta_s, self.n)]
        zt = np.ascontiguousarray(zt, dtype=np.float64)
        inN = np.ascontiguousarray(inN, dtype=np.uint8)
        D = np.zeros(1)
        ga, gb = np.empty(self.m), np.empty(self.n)
        skipped = np.zeros((self.L, self.n), dtype=np.uint8)
        counts = np.zeros(4, dtype=np.int64)
        self._lib.orc_gradpsi(self._h, *[_p(x) for x in args], _p(zt), _p(inN), _p(D), _p(ga),
                              _p(gb), _p(skipped), _p(counts))
        return float(D[0]), ga, gb, skipped.astype(bool), counts

    def gpu_screen_rule(self, alpha, beta, alpha_s, beta_s, zt, ot, Nmask=None):
        """Replica of the CUDA path's FP32 screening rule (Eq. 6-8 with
        directed rounding and margin).  zt, ot: float32 (L, ldz); Nmask:
        uint32 (L, ntiles) or None.  Returns (skip words, N words, counts)."""
        args = [_f64(alpha, self.m), _f64(beta, self.n), _f64(alpha_s, self.m),
                _f64(beta_s, self.n)]
        zt = np.ascontiguousarray(zt, dtype=np.float32)
        ot = np.ascontiguousarray(ot, dtype=np.float32)
        ntiles = (self.n + 31) // 32
        assert zt.shape[0] == self.L and zt.shape[1] >= self.n and ot.shape == zt.shape
        Nm = None if Nmask is None else np.ascontiguousarray(Nmask, dtype=np.uint32).reshape(self.L, ntiles)
        skip = np.zeros((self.L, ntiles), dtype=np.uint32)
        Nout = np.zeros((self.L, ntiles), dtype=np.uint32)
        counts = np.zeros(3, dtype=np.int64)
        self._lib.orc_gpu_screen(self._h, *[_p(x) for x in args], _p(zt), _p(ot), zt.shape[1], _p(Nm),
                                 ntiles, _p(skip), _p(Nout), _p(counts))
        return skip, Nout, counts

    def solve(self, tol=1e-8, maxit=1000, M=10, screening=False, use_lower=True, r=10,
              alpha0=None, beta0=None, trace=False):
        """L-BFGS on -D (dense, or Alg. 1 with screening=True)."""
        alpha = np.zeros(self.m) if alpha0 is None else _f64(alpha0, self.m).copy()
        beta = np.zeros(self.n) if beta0 is None else _f64(beta0, self.n).copy()
        D = np.zeros(1)
        ginf = np.zeros(1)
        counts = np.zeros(10, dtype=np.int64)
        tr = np.full(maxit + 1, np.nan) if trace else None
        st = self._lib.orc_solve(self._h, _p(alpha), _p(beta), float(tol), int(maxit), int(M),
                                 int(bool(screening)), int(bool(use_lower)), int(r), _p(D),
                                 _p(counts), _p(tr), 0 if tr is None else len(tr), _p(ginf))
        res = dict(D=float(D[0]), alpha=alpha, beta=beta, status=STATUS.get(st, str(st)),
                   iters=int(counts[0]), evals=int(counts[1]), in_N=int(counts[3]),
                   checked=int(counts[4]), skipped=int(counts[5]), unskipped=int(counts[6]),
                   snapshot_blocks=int(counts[7]), grad_inf=float(ginf[0]))
        if trace:
            res["trace"] = tr[: res["iters"] + 1]
        return res
