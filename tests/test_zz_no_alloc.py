"""The allocation-free evaluation entry point (ot_gs_grad_noalloc).

It serves callers that cannot allocate device memory; its scratch lives in a
static device array.  Its results must match the handle-based ot_gs_grad
within the tolerances the other parity tests use, on two calls in a row (the
second call reuses the array the first one left behind).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2303_07597_gb300 as pk
import synth


def _check(out, ref, alpha, beta, a, b):
    o, r = out.cpu().numpy(), ref.cpu().numpy()
    m = len(a)
    scale = abs(alpha @ a) + abs(beta @ b) + abs(alpha @ a + beta @ b - r[0])
    assert abs(o[0] - r[0]) <= 1e-9 * max(scale, 1e-300)
    assert (np.abs(o[1:1 + m] - r[1:1 + m]) / np.maximum(np.abs(r[1:1 + m]), a)).max() <= 1e-5
    assert (np.abs(o[1 + m:] - r[1 + m:]) / np.maximum(np.abs(r[1 + m:]), b)).max() <= 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("mk,gamma,mu", [
    (lambda: synth.tiny(seed=0), 1.0, 0.1),
    (lambda: synth.random_instance(520, 128, 6, seed=3, shuffle_rows=False), 0.7, 0.3),
])
def test_noalloc_matches_handle_twice(mk, gamma, mu):
    p = mk()
    dev = "cuda:0"
    C = torch.from_numpy(p.C).to(dev)
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    s = pk.GroupSparseOT(C, a, b, torch.from_numpy(p.labels).to(dev), p.L, gamma, mu)
    for call in range(2):
        al, be = synth.random_duals(p.m, p.n, seed=10 + call)
        at, bt = torch.from_numpy(al).to(dev), torch.from_numpy(be).to(dev)
        out = torch.full((1 + p.m + p.n,), float("nan"), dtype=torch.float64, device=dev)
        pk.ot_gs_grad_noalloc(C, a, b, p.labels, p.L, gamma, mu, at, bt, out)
        ref = s.grad(at, bt)
        torch.cuda.synchronize()
        _check(out, ref, al, be, p.a, p.b)
    s.close()


def test_noalloc_rejects_oversized_problem_before_gpu_work():
    """The size check runs on the host before any CUDA call."""
    # scratch is about 44 B per row: two million rows do not fit in 64 MB
    m, n, L = 2_000_000, 1000, 1000
    lab = synth.labels_from_sizes(synth.class_sizes_zipf(m, L, 1.1, 2))
    rc = pk.lib().ot_gs_grad_noalloc(ctypes.c_void_p(16), n, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     lab.ctypes.data_as(ctypes.c_void_p), m, n, L, 1.0, 0.5,
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == pk.OTGS_EINVAL
    assert "bytes of scratch" in pk.lib().ot_gs_noalloc_last_error().decode()
