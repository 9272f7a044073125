"""The allocation-free evaluation entry point (ot_gs_grad_noalloc).

It serves callers that cannot allocate device memory; its scratch lives in a
static device array.  Its results must match the FP64 oracle and the
handle-based ot_gs_grad within the tolerances the other parity tests use, on
two calls in a row (the second call reuses the array the first one left
behind).  The cases reach the path of a class taller than the split height
(its pieces' partial sums and their finishing kernel) and many flagged
blocks (thousands of block sets for the exact-sum kernel).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth


def _check(out, ref, alpha, beta, a, b):
    o = out.cpu().numpy()
    D, ga, gb = ref
    m = len(a)
    scale = abs(alpha @ a) + abs(beta @ b) + abs(alpha @ a + beta @ b - D)
    assert abs(o[0] - D) <= 1e-9 * max(scale, 1e-300), (o[0], D)
    assert (np.abs(o[1:1 + m] - ga) / np.maximum(np.abs(ga), a)).max() <= 1e-5
    assert (np.abs(o[1 + m:] - gb) / np.maximum(np.abs(gb), b)).max() <= 1e-5


def _sized(sizes, n, seed, d=4):
    """Class-sorted problem with the given class sizes (mixture features)."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes)
    XS, XT, lab = synth.mixture_features(sizes, n, d, rng)
    return synth.make_problem(XS, XT, lab, len(sizes), name=f"sized_{int(sizes.sum())}x{n}")


def _many_deferred():
    """100 classes of 40 rows (each a panel of its own, its blocks spanning
    two stages) x 4096 columns: with the duals of the test several thousand
    (class, 32-column tile) block sets hold active blocks."""
    return _sized(np.full(100, 40), 4096, seed=7)


CASES = [
    ("tiny", lambda: synth.tiny(seed=0), 1.0, 0.1),
    ("random520", lambda: synth.random_instance(520, 128, 6, seed=3, shuffle_rows=False), 0.7, 0.3),
    ("tall_class", lambda: _sized([1500, 300, 180, 20], 300, seed=5), 0.7, 0.3),
    ("many_deferred", _many_deferred, 0.7, 0.3),
]


@pytest.mark.gpu
@pytest.mark.parametrize("name,mk,gamma,mu", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_and_handle_twice(name, mk, gamma, mu):
    p = mk()
    dev = "cuda:0"
    C = torch.from_numpy(p.C).to(dev)
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    s = pk.GroupSparseOT(C, a, b, torch.from_numpy(p.labels).to(dev), p.L, gamma, mu)
    o = oracle.Oracle.from_problem(p, gamma, mu)
    for call in range(2):
        al, be = synth.random_duals(p.m, p.n, seed=10 + call)
        ref = o.dual(al, be)
        if name == "many_deferred":
            # (class, 32-column tile) block sets with a nonzero plan entry
            T = o.plan(al, be)
            act = (T.reshape(p.L, 40, p.n // 32, 32) != 0).any(axis=(1, 3))
            assert int(act.sum()) > 4096
            del T
        at, bt = torch.from_numpy(al).to(dev), torch.from_numpy(be).to(dev)
        out = torch.full((1 + p.m + p.n,), float("nan"), dtype=torch.float64, device=dev)
        pk.ot_gs_grad_noalloc(C, a, b, p.labels, p.L, gamma, mu, at, bt, out)
        hout = s.grad(at, bt)
        torch.cuda.synchronize()
        _check(out, ref, al, be, p.a, p.b)
        _check(out, (hout[0].item(), hout[1:1 + p.m].cpu().numpy(), hout[1 + p.m:].cpu().numpy()),
               al, be, p.a, p.b)
    s.close()


def test_noalloc_rejects_oversized_problem_before_gpu_work():
    """The size check runs on the host before any CUDA call."""
    # 52 B per row alone: two million rows do not fit in 64 MB
    m, n, L = 2_000_000, 1000, 1000
    lab = synth.labels_from_sizes(synth.class_sizes_zipf(m, L, 1.1, 2))
    rc = pk.lib().ot_gs_grad_noalloc(ctypes.c_void_p(16), n, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                     lab.ctypes.data_as(ctypes.c_void_p), m, n, L, 1.0, 0.5,
                                     ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == pk.OTGS_EINVAL
    assert "bytes of scratch" in pk.lib().ot_gs_noalloc_last_error().decode()


def test_noalloc_wrapper_checks_C():
    """The binding refuses a C the library would misread (no GPU needed: it
    raises before any call)."""
    with pytest.raises(TypeError):
        pk.ot_gs_grad_noalloc(torch.zeros(4, 4, dtype=torch.float64), None, None, np.zeros(4, np.int32), 1,
                              1.0, 0.1, None, None, None)
