"""Parity of the CUDA dense evaluation (ot_gs_grad, Eq. 4-5) with the FP64
oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, check_grad, solver

pytestmark = pytest.mark.gpu


def _run(p, gamma, mu, alpha, beta):
    """Two evaluations at the point, both against the oracle and equal bit
    for bit (the kernels' sums have a fixed order or are exact integers)."""
    s = solver(p, gamma, mu)
    a_t, b_t = torch.from_numpy(alpha).to(DEV), torch.from_numpy(beta).to(DEV)
    cold = s.grad(a_t, b_t).clone()
    warm = s.grad(a_t, b_t)
    torch.cuda.synchronize()
    o = oracle.Oracle.from_problem(p, gamma, mu)
    ref = o.dual(alpha, beta)
    check_grad(cold, ref, alpha, beta, p.a, p.b)
    assert torch.equal(cold, warm)
    return check_grad(warm, ref, alpha, beta, p.a, p.b)


def test_zero_start_is_exact():
    p = synth.tiny()
    s = solver(p, 1.0, 0.1)
    out = s.grad(torch.zeros(p.m, dtype=torch.float64, device=DEV),
                 torch.zeros(p.n, dtype=torch.float64, device=DEV)).cpu().numpy()
    assert out[0] == 0.0
    assert np.array_equal(out[1:1 + p.m], p.a) and np.array_equal(out[1 + p.m:], p.b)


@pytest.mark.parametrize("gamma,mu", [(1.0, 0.1), (0.1, 1.0), (10.0, 0.01), (1.0, 0.0)])
def test_tiny_random_points(gamma, mu):
    p = synth.tiny()
    for s in range(3):
        al, be = synth.random_duals(p.m, p.n, seed=s, scale=0.5, offset=0.3)
        _run(p, gamma, mu, al, be)


def test_tiny_near_optimum():
    """Near the optimum z - theta is ~1e-5 of z: the cancellation case."""
    p = synth.tiny()
    o = oracle.Oracle.from_problem(p, 1.0, 0.1)
    r = o.solve(tol=1e-9, maxit=3000)
    _run(p, 1.0, 0.1, r["alpha"], r["beta"])
    # shifted by a constant (D is invariant under alpha + s, beta - s)
    _run(p, 1.0, 0.1, r["alpha"] + 3.0, r["beta"] - 3.0)


@pytest.mark.parametrize("m,n,L,seed", [
    (300, 77, 7, 0),      # ragged n, unsorted labels
    (513, 129, 3, 1),     # big groups (> 64 rows), ragged
    (200, 1, 5, 2),       # one column
    (1, 40, 1, 3),        # one source row
    (700, 96, 40, 4),     # many small groups, some empty after Dirichlet
])
def test_random_shapes(m, n, L, seed):
    p = synth.random_instance(m, n, L, seed=seed, min_size=0 if L == 40 else 1)
    al, be = synth.random_duals(p.m, p.n, seed=seed + 10, scale=0.6, offset=0.35)
    _run(p, 0.7, 0.3, al, be)


def test_giant_group_uses_global_row_accumulators():
    """A group larger than the shared-memory row budget (4096 rows)."""
    rng = np.random.default_rng(5)
    sizes = np.array([4500, 30, 2])
    XS, XT, lab = synth.mixture_features(sizes, 70, 3, rng)
    p = synth.make_problem(XS, XT, lab, 3)
    al, be = synth.random_duals(p.m, p.n, seed=6, scale=0.3, offset=0.3)
    _run(p, 1.0, 0.05, al, be)


def test_deterministic_repeat():
    p = synth.random_instance(400, 300, 6, seed=7)
    s = solver(p, 1.0, 0.2)
    al, be = synth.random_duals(p.m, p.n, seed=8)
    a_t, b_t = torch.from_numpy(al).to(DEV), torch.from_numpy(be).to(DEV)
    o1 = s.grad(a_t, b_t).clone()
    o2 = s.grad(a_t, b_t)
    assert torch.equal(o1, o2)


def test_result_does_not_depend_on_earlier_evaluations():
    """An evaluation leaves no state that changes the next one: at x1 the
    result is the same bit for bit whether it follows nothing, an evaluation
    at x1, or one at a far point x2, and the snapshot pass gives it too."""
    p = synth.random_instance(700, 300, 9, seed=11)
    gamma, mu = 1.0, 0.3
    o = oracle.Oracle.from_problem(p, gamma, mu)
    x1 = synth.random_duals(p.m, p.n, seed=12, scale=0.6, offset=0.35)
    x2 = synth.random_duals(p.m, p.n, seed=13, scale=0.6, offset=0.2)
    t = lambda v: torch.from_numpy(v).to(DEV)
    s = solver(p, gamma, mu)
    first = s.grad(t(x1[0]), t(x1[1])).clone()
    again = s.grad(t(x1[0]), t(x1[1])).clone()
    s.grad(t(x2[0]), t(x2[1]))
    after_x2 = s.grad(t(x1[0]), t(x1[1])).clone()
    snap = torch.empty_like(first)
    s.snapshot(t(x1[0]), t(x1[1]), build_N=False, out=snap)
    torch.cuda.synchronize()
    assert torch.equal(first, again) and torch.equal(first, after_x2) and torch.equal(first, snap)
    check_grad(first, o.dual(*x1), x1[0], x1[1], p.a, p.b)
