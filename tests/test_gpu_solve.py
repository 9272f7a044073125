"""The device L-BFGS solver (ot_gs_solve) against the FP64 oracle: the same
optimum D*, a converged gradient, screened == dense (Thm. 2, here bit for bit
because each screened evaluation equals the dense one), warm starts and the
stopping statuses."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, solver

pytestmark = pytest.mark.gpu


def _solve(p, gamma, mu, tol, maxit=5000, screening=False, use_lower=True):
    s = solver(p, gamma, mu)
    s.set_params(use_screening=int(screening), use_lower_bound=int(use_lower))
    rc = s.solve(tol, maxit)
    sol = s.solution()
    return s, rc, sol


@pytest.mark.parametrize("gamma,mu", [(1.0, 0.1), (10.0, 0.01), (0.1, 1.0)])
def test_solve_matches_oracle_optimum(gamma, mu):
    p = synth.tiny(seed=1)
    o = oracle.Oracle.from_problem(p, gamma, mu)
    ref = o.solve(tol=1e-10, maxit=5000)
    s, rc, sol = _solve(p, gamma, mu, 1e-9)
    assert rc == pk.OTGS_OK, pk.ot_gs_last_error(s.h)
    al, be = sol["alpha"].cpu().numpy(), sol["beta"].cpu().numpy()
    D, ga, gb = o.dual(al, be)
    assert abs(D - ref["D"]) <= 1e-9 * abs(ref["D"])
    assert abs(sol["D"] - D) <= 1e-9 * abs(D)
    # the oracle confirms convergence at the GPU's point (within FP32-f error)
    assert max(np.abs(ga).max(), np.abs(gb).max()) <= 1e-8


@pytest.mark.parametrize("use_lower", [True, False])
def test_screened_solve_is_bitwise_dense(use_lower):
    p = synth.random_instance(500, 160, 12, seed=2)
    s0, rc0, sol0 = _solve(p, 1.0, 0.3, 1e-9)
    s1, rc1, sol1 = _solve(p, 1.0, 0.3, 1e-9, screening=True, use_lower=use_lower)
    assert rc0 == rc1 == pk.OTGS_OK
    assert sol0["iters"] == sol1["iters"]
    assert sol0["D"] == sol1["D"]
    assert torch.equal(sol0["alpha"], sol1["alpha"]) and torch.equal(sol0["beta"], sol1["beta"])
    st = s1.stats()
    assert st["blocks_skipped"] > 0.5 * st["blocks_checked"]
    assert st["snapshots"] >= sol1["iters"] // 10


def test_warm_start_from_solution_converges_at_once():
    p = synth.tiny(seed=3)
    o = oracle.Oracle.from_problem(p, 1.0, 0.1)
    ref = o.solve(tol=1e-11, maxit=5000)
    s = solver(p, 1.0, 0.1)
    s.set_state(torch.from_numpy(ref["alpha"]).to(DEV), torch.from_numpy(ref["beta"]).to(DEV))
    rc = s.solve(1e-8, 100)
    sol = s.solution()
    assert rc == pk.OTGS_OK and sol["iters"] <= 1
    assert abs(sol["D"] - ref["D"]) <= 1e-10 * abs(ref["D"])


def test_maxit_and_time_budget_statuses():
    p = synth.tiny(seed=4)
    s = solver(p, 1.0, 0.1)
    assert s.solve(1e-12, 3) == pk.OTGS_ENOTCONV
    assert s.solution()["iters"] == 3
    s2 = solver(p, 1.0, 0.1)
    s2.set_params(time_budget_ms=1e-6)
    assert s2.solve(1e-12, 1000) == pk.OTGS_ETIMEOUT


def test_unsorted_labels_and_ragged_solve():
    p = synth.random_instance(333, 95, 9, seed=5)
    o = oracle.Oracle.from_problem(p, 0.5, 0.4)
    ref = o.solve(tol=1e-10, maxit=5000)
    s, rc, sol = _solve(p, 0.5, 0.4, 1e-9)
    assert rc == pk.OTGS_OK
    D, _, _ = o.dual(sol["alpha"].cpu().numpy(), sol["beta"].cpu().numpy())
    assert abs(D - ref["D"]) <= 1e-9 * abs(ref["D"])


def test_objective_trace_follows_the_solve():
    """ot_gs_get_trace: one entry for the start point and one per accepted
    iteration; the line search accepts ascent steps of D (or, by its
    approximate sufficient-decrease rule, a change within 1e-12 |D|), device
    time grows, and the last entry is the reported optimum."""
    p = synth.tiny(seed=4)
    s, rc, sol = _solve(p, 1.0, 0.1, 1e-9)
    assert rc == pk.OTGS_OK
    D, t, ev = s.trace()
    assert len(D) == sol["iters"] + 1
    assert D[0] == 0.0  # Alg. 1 starts at alpha = beta = 0 where D = 0
    assert np.all(np.diff(D) >= -1e-12 * np.abs(D[1:]))
    assert np.all(np.diff(t) >= 0.0) and t[0] >= 0.0
    assert np.all(np.diff(ev) >= 1) and ev[0] == 1
    assert D[-1] == sol["D"]
    # every evaluation of the (dense) solve is counted once: the start point
    # and each line-search trial the device ran
    assert s.stats()["evals"] == ev[-1]
