"""Batches of independent problems (ot_gs_create_batch): one evaluation
kernel for all problems, one L-BFGS state per problem.  Each problem's
objective and gradient are compared with the FP64 oracle element by element;
solves with the oracle's solve and with the single-problem solver."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, check_grad, solver, to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(300, 77, 7, 0), (64, 1, 5, 1), (1, 40, 1, 2), (513, 129, 3, 3), (200, 255, 12, 4),
          (700, 96, 40, 5), (37, 513, 4, 6)]


def make_batch(problems, gamma, mu):
    devs = [to_dev(p) for p in problems]
    return pk.GroupSparseOTBatch([d[0] for d in devs], [d[1] for d in devs], [d[2] for d in devs],
                                 [d[3] for d in devs], [p.L for p in problems], gamma, mu)


def concat_duals(problems, seed):
    al, be = [], []
    for k, p in enumerate(problems):
        a, b = synth.random_duals(p.m, p.n, seed=seed + k, scale=0.6, offset=0.35)
        al.append(a)
        be.append(b)
    return al, be


def check_batch(B, problems, gamma, mu, al, be):
    D, g = B.grad(torch.from_numpy(np.concatenate(al)).to(DEV), torch.from_numpy(np.concatenate(be)).to(DEV))
    D, g = D.cpu().numpy(), g.cpu().numpy()
    worst = 0.0
    for k, p in enumerate(problems):
        o = oracle.Oracle.from_problem(p, gamma, mu)
        out = np.concatenate([[D[k]], g[B.row_off[k]:B.row_off[k + 1]],
                              g[B.m + B.col_off[k]:B.m + B.col_off[k + 1]]])
        r = check_grad(torch.from_numpy(out), o.dual(al[k], be[k]), al[k], be[k], p.a, p.b, what=p.name)
        worst = max(worst, r["D_rel"])
    return D, g


def test_batch_grad_matches_oracle_per_problem():
    problems = [synth.random_instance(m, n, L, seed=s) for m, n, L, s in SHAPES]
    B = make_batch(problems, 0.7, 0.3)
    al, be = concat_duals(problems, 10)
    check_batch(B, problems, 0.7, 0.3, al, be)


def test_batch_grad_generator_shapes():
    """Problems of the batched workload's generator (smaller sizes)."""
    problems = synth.batch(seed=3, nprob=12, m_range=(20, 400), n_range=(20, 400), L_range=(5, 60), d=16)
    B = make_batch(problems, 1.0, 0.1)
    al, be = concat_duals(problems, 30)
    check_batch(B, problems, 1.0, 0.1, al, be)


def test_batch_plans_agree():
    """Row sums are fixed point and a block's rows are summed in the same
    order in any panel: plans with the same split height give the same alpha
    gradient bit for bit.  A column's contributions are added in FP64 over an
    item's blocks before the fixed-point conversion, and another split height
    changes the order in which a tall group's norm is summed (piece by
    piece): the rest moves in its last bits only."""
    problems = [synth.random_instance(m, n, L, seed=s) for m, n, L, s in SHAPES]
    B = make_batch(problems, 1.0, 0.2)
    al, be = concat_duals(problems, 40)
    at, bt = torch.from_numpy(np.concatenate(al)).to(DEV), torch.from_numpy(np.concatenate(be)).to(DEV)
    D0, g0 = B.grad(at, bt)
    scale = torch.maximum(g0.abs(), torch.from_numpy(np.concatenate([p.a for p in problems] +
                                                                     [p.b for p in problems])).to(DEV))
    for pr, sr, sf in [(32, 256, 0), (1024, 256, 0), (32, 64, 0), (64, 128, 16), (512, 1024, 0), (256, 256, 16),
                       (512, 256, 1)]:
        B.set_plan(pr, sr, sf)
        pl = B.plan()
        assert (pl["panel_rows"], pl["split_rows"], pl["stage_fill"]) == (pr, sr, sf)
        D1, g1 = B.grad(at, bt)
        if sr == 256:
            assert torch.equal(g0[:B.m], g1[:B.m]), (pr, sr, sf)
        assert ((g1 - g0).abs() / scale).max().item() <= 1e-11, (pr, sr)
        assert torch.allclose(D0, D1, rtol=1e-12, atol=0), (pr, sr, (D0 - D1).abs().max().item())


def test_autotune_picks_a_shape_and_caches():
    pk.ot_gs_autotune_clear_cache()
    problems = synth.batch(seed=5, nprob=10, m_range=(50, 300), n_range=(50, 300), L_range=(5, 30), d=8)
    B = make_batch(problems, 1.0, 0.1)
    al, be = concat_duals(problems, 50)
    at, bt = torch.from_numpy(np.concatenate(al)).to(DEV), torch.from_numpy(np.concatenate(be)).to(DEV)
    r = B.autotune(at, bt, evals=2)
    assert r["best_ms"] > 0
    pl = B.plan()
    assert (pl["panel_rows"], pl["split_rows"], pl["stage_fill"]) == (r["panel_rows"], r["split_rows"], r["stage_fill"])
    r2 = B.autotune(at, bt, evals=2)
    assert r2["best_ms"] == 0.0
    assert (r2["panel_rows"], r2["split_rows"], r2["stage_fill"]) == (r["panel_rows"], r["split_rows"], r["stage_fill"])
    check_batch(B, problems, 1.0, 0.1, al, be)


SOLVE_SHAPES = [(120, 90, 6, 1), (60, 140, 4, 2), (200, 33, 9, 3), (40, 17, 3, 4)]


def test_batch_solve_matches_oracle_solve():
    problems = [synth.random_instance(m, n, L, seed=s, d=3) for m, n, L, s in SOLVE_SHAPES]
    gamma, mu, tol = 1.0, 0.1, 1e-8
    B = make_batch(problems, gamma, mu)
    st = B.solve(tol=tol, maxit=5000)
    r = B.result()
    assert st == pk.OTGS_OK and np.all(r["status"] == 0), r["status"]
    assert np.all(r["grad_inf"] <= tol)
    D, g = B.grad(r["alpha"], r["beta"])
    assert np.allclose(D.cpu().numpy(), r["D"], rtol=1e-12, atol=0)
    for k, p in enumerate(problems):
        o = oracle.Oracle.from_problem(p, gamma, mu)
        ro = o.solve(tol=tol, maxit=5000)
        assert ro["status"] == "ok"
        assert abs(r["D"][k] - ro["D"]) <= 1e-9 * abs(ro["D"]), (k, r["D"][k], ro["D"])
        assert r["iters"][k] > 0
        assert r["evals"][k] >= r["iters"][k] + 1
    assert np.all(r["t_ms"] > 0)


def test_batch_iterates_like_each_problem_alone():
    """One L-BFGS state per problem and per-problem fixed-point scales: a
    problem takes the same iterates in a batch as in a batch of its own, bit
    for bit, whatever the other problems do (here some stop early on maxit
    while the others run on)."""
    problems = [synth.random_instance(m, n, L, seed=s, d=3) for m, n, L, s in SOLVE_SHAPES]
    gamma, mu, tol, maxit = 1.0, 0.1, 1e-8, 150
    B = make_batch(problems, gamma, mu)
    B.solve(tol=tol, maxit=maxit)
    r = B.result()
    for k, p in enumerate(problems):
        B1 = make_batch([p], gamma, mu)
        B1.solve(tol=tol, maxit=maxit)
        r1 = B1.result()
        assert r1["iters"][0] == r["iters"][k] and r1["evals"][0] == r["evals"][k], k
        assert r1["D"][0] == r["D"][k] and r1["status"][0] == r["status"][k], k
        assert torch.equal(r1["alpha"], B.split(r["alpha"], k, "alpha"))
        assert torch.equal(r1["beta"], B.split(r["beta"], k, "beta"))


def test_batch_of_one_follows_the_single_solver():
    p = synth.random_instance(300, 200, 8, seed=9, d=3)
    gamma, mu, tol = 1.0, 0.2, 1e-8
    B = make_batch([p], gamma, mu)
    assert B.solve(tol=tol, maxit=3000) == pk.OTGS_OK
    rb = B.result()
    s = solver(p, gamma, mu)
    assert s.solve(tol=tol, maxit=3000) == pk.OTGS_OK
    rs = s.solution()
    assert abs(rb["D"][0] - rs["D"]) <= 1e-10 * abs(rs["D"])
    # the same iteration up to the last bits of the reductions
    assert abs(int(rb["iters"][0]) - rs["iters"]) <= max(3, rs["iters"] // 5)


def test_batch_target_stop_and_warm_start():
    problems = [synth.random_instance(m, n, L, seed=s, d=3) for m, n, L, s in
                [(150, 120, 6, 11), (90, 200, 5, 12), (250, 60, 10, 13)]]
    gamma, mu = 1.0, 0.1
    B = make_batch(problems, gamma, mu)
    assert B.solve(tol=1e-8, maxit=20000) == pk.OTGS_OK
    ref = B.result()
    Dstar = ref["D"].copy()
    zero_a = torch.zeros(B.m, dtype=torch.float64, device=DEV)
    zero_b = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    B.set_state(zero_a, zero_b)
    assert B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6) == pk.OTGS_OK
    cold = B.result()
    assert np.all(cold["D"] >= Dstar - 1e-6 * np.abs(Dstar))
    assert np.all(cold["iters"] <= ref["iters"])
    # from the optimum the target holds at the start point: no iteration
    B.set_state(ref["alpha"], ref["beta"])
    assert B.solve(tol=0.0, maxit=100, target_D=Dstar, target_rtol=1e-6) == pk.OTGS_OK
    warm = B.result()
    assert np.all(warm["iters"] == 0) and np.all(warm["evals"] == 1)


def test_batch_rejects_single_problem_calls():
    problems = [synth.random_instance(50, 40, 3, seed=s) for s in (1, 2)]
    B = make_batch(problems, 1.0, 0.1)
    out = torch.empty(1 + B.m + B.n, dtype=torch.float64, device=DEV)
    al = torch.zeros(B.m, dtype=torch.float64, device=DEV)
    be = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    with pytest.raises(pk.OTGSError) as e:
        pk.ot_gs_grad(B.h, al, be, out)
    assert e.value.code == pk.OTGS_EINVAL
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_solve(B.h, 1e-6, 10)


def test_batch_solve_after_changing_mu():
    """The batched solver's captured trials hold theta = mu gamma and 1 / (2
    gamma): after set_params changes mu (or gamma) the next solve must use the
    new values.  Solve, change mu, solve again from zero: D* is the oracle's
    at the new mu, for every problem."""
    problems = [synth.random_instance(m, n, L, seed=s, d=3) for m, n, L, s in SOLVE_SHAPES[:3]]
    gamma, tol = 1.0, 1e-8
    B = make_batch(problems, gamma, 0.1)
    assert B.solve(tol=tol, maxit=5000) == pk.OTGS_OK
    zero_a = torch.zeros(B.m, dtype=torch.float64, device=DEV)
    zero_b = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    for g2, mu2 in [(gamma, 0.4), (0.5, 0.4)]:
        B.set_params(gamma=g2, mu=mu2)
        B.set_state(zero_a, zero_b)
        assert B.solve(tol=tol, maxit=5000) == pk.OTGS_OK
        r = B.result()
        for k, p in enumerate(problems):
            ro = oracle.Oracle.from_problem(p, g2, mu2).solve(tol=tol, maxit=5000)
            assert ro["status"] == "ok"
            assert abs(r["D"][k] - ro["D"]) <= 1e-9 * abs(ro["D"]), (g2, mu2, k, r["D"][k], ro["D"])
