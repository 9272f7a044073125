"""Screening on the GPU (Alg. 2, Eq. 6-8) against the oracle: the skip set and
the set N bit for bit against the oracle's FP32 rule (given the GPU's stored
snapshot), and against the paper's rule in FP64: every block the GPU skips the
paper's rule skips, the rest differs only within the FP32 rounding band;
skipped blocks safe (zero gradient in exact FP64), and screened evaluation ==
dense evaluation bit for bit (Thm. 2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, check_grad, solver

pytestmark = pytest.mark.gpu


def _state(s, p):
    nt = (p.n + 31) // 32
    zt = torch.empty(p.L * nt * 32, dtype=torch.float32, device=DEV)
    ot = torch.empty_like(zt)
    al = torch.empty(p.m, dtype=torch.float64, device=DEV)
    be = torch.empty(p.n, dtype=torch.float64, device=DEV)
    Nm = torch.empty(p.L * nt, dtype=torch.int32, device=DEV)
    import paper_2303_07597_gb300 as pk
    pk.ot_gs_get_screen_state(s.h, zt, ot, al, be, Nm)
    torch.cuda.synchronize()
    return (zt.cpu().numpy().reshape(p.L, nt * 32), ot.cpu().numpy().reshape(p.L, nt * 32),
            al.cpu().numpy(), be.cpu().numpy(), Nm.cpu().numpy().view(np.uint32).reshape(p.L, nt))


def _points(p, gamma, mu, seed):
    """A snapshot point x0 after a few oracle iterations and a nearby x1."""
    o = oracle.Oracle.from_problem(p, gamma, mu)
    r0 = o.solve(tol=1e-12, maxit=15)
    r1 = o.solve(tol=1e-12, maxit=25)
    return o, (r0["alpha"], r0["beta"]), (r1["alpha"], r1["beta"])


CASES = [
    ("tiny", lambda: synth.tiny(seed=0), 1.0, 0.1),
    ("ragged", lambda: synth.random_instance(300, 77, 7, seed=0), 0.7, 0.3),
    ("biggroups", lambda: synth.random_instance(513, 129, 3, seed=1), 1.0, 0.2),
    ("mixed", lambda: synth.random_instance(700, 96, 40, seed=4, min_size=0), 0.5, 0.5),
]


@pytest.mark.parametrize("name,mk,gamma,mu", CASES)
def test_screened_equals_dense_and_skip_set_matches_oracle(name, mk, gamma, mu):
    p = mk()
    o, x0, x1 = _points(p, gamma, mu, 0)
    s = solver(p, gamma, mu)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)
    s.snapshot(t(x0[0]), t(x0[1]), build_N=False)
    nt = (p.n + 31) // 32
    skip = torch.zeros(p.L * nt, dtype=torch.int32, device=DEV)
    out_s = s.grad_screened(t(x1[0]), t(x1[1]), skip_mask=skip)
    out_d = s.grad(t(x1[0]), t(x1[1]))
    torch.cuda.synchronize()
    # Thm. 2: identical results, bit for bit
    assert torch.equal(out_s, out_d), (out_s - out_d).abs().max().item()
    check_grad(out_s, o.dual(x1[0], x1[1]), x1[0], x1[1], p.a, p.b, name)
    # skip set == oracle replica of the rule on the GPU's stored snapshot
    zt, ot, als, bes, Nm = _state(s, p)
    assert np.allclose(als, x0[0], rtol=0, atol=0) and np.array_equal(bes, x0[1])
    sk_ref, _, cnt = o.gpu_screen_rule(x1[0], x1[1], als, bes, zt, ot, Nm)
    sk_gpu = skip.cpu().numpy().view(np.uint32).reshape(p.L, nt)
    assert np.array_equal(sk_gpu, sk_ref)
    assert cnt[2] > 0, "expected some skipped blocks"
    # safety (Lemma 2): every skipped block has z <= theta in exact FP64
    _, _, _, z, _ = o.dual(x1[0], x1[1], want_norms=True)
    bits = np.unpackbits(sk_gpu.view(np.uint8), bitorder="little").reshape(p.L, nt * 32)[:, :p.n].astype(bool)
    assert (z[bits] <= o.theta).all()
    # the paper's rule (Eq. 6 and Alg. 2 in FP64) on the same snapshot: every
    # block the GPU skips, it skips too; the blocks it skips and the GPU keeps
    # lie within the FP32 rule's rounding band (directed rounding and margin)
    zt64 = zt[:, :p.n].astype(np.float64)
    inN = np.unpackbits(Nm.view(np.uint8), bitorder="little").reshape(p.L, nt * 32)[:, :p.n].astype(bool)
    D64, ga64, gb64, sk64, _ = o.gradpsi(x1[0], x1[1], als, bes, zt64, inN.astype(np.uint8))
    assert not (bits & ~sk64).any()
    missed = sk64 & ~bits
    zbar, _ = o.bounds(x1[0], x1[1], als, bes, zt64, ot[:, :p.n].astype(np.float64))
    g = np.bincount(p.labels, minlength=p.L).astype(np.float64)
    band = np.ldexp(zbar, -21) + np.ldexp(g * zbar.max(), -23)[:, None] + np.ldexp(g, -20)[:, None]
    assert (zbar[missed] >= o.theta - band[missed]).all()
    print(f"{name}: paper rule skips {int(sk64.sum())} blocks, GPU {int(bits.sum())}, missed {int(missed.sum())}")
    # Alg. 2 in FP64 gives the dense result (Thm. 2), which the GPU matches
    check_grad(out_s, (D64, ga64, gb64), x1[0], x1[1], p.a, p.b, name + " (paper rule)")


@pytest.mark.parametrize("name,mk,gamma,mu", CASES[:3])
def test_N_rebuild_matches_oracle(name, mk, gamma, mu):
    p = mk()
    o, x0, x1 = _points(p, gamma, mu, 1)
    s = solver(p, gamma, mu)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)
    s.snapshot(t(x0[0]), t(x0[1]), build_N=False)
    zt0, ot0, als, bes, _ = _state(s, p)
    s.snapshot(t(x1[0]), t(x1[1]), build_N=True)
    _, _, _, _, Nm = _state(s, p)
    _, N_ref, _ = o.gpu_screen_rule(x1[0], x1[1], als, bes, zt0, ot0, None)
    assert np.array_equal(Nm, N_ref)
    # against the paper's Eq. 7 in FP64 on the same snapshot: differences only
    # where the FP64 lower bound is within the FP32 rounding band of theta
    nt = (p.n + 31) // 32
    N_gpu = np.unpackbits(Nm.view(np.uint8), bitorder="little").reshape(p.L, nt * 32)[:, :p.n].astype(bool)
    _, zlow = o.bounds(x1[0], x1[1], als, bes, zt0[:, :p.n].astype(np.float64), ot0[:, :p.n].astype(np.float64))
    g = np.bincount(p.labels, minlength=p.L).astype(np.float64)
    diff = N_gpu != (zlow > o.theta)
    band = np.ldexp(np.abs(zlow) + 4.0, -19) + np.ldexp(g, -18)[:, None]
    assert (np.abs(zlow[diff] - o.theta) <= band[diff]).all()
    print(f"{name}: |N| GPU {int(N_gpu.sum())}, FP64 {int((zlow > o.theta).sum())}, differ {int(diff.sum())}")
    # Lemma 4: every block of N has a nonzero gradient block (z > theta)
    _, _, _, z, _ = o.dual(x1[0], x1[1], want_norms=True)
    bits = np.unpackbits(Nm.view(np.uint8), bitorder="little").reshape(p.L, nt * 32)[:, :p.n]
    assert (z[bits.astype(bool)] > o.theta).all()


def test_snapshot_values_bound_the_exact_norms():
    """Stored z~ is an upper bound of the exact z (Def. 1; Lemma 1 needs no
    more): the exact value rounded up for the blocks whose FP32 bound does not
    rule out z > theta, the FP32 bound itself (above z by at most its stated
    error, ~2^-19 of |alpha| + |beta| per element) for the others; o~ ~
    exact."""
    p = synth.random_instance(400, 100, 5, seed=3)
    o = oracle.Oracle.from_problem(p, 1.0, 0.2)
    al, be = synth.random_duals(p.m, p.n, seed=4)
    s = solver(p, 1.0, 0.2)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)
    s.snapshot(t(al), t(be), build_N=False)
    zt, ot, _, _, _ = _state(s, p)
    _, _, _, z, oo = o.dual(al, be, want_norms=True)
    z32 = zt[:, :p.n].astype(np.float64)
    assert (z32 >= z * (1 - 1e-12)).all()
    g = np.bincount(p.labels, minlength=p.L).astype(np.float64)[:, None]
    M = np.abs(al).max() + np.abs(be).max()
    assert (z32 <= z * (1 + (g + 8) * 2.0 ** -23) + np.sqrt(g) * M * 2.0 ** -18 + 1e-30).all()
    near = z > o.theta * (1 - 1e-4)  # flagged: exact sums, rounded up
    assert near.sum() > 0 and np.allclose(z32[near], z[near], rtol=1e-6, atol=0)
    assert np.allclose(ot[:, :p.n], oo, rtol=1e-4, atol=1e-6)


def test_screened_items_whose_first_stages_are_not_sent():
    """Panels of 64 rows (m ceil(n/256) / 2048 = 64 here): a far class of 40
    rows, then a near class of 24.  At this point no far block has a positive
    part, so screening drops them and each work item's first 32-row stage
    holds no needed row and is not sent; the item's column data must come with
    its first stage that is.  Screened == dense bit for bit, and dense agrees
    with the oracle."""
    import paper_2303_07597_gb300 as pk
    p = synth.two_band(seed=3)
    assert pk.ot_gs_plan_info(p.labels, p.n, p.L)["n_panels"] == 64
    s = solver(p, 1.0, 0.1)
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0.0, 0.1, p.m)
    beta = rng.uniform(0.2, 0.4, p.n)
    al, be = torch.from_numpy(alpha).to(DEV), torch.from_numpy(beta).to(DEV)
    out_d = torch.empty(1 + p.m + p.n, dtype=torch.float64, device=DEV)
    out_s = torch.empty_like(out_d)
    s.snapshot(al, be, build_N=False, out=out_d)
    # a nearby point: the snapshot's bounds still drop every far block
    al2, be2 = al * (1 + 1e-3), be * (1 - 1e-3)
    pk.ot_gs_grad(s.h, al2, be2, out_d)
    s.grad_screened(al2, be2, out_s)
    torch.cuda.synchronize()
    assert torch.equal(out_d, out_s)
    st = s.stats()
    assert st["units_computed"] < st["units_total"]  # far units were skipped
    o = oracle.Oracle.from_problem(p, 1.0, 0.1)
    a2, b2 = al2.cpu().numpy(), be2.cpu().numpy()
    check_grad(out_s, o.dual(a2, b2), a2, b2, p.a, p.b, "two_band")
