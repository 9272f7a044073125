"""The learned warm start on the GPU: the network's forward pass, loss and
gradients, Adam and the input features against the FP64 oracle
(oracle/mlp.py, with the same bfloat16 operand rounding), and what the
trained network gains over the zero start on held-out problems."""
import numpy as np
import pytest
import torch

import paper_2303_07597_gb300 as pk
import synth
from oracle import mlp as omlp
from paper_2303_07597_gb300 import warmstart as ws

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def flat(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, np.atleast_1d(b3)]).astype(np.float32)


def random_params(K, H, seed):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, K)) * np.sqrt(6 / K)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6 / H)
    w3 = rng.uniform(-1, 1, H) * np.sqrt(3 / H)
    return [W1, rng.normal(0, 0.1, H), W2, rng.normal(0, 0.1, H), w3, np.array([0.07])]


def oracle_net(params):
    p32 = [np.asarray(x, dtype=np.float32).astype(np.float64) for x in params]  # the FP32 masters
    return omlp.MLP(*p32[:5], p32[5][0], bf16_ops=True)


@pytest.mark.parametrize("K,H,B", [(16, 16, 5), (144, 256, 1000), (48, 64, 777)])
def test_forward_loss_and_gradients_match_oracle(K, H, B):
    params = random_params(K, H, 1)
    net = pk.WarmStartMLP(K, H, max_batch=1024, seed=3)
    net.set_params(torch.from_numpy(flat(*params)).to(DEV))
    rng = np.random.default_rng(2)
    X = rng.normal(size=(B, K)).astype(np.float32)
    t = rng.normal(0.2, 0.3, size=B).astype(np.float32)
    y = net.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()
    loss, g = net.grad(torch.from_numpy(X).to(DEV), torch.from_numpy(t).to(DEV), want_grad=True)
    o = oracle_net(params)
    yo, _ = o.forward(X.astype(np.float64))
    lo, go = o.loss_and_grads(X.astype(np.float64), t.astype(np.float64))
    # FP32 accumulation against FP64; an activation next to a bfloat16 rounding
    # boundary may round to the other neighbour (2^-8 relative) on one side
    assert np.max(np.abs(y - yo)) <= 2e-3 * np.max(np.abs(yo)) + 1e-5
    assert abs(loss.item() - lo) <= 2e-3 * lo
    g = g.cpu().numpy()
    off = 0
    for name, ref in zip(["W1", "b1", "W2", "b2", "w3", "b3"], go):
        part = g[off:off + ref.size].reshape(ref.shape)
        off += ref.size
        assert np.max(np.abs(part - ref)) <= 5e-3 * np.max(np.abs(ref)) + 1e-7, name


def test_adam_step_matches_oracle():
    K, H, B = 32, 32, 200
    params = random_params(K, H, 4)
    net = pk.WarmStartMLP(K, H, max_batch=256, seed=5)
    net.set_params(torch.from_numpy(flat(*params)).to(DEV))
    rng = np.random.default_rng(6)
    X = rng.normal(size=(B, K)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    o = oracle_net(params)
    for step in (1, 2, 3):
        net.grad(torch.from_numpy(X).to(DEV), torch.from_numpy(t).to(DEV))
        net.adam(1e-2)
        _, go = o.loss_and_grads(X.astype(np.float64), t.astype(np.float64))
        if step == 1:
            mo = [np.zeros_like(p) for p in o.params()]
            vo = [np.zeros_like(p) for p in o.params()]
        omlp.adam_step(o.params(), go, mo, vo, step, lr=1e-2)
    p = net.params().cpu().numpy()
    ref = np.concatenate([x.ravel() for x in o.params()])
    # a step moves a parameter by about lr m / sqrt(v): where the gradients
    # agree to bfloat16 accuracy the updates agree to a fraction of lr; where
    # a gradient is near zero its sign (and the update) may differ
    dlt = np.abs(p - ref)
    assert dlt.max() <= 3 * 2 * 1e-2
    assert np.mean(dlt) <= 5e-4 and np.quantile(dlt, 0.99) <= 2e-3


def test_features_match_oracle():
    rng = np.random.default_rng(7)
    m, n, d, L = 53, 41, 8, 6
    sizes = np.array([10, 0, 20, 3, 15, 5])  # class 1 empty
    XS, XT, lab = synth.mixture_features(sizes, n, d, rng)
    p = synth.make_problem(XS, XT, lab, L, keep_features=True)
    K = ws.in_dim_for(d)
    F = ws.problem_features(p, DEV, K, 0.8).cpu().numpy()
    So, To = omlp.features(p.C, XS.astype(np.float32), XT.astype(np.float32), lab, L, 0.8, kpad=K)
    ref = np.concatenate([So, To])
    assert F.shape == ref.shape
    # stats in FP32 (sums of C in FP64, water levels by Newton steps),
    # class means rounded from FP64 sums
    assert np.allclose(F[:, :omlp.NSTAT], ref[:, :omlp.NSTAT], rtol=2e-6, atol=2e-7)
    assert np.allclose(F[:, omlp.NSTAT:], ref[:, omlp.NSTAT:], rtol=1e-6, atol=1e-7)


def test_batched_features_equal_per_problem_features():
    problems = [synth.large(seed=s, m=m, n=n, L=L, d=5, keep_features=True)
                for s, (m, n, L) in enumerate([(40, 33, 4), (64, 64, 5), (17, 90, 3)])]
    K = ws.in_dim_for(5)
    devp = [(torch.from_numpy(p.C).to(DEV), torch.from_numpy(np.ascontiguousarray(p.XS, dtype=np.float32)).to(DEV),
             torch.from_numpy(np.ascontiguousarray(p.XT, dtype=np.float32)).to(DEV),
             torch.from_numpy(p.labels).to(DEV)) for p in problems]
    F = pk.mlp_features_batch([q[0] for q in devp], [q[1] for q in devp], [q[2] for q in devp],
                              [q[3] for q in devp], [p.L for p in problems], 1.0, K)
    M = sum(p.m for p in problems)
    ro, co = 0, M
    for p, q in zip(problems, devp):
        Fk = pk.mlp_features(q[0], q[1], q[2], q[3], p.L, 1.0, K)
        assert torch.equal(F[ro:ro + p.m], Fk[:p.m])
        assert torch.equal(F[co:co + p.n], Fk[p.m:])
        ro += p.m
        co += p.n


def test_refine_features_match_oracle_and_touch_only_their_columns():
    """Second-pass inputs of a batch of two problems against the oracle, from
    a random first prediction: water levels against the other side's
    prediction (FP32 differences, Newton steps) and the own prediction; the
    other columns of the features keep their values."""
    problems = [synth.large(seed=s, m=m, n=n, L=L, d=4, keep_features=True)
                for s, (m, n, L) in enumerate([(45, 38, 4), (30, 61, 3)])]
    K = ws.in_dim_refine(4)
    col0 = ws.col_refine(4)
    devp = [(torch.from_numpy(p.C).to(DEV), torch.from_numpy(np.ascontiguousarray(p.XS, dtype=np.float32)).to(DEV),
             torch.from_numpy(np.ascontiguousarray(p.XT, dtype=np.float32)).to(DEV),
             torch.from_numpy(p.labels).to(DEV)) for p in problems]
    F = pk.mlp_features_batch([q[0] for q in devp], [q[1] for q in devp], [q[2] for q in devp],
                              [q[3] for q in devp], [p.L for p in problems], 0.9, K)
    F0 = F.clone()
    rng = np.random.default_rng(11)
    M, N = sum(p.m for p in problems), sum(p.n for p in problems)
    ah = rng.normal(0.2, 0.3, M).astype(np.float32)
    bh = rng.normal(-0.1, 0.3, N).astype(np.float32)
    pk.mlp_refine_features([q[0] for q in devp], torch.from_numpy(ah).to(DEV), torch.from_numpy(bh).to(DEV), 0.9,
                           col0, F)
    keep = [c for c in range(K) if not col0 <= c < col0 + omlp.NREF]
    assert torch.equal(F[:, keep], F0[:, keep])
    G = F.cpu().numpy()
    ro, co = 0, M
    for p in problems:
        So, To = omlp.refine_features(p.C, ah[ro:ro + p.m], bh[co - M:co - M + p.n], 0.9)
        assert np.allclose(G[ro:ro + p.m, col0:col0 + 4], So, rtol=2e-6, atol=2e-7)
        assert np.allclose(G[co:co + p.n, col0:col0 + 4], To, rtol=2e-6, atol=2e-7)
        ro += p.m
        co += p.n


def test_training_lowers_the_loss():
    K, H = 32, 64
    rng = np.random.default_rng(8)
    X = torch.from_numpy(rng.normal(size=(4096, K)).astype(np.float32)).to(DEV)
    w = rng.normal(size=K).astype(np.float32)
    t = torch.from_numpy(np.tanh(X.cpu().numpy() @ w / np.sqrt(K)).astype(np.float32)).to(DEV)
    net = pk.WarmStartMLP(K, H, max_batch=1024, seed=9)
    trace = ws.train(net, X, t, steps=400, batch=1024, lr=3e-3, lr_end=3e-4)
    assert trace[-1] < 0.25 * trace[0]


def test_shift_search_finds_the_best_shift():
    """The shift search maximises D(alpha + k, beta) over k: no k on a fine
    grid around its answer does better, and D never decreases."""
    problems = [synth.random_instance(120, 90, 6, seed=s, d=3) for s in (1, 2, 3)]
    B = ws.batch_of(problems, DEV, 1.0, 0.1)
    rng = np.random.default_rng(3)
    al = torch.from_numpy(rng.normal(0.3, 0.2, B.m)).to(DEV)
    be = torch.from_numpy(rng.normal(0.1, 0.2, B.n)).to(DEV)
    D0, _ = B.grad(al, be, with_grad=False)
    al2 = al.clone()
    B.shift(al2, be, 60)
    D1, _ = B.grad(al2, be, with_grad=False)
    assert torch.all(D1 >= D0)
    k = (al2 - al).cpu().numpy()
    for q in range(B.nprob):
        seg = k[B.row_off[q]:B.row_off[q + 1]]
        assert np.allclose(seg, seg[0], rtol=0, atol=1e-15)  # one shift per problem
    for dk in (-1e-3, -1e-5, 1e-5, 1e-3):
        D2, _ = B.grad(al2 + dk, be, with_grad=False)
        assert torch.all(D2 <= D1 + 1e-12 * D1.abs())


def test_warm_start_beats_zero_start_on_held_out_problems():
    """Train on solutions of problems from the Zipf-class generator family,
    then solve held-out problems of the family from the network's prediction
    (moved to its best shift) and from zero: the warm start needs fewer L-BFGS
    iterations on average to reach the same objective (within 1e-6 relative
    of the reference D*)."""
    gamma, mu, d = 1.0, 0.1, 8
    m = n = 192
    L = 10
    ntrain = 2048
    train_p = [synth.large(seed=100 + s, m=m, n=n, L=L, d=d, keep_features=True) for s in range(ntrain)]
    test_p = [synth.large(seed=90000 + s, m=m, n=n, L=L, d=d, keep_features=True) for s in range(16)]
    K = ws.in_dim_for(d)
    targets = []
    for c0 in range(0, ntrain, 512):
        _, tg, _ = ws.solve_targets(train_p[c0:c0 + 512], DEV, gamma, mu)
        targets += tg
    X, t = ws.dataset(train_p, targets, DEV, K, gamma)
    net = pk.WarmStartMLP(K, 256, max_batch=4096, seed=1)
    trace = ws.train(net, X, t, steps=6000, batch=4096, lr=1e-3, lr_end=1e-4)
    assert trace[-1] < 0.5 * trace[0]
    # held out: reference objectives, then cold and warm solves to D* within 1e-6
    B, _, ref = ws.solve_targets(test_p, DEV, gamma, mu)
    Dstar = ref["D"].copy()
    B.set_params(ftol=0.0)
    za = torch.zeros(B.m, dtype=torch.float64, device=DEV)
    zb = torch.zeros(B.n, dtype=torch.float64, device=DEV)
    B.set_state(za, zb)
    assert B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6) == pk.OTGS_OK
    cold = B.result(with_iterate=False)
    preds = ws.predict(net, test_p, DEV, K, gamma)
    al, be, used = ws.warm_state(B, preds)
    assert used.mean() >= 0.5
    B.set_state(al, be)
    assert B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6) == pk.OTGS_OK
    warm = B.result(with_iterate=False)
    assert np.all(warm["status"] == 0) and np.all(warm["D"] >= Dstar - 1e-6 * np.abs(Dstar))
    assert warm["iters"].mean() < 0.95 * cold["iters"].mean(), (warm["iters"], cold["iters"])
