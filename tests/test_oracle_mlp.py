"""Pins of the warm-start oracle (oracle/mlp.py) to things other than
itself: the bfloat16 format's definition, central finite differences of the
loss, Adam's closed form after one step, and the definitions of the
per-sample features on small cases checked by brute force."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp


def test_bf16_rounding_follows_the_format():
    # bfloat16 keeps 7 fraction bits: spacing 2^-7 on [1, 2)
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0                         # halfway: to the even neighbour
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6           # halfway: to the even neighbour
    assert mlp.bf16(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7    # above halfway
    assert mlp.bf16(-(1.0 + 2 ** -8 + 2 ** -20)) == -(1.0 + 2 ** -7)
    assert mlp.bf16(3.0e38) == np.inf or mlp.bf16(3.0e38) > 3.0e38 * 0.99
    assert mlp.bf16(2.0 ** -130) == 2.0 ** -130                   # subnormal, exactly representable
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) + 1e-45)
    # representable values are fixed points
    assert np.array_equal(mlp.bf16(r), r)


def _rand_net(K, H, seed, bf16_ops=False):
    rng = np.random.default_rng(seed)
    return mlp.MLP(rng.normal(0, 1 / np.sqrt(K), (H, K)), rng.normal(0, 0.1, H),
                   rng.normal(0, 1 / np.sqrt(H), (H, H)), rng.normal(0, 0.1, H),
                   rng.normal(0, 1 / np.sqrt(H), H), 0.05, bf16_ops=bf16_ops)


def test_exact_gradients_match_central_differences():
    K, H, B = 7, 6, 9
    net = _rand_net(K, H, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(B, K))
    t = rng.normal(size=B)
    loss, grads = net.loss_and_grads(X, t)
    h = 1e-6
    for p, g in zip(net.params(), grads):
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + h
            lp, _ = net.loss_and_grads(X, t)
            p[idx] = old - h
            lm, _ = net.loss_and_grads(X, t)
            p[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_bf16_gradients_are_the_exact_ones_to_bf16_accuracy():
    K, H, B = 32, 16, 64
    ex = _rand_net(K, H, 3, bf16_ops=False)
    q = _rand_net(K, H, 3, bf16_ops=True)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(B, K))
    t = rng.normal(size=B)
    le, ge = ex.loss_and_grads(X, t)
    lq, gq = q.loss_and_grads(X, t)
    assert abs(le - lq) <= 0.03 * le
    for a, b in zip(ge, gq):
        assert np.max(np.abs(a - b)) <= 0.05 * np.max(np.abs(a)) + 1e-12


def test_linear_regime_is_a_matrix_product():
    """With every pre-activation positive the network is affine: y = X W1^T
    W2^T w3 + (b1 W2^T + b2) . w3 + b3."""
    K, H = 5, 4
    rng = np.random.default_rng(5)
    W1 = np.abs(rng.normal(size=(H, K)))
    W2 = np.abs(rng.normal(size=(H, H)))
    net = mlp.MLP(W1, np.ones(H), W2, np.ones(H), rng.normal(size=H), 0.3, bf16_ops=False)
    X = np.abs(rng.normal(size=(6, K)))
    y, _ = net.forward(X)
    ref = X @ W1.T @ W2.T @ net.w3 + (np.ones(H) @ W2.T + np.ones(H)) @ net.w3 + 0.3
    assert np.allclose(y, ref, rtol=1e-14, atol=1e-14)


def test_adam_first_step_closed_form():
    """After one step from zero moments the bias-corrected moments are g and
    g^2: each parameter moves by lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    m, v = [np.zeros(4)], [np.zeros(4)]
    mlp.adam_step([p], [g], m, v, 1, lr=0.1, eps=1e-8)
    assert np.allclose(p, 1.0 - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-15, atol=1e-15)


def test_features_by_brute_force():
    rng = np.random.default_rng(6)
    m, n, d, L = 7, 5, 3, 4
    XS = rng.normal(size=(m, d))
    XT = rng.normal(size=(n, d))
    lab = np.array([0, 0, 2, 2, 2, 3, 0])  # class 1 empty
    C = rng.uniform(size=(m, n))
    gamma = 0.7
    S, T = mlp.features(C, XS, XT, lab, L, gamma, kpad=32)
    assert S.shape == (m, 32) and T.shape == (n, 32)
    for i in range(m):
        l = lab[i]
        mu = XS[lab == l].mean(0)
        row = C[i]
        sm = [-tau * np.log(np.mean(np.exp(-row / tau))) for tau in mlp.TAUS]
        wl = [_level_bisect(row, s * gamma / m) for s in mlp.WL]
        ref = [0.0, row.min(), row.mean(), sm[0], sm[1], (lab == l).sum() / m, *wl, *XS[i], *mu]
        assert np.allclose(S[i, :len(ref)], ref, rtol=1e-12, atol=1e-12)
        assert np.all(S[i, len(ref):] == 0)
    for j in range(n):
        cand = [l for l in range(L) if (lab == l).any()]
        dist = [np.sum((XT[j] - XS[lab == l].mean(0)) ** 2) for l in cand]
        k = cand[int(np.argmin(dist))]
        col = C[:, j]
        sm = [-tau * np.log(np.mean(np.exp(-col / tau))) for tau in mlp.TAUS]
        wl = [_level_bisect(col, s * gamma / n) for s in mlp.WL]
        ref = [1.0, col.min(), col.mean(), sm[0], sm[1], (lab == k).sum() / m, *wl, *XT[j], *XS[lab == k].mean(0)]
        assert np.allclose(T[j, :len(ref)], ref, rtol=1e-12, atol=1e-12)


def _level_bisect(v, w):
    """sum [L - v]_+ = w by bisection (a method independent of the oracle's sort)."""
    lo, hi = v.min(), v.min() + w
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(mid - v, 0).sum() < w:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_water_level_closed_forms():
    # one value: L = v + w; equal values: L = v + w / k; the level solves its equation
    assert mlp.water_level([0.3], 0.2) == pytest.approx(0.5, abs=1e-15)
    assert mlp.water_level([0.1] * 4, 0.2) == pytest.approx(0.15, abs=1e-15)
    v = np.random.default_rng(9).uniform(size=37)
    for w in (1e-4, 0.05, 3.0):
        lev = mlp.water_level(v, w)
        assert np.maximum(lev - v, 0).sum() == pytest.approx(w, rel=1e-12)


def _newton_level_f32(v, w, max_steps=32):
    """The feature kernels' water-level method, step for step in FP32:
    Newton from L = min + w (where sum [L - v]_+ >= w) on the convex,
    piecewise-linear sum, stopping when the sum no longer exceeds w or L
    stops decreasing."""
    v = np.asarray(v, dtype=np.float32)
    w = np.float32(w)
    L = np.float32(v.min() + w)
    for _ in range(max_steps):
        d = L - v
        pos = d > 0
        f = np.float32(d[pos].sum(dtype=np.float32)) - w
        if not f > 0:
            break
        Ln = np.float32(L - f / np.float32(pos.sum()))
        if not Ln < L:
            break
        L = Ln
    return float(L)


@pytest.mark.parametrize("seed", range(6))
def test_newton_water_level_reaches_the_sorted_level(seed):
    """The kernels' method (Newton steps from the right) against the
    oracle's sort-based level: equal to FP32 accuracy within a few steps, on
    spread, clustered, tied and single-valued inputs and masses from tiny to
    larger than the spread."""
    rng = np.random.default_rng(seed)
    cases = [rng.uniform(size=256), rng.exponential(0.05, size=200), np.round(rng.uniform(size=64), 1),
             np.full(17, 0.25), np.array([0.7]), np.concatenate([rng.normal(0.5, 1e-3, 50), [0.0]])]
    for v in cases:
        v32 = np.asarray(v, dtype=np.float32)
        for w in (1e-6, 1e-3, 0.05, 1.0, 10.0):
            ref = mlp.water_level(v32.astype(np.float64), float(np.float32(w)))
            got = _newton_level_f32(v32, w)
            assert abs(got - ref) <= 4e-7 * max(1.0, abs(ref)), (seed, len(v), w, got, ref)


def test_softmin_between_min_and_mean():
    v = np.random.default_rng(7).uniform(size=(3, 50))
    for tau in (1e-3, 0.02, 0.1, 10.0):
        s = mlp.softmin(v, tau, 1)
        assert np.all(s >= v.min(1) - 1e-15) and np.all(s <= v.mean(1) + 1e-15)
    assert np.allclose(mlp.softmin(v, 1e-4, 1), v.min(1), atol=1e-3)
    assert np.allclose(mlp.softmin(np.full((2, 9), 0.3), 0.05, 1), 0.3, rtol=1e-15)


def test_gauge_fix_keeps_the_dual_objective():
    p = synth.tiny()
    o = oracle.Oracle.from_problem(p, 1.0, 0.1)
    al, be = synth.random_duals(p.m, p.n, seed=3)
    a2, b2 = mlp.gauge_fix(al, be)
    assert abs(np.mean(a2) - np.mean(b2)) < 1e-15
    D1 = o.dual(al, be)[0]
    D2 = o.dual(a2, b2)[0]
    assert abs(D1 - D2) <= 1e-13 * abs(D1)


def test_refine_features_reduce_to_the_base_levels_and_shift_with_the_prediction():
    """Second-pass inputs: against zero predictions the water levels are the
    first pass's (the same values, the same masses); a constant prediction k
    on the other side moves every level by -k (sum [L - (v - k)]_+ = sum
    [(L + k) - v]_+); the last column is the sample's own prediction."""
    rng = np.random.default_rng(4)
    m, n, d, L = 23, 17, 3, 4
    sizes = np.array([8, 6, 0, 9])
    XS, XT, lab = synth.mixture_features(sizes, n, d, rng)
    p = synth.make_problem(XS, XT, lab, L, keep_features=True)
    S0, T0 = mlp.features(p.C, XS, XT, lab, L, 0.7)
    Sz, Tz = mlp.refine_features(p.C, np.zeros(m), np.zeros(n), 0.7)
    assert np.array_equal(Sz[:, :3], S0[:, 6:9]) and np.array_equal(Tz[:, :3], T0[:, 6:9])
    ah = rng.normal(size=m)
    Sk, Tk = mlp.refine_features(p.C, ah, np.full(n, 0.375), 0.7)
    assert np.allclose(Sk[:, :3], S0[:, 6:9] - 0.375, atol=1e-7)
    assert np.array_equal(Sk[:, 3], ah.astype(np.float32).astype(np.float64))
    assert np.array_equal(Tk[:, 3], np.full(n, 0.375))
