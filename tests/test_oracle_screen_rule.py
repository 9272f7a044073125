"""Pins of the oracle's FP32 screening rule (``Oracle.gpu_screen_rule``)
against the paper's rule evaluated in FP64 (``Oracle.bounds``).

The FP32 rule is Eq. 6 with every operation rounded toward +inf and a skip
threshold lowered by a margin tau_l, and Eq. 7 rounded to nearest.  The
paper's rule is Eq. 6 / Eq. 7 in exact arithmetic (FP64 here).  What the
pins fix, on random snapshot / current pairs with groups of 1 to 200 rows and
mixed-sign changes of alpha and beta:

* soundness (Lemma 1-2 survive the rounding): a block the FP32 rule skips
  has an FP64 upper bound at most theta - tau_l / 2, so the paper's rule
  skips it too;
* completeness up to the rounding: a block whose FP64 upper bound is below
  theta by more than the FP32 error bound of the expression (plus tau_l) is
  skipped by the FP32 rule;
* the set N (Def. 3): the FP32 rule's set and the FP64 set differ only on
  blocks whose FP64 lower bound lies within the FP32 error bound of theta;
* exactness: on dyadic inputs where every FP32 operation is exact, the FP32
  rule decides exactly as the paper's rule, except on ties zbar == theta,
  which the paper skips (zbar <= theta) and the margin keeps.

A dropped term, a wrong sign of a change, or sqrt(g) in place of g moves
some bound by far more than these bands and fails a pin.  CPU only.
"""
import numpy as np
import pytest

import oracle
import synth


def _problem(sizes, n, seed):
    rng = np.random.default_rng(seed)
    lab = synth.labels_from_sizes(np.asarray(sizes))
    m = len(lab)
    C = rng.uniform(0.0, 1.0, (m, n)).astype(np.float32)
    return synth.Problem(C=C, labels=lab, a=np.full(m, 1.0 / m), b=np.full(n, 1.0 / n), L=len(sizes))


def _bits(words, n):
    """uint32 (L, ntiles) words -> bool (L, n) (bit j % 32 of word j // 32)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    return np.unpackbits(w.view(np.uint8), bitorder="little").reshape(w.shape[0], -1)[:, :n].astype(bool)


def _group_stats(p, al, als):
    """FP64 ||[dalpha_l]_+||, ||dalpha_l||, ||[dalpha_l]_-|| and g_l."""
    d = al - als
    L = p.L
    npos = np.sqrt(np.bincount(p.labels, weights=np.maximum(d, 0) ** 2, minlength=L))
    nneg = np.sqrt(np.bincount(p.labels, weights=np.minimum(d, 0) ** 2, minlength=L))
    nabs = np.sqrt(np.bincount(p.labels, weights=d * d, minlength=L))
    g = np.bincount(p.labels, minlength=L).astype(np.float64)
    return npos, nabs, nneg, g


def _tau(p, o, al, be, als, bes, g):
    M = (np.abs(al).max().astype(np.float32).astype(np.float64) + np.abs(be).max() + np.abs(als).max()
         + np.abs(bes).max() + float(p.C.max()))
    return np.ldexp(np.sqrt(g) * M * (1 + 1e-6) + g * o.theta, -36)


CASES = [
    # (class sizes, n, seed, gamma, mu, scale of the change)
    ([1, 2, 5, 31, 32, 33, 64, 200, 17, 3], 70, 0, 1.0, 0.5, 0.05),
    ([1] * 12 + [40, 7], 100, 1, 0.7, 0.3, 0.02),
    ([100, 150, 3, 9], 33, 2, 2.0, 0.1, 0.004),
]


@pytest.mark.parametrize("sizes,n,seed,gamma,mu,scale", CASES)
def test_fp32_rule_against_paper_rule_random(sizes, n, seed, gamma, mu, scale):
    p = _problem(sizes, n, seed)
    o = oracle.Oracle.from_problem(p, gamma, mu)
    rng = np.random.default_rng(100 + seed)
    theta = o.theta
    als = rng.normal(0.3, 0.2, p.m)
    bes = rng.normal(0.3, 0.2, p.n)
    al = als + scale * rng.standard_normal(p.m)
    be = bes + scale * rng.standard_normal(p.n)
    npos, nabs, nneg, g = _group_stats(p, al, als)
    sg = np.sqrt(g)
    db = be - bes
    # snapshot values spread across theta so that the decisions are not trivial
    zt = rng.uniform(0.0, 2.0 * theta, (p.L, p.n)).astype(np.float32)
    ot = rng.uniform(0.0, 2.0 * theta, (p.L, p.n)).astype(np.float32)
    ldz = (p.n + 31) // 32 * 32
    zt_p = np.zeros((p.L, ldz), np.float32)
    ot_p = np.zeros((p.L, ldz), np.float32)
    zt_p[:, :p.n], ot_p[:, :p.n] = zt, ot
    skip_w, N_w, cnt = o.gpu_screen_rule(al, be, als, bes, zt_p, ot_p, None)
    skip32, N32 = _bits(skip_w, p.n), _bits(N_w, p.n)
    zbar, zlow = o.bounds(al, be, als, bes, zt.astype(np.float64), ot.astype(np.float64))
    tau = _tau(p, o, al, be, als, bes, g)[:, None]
    # soundness: FP32 skips => the paper's rule skips, with the margin to spare
    assert (zbar[skip32] <= theta - 0.5 * np.broadcast_to(tau, zbar.shape)[skip32]).all()
    # completeness up to the FP32 error bound of Eq. 6 (directed rounding,
    # sums of g squares): a relative 2^-21 of the whole bound plus
    # (g + 12) 2^-23 of the group norm
    band_up = np.ldexp(zbar, -21) + np.ldexp((g + 12.0) * npos, -23)[:, None] + tau
    must = zbar <= theta - band_up
    assert (skip32[must]).all()
    assert must.sum() > 0.2 * zbar.size and (~skip32).sum() > 0.2 * zbar.size
    undecided = ~must & (zbar <= theta)
    assert undecided.sum() <= 0.02 * zbar.size
    # N (Eq. 7, Def. 3): differences only within the rounding band of theta
    kt = np.sqrt(zt.astype(np.float64) ** 2 + ot.astype(np.float64) ** 2)
    terms = (kt + nabs[:, None] + sg[:, None] * np.abs(db)[None, :] + ot
             + nneg[:, None] + sg[:, None] * np.maximum(-db, 0)[None, :])
    band_lo = np.ldexp(terms, -20) + np.ldexp((g + 12.0) * (nabs + nneg), -23)[:, None]
    N64 = zlow > theta
    diff = N32 != N64
    assert (np.abs(zlow[diff] - theta) <= band_lo[diff]).all()
    assert N64.sum() > 0 and (~N64).sum() > 0
    # the counts the rule reports are those of its masks
    assert cnt[0] == 0 and cnt[1] == p.L * p.n and cnt[2] == skip32.sum()


def test_fp32_rule_in_N_blocks_are_not_checked():
    """Blocks of the input set N are computed without a check (Alg. 2's first
    loop): never skipped, counted apart."""
    p = _problem([3, 40, 1, 9], 45, 5)
    o = oracle.Oracle.from_problem(p, 1.0, 0.5)
    rng = np.random.default_rng(6)
    als = rng.normal(0.3, 0.2, p.m)
    bes = rng.normal(0.3, 0.2, p.n)
    ldz = 64
    zt = np.zeros((p.L, ldz), np.float32)  # every block would be skipped
    ot = np.zeros((p.L, ldz), np.float32)
    Nm = np.zeros((p.L, 2), np.uint32)
    Nm[1, 0] = 0xF0F0F0F0
    Nm[2, 1] = 0x1FFF  # columns 32..44
    skip_w, _, cnt = o.gpu_screen_rule(als, bes, als, bes, zt, ot, Nm)
    skip = _bits(skip_w, p.n)
    inN = _bits(Nm, p.n)
    assert not (skip & inN).any()
    assert skip[~inN].all()
    assert cnt[0] == inN.sum() and cnt[1] == (~inN).sum() and cnt[2] == skip.sum()


@pytest.mark.parametrize("with_o", [False, True])
def test_fp32_rule_exact_on_dyadic_inputs(with_o):
    """Every FP32 operation exact: groups of perfect-square sizes (sqrt(g)
    exact), one changed row per group (the group norms are that change),
    changes and snapshot values on a 2^-7 grid, (z~, o~) from the triple
    (4, 3, 5) so k~ is exact.  Then the FP32 rule equals the paper's rule on
    every block, except ties zbar == theta: skipped by the paper (zbar <=
    theta), kept by the margin."""
    sizes = [1, 4, 9, 16, 36, 64]
    n = 70
    p = _problem(sizes, n, 7)
    o = oracle.Oracle.from_problem(p, 1.0, 0.5)  # theta = 0.5
    theta = o.theta
    rng = np.random.default_rng(8)
    q = 2.0 ** -7
    als = rng.integers(-40, 40, p.m) * q
    bes = rng.integers(-40, 40, p.n) * q
    dal = np.zeros(p.m)
    goff = np.concatenate([[0], np.cumsum(sizes)])
    for l in range(p.L):
        dal[rng.integers(goff[l], goff[l + 1])] = rng.integers(-12, 13) * q
    al = als + dal
    be = bes + rng.integers(-6, 7, p.n) * q
    npos, nabs, nneg, g = _group_stats(p, al, als)
    sg = np.sqrt(g)
    dbp = np.maximum(be - bes, 0)
    s = rng.integers(0, 60 if with_o else 22, (p.L, n)) * q
    zt = 4 * s if with_o else 6 * s
    ot = 3 * s if with_o else np.zeros_like(s)
    # force ties zbar == theta on a quarter of the blocks where z~ can take them
    tie = theta - npos[:, None] - sg[:, None] * dbp[None, :]
    force = (rng.uniform(size=zt.shape) < 0.25) & (tie >= 0)
    zt = np.where(force, tie, zt)
    ot = np.where(force, 0.0, ot)
    ldz = 96
    zt_p = np.zeros((p.L, ldz), np.float32)
    ot_p = np.zeros((p.L, ldz), np.float32)
    zt_p[:, :n], ot_p[:, :n] = zt, ot
    assert np.array_equal(zt_p[:, :n].astype(np.float64), zt)  # representable
    skip_w, N_w, _ = o.gpu_screen_rule(al, be, als, bes, zt_p, ot_p, None)
    skip32, N32 = _bits(skip_w, n), _bits(N_w, n)
    zbar, zlow = o.bounds(al, be, als, bes, zt, ot)
    ties = zbar == theta
    assert ties.sum() > 20
    assert np.array_equal(skip32[~ties], (zbar <= theta)[~ties])
    assert not skip32[ties].any()
    assert np.array_equal(N32, zlow > theta)
    assert (zlow > theta).sum() > 10 and (zbar < theta).sum() > 10
