"""Seeded synthetic inputs for group-sparse optimal transport.

This module is shared by the FP64 oracle (``oracle/``), the tests and the
benchmark.  It builds problem *inputs* only -- features, class labels,
marginals and the squared-Euclidean cost matrix -- and holds none of the
method's arithmetic (no dual objective, gradient, bound or solver step).

Every generator is seeded (numpy PCG64) and returns a :class:`Problem`:

* ``C``      float32 (m, n), row-major, C >= 0, scaled so that max(C) == 1
* ``labels`` int32 (m,), class of each source row, values in [0, L)
* ``a``, ``b`` float64 marginals, uniform 1/m and 1/n (Sec. 2.1)

Workloads (shapes follow the paper's domain-adaptation problems, Sec. 5.1):

* :func:`tiny`   m=n=200, 10 classes x 20 rows, d=10
* :func:`mid`    m=n=4000, 100 classes with Dirichlet(2) sizes, d=256
* :func:`large`  m=n=20000, 1000 classes with Zipf(1.1) sizes (min 2), d=512
* :func:`batch`  many independent problems, m, n ~ U[64, 2048], L ~ U[5, 100]
  with Dirichlet(2) sizes, d=64
* :func:`paper_synthetic` the paper's controlled-class data set (Sec. 5.1):
  d=2, g rows per class, class means (5l, -5) for sources and (5l, 5) for
  targets, unit Gaussian noise.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Problem", "class_sizes_dirichlet", "class_sizes_zipf", "labels_from_sizes",
    "mixture_features", "cost_matrix", "make_problem", "tiny", "mid", "large",
    "paper_synthetic", "random_duals", "random_instance", "batch",
]


@dataclasses.dataclass
class Problem:
    C: np.ndarray          # float32 (m, n)
    labels: np.ndarray     # int32 (m,)
    a: np.ndarray          # float64 (m,)
    b: np.ndarray          # float64 (n,)
    L: int
    name: str = ""
    XS: np.ndarray | None = None
    XT: np.ndarray | None = None

    @property
    def m(self) -> int:
        return int(self.C.shape[0])

    @property
    def n(self) -> int:
        return int(self.C.shape[1])


def _largest_remainder(total: int, weights: np.ndarray) -> np.ndarray:
    """Integer sizes summing to ``total`` proportional to ``weights``."""
    w = np.asarray(weights, dtype=np.float64)
    share = total * w / w.sum()
    base = np.floor(share).astype(np.int64)
    rem = total - int(base.sum())
    order = np.argsort(-(share - base), kind="stable")
    base[order[:rem]] += 1
    return base


def class_sizes_dirichlet(m: int, L: int, conc: float, rng: np.random.Generator,
                          min_size: int = 1) -> np.ndarray:
    """Class sizes: ``min_size`` each plus a largest-remainder share of the
    rest drawn from Dirichlet(conc * 1_L)."""
    p = rng.dirichlet(np.full(L, conc))
    return min_size + _largest_remainder(m - min_size * L, p)


def class_sizes_zipf(m: int, L: int, s: float, min_size: int = 2) -> np.ndarray:
    """Class sizes: ``min_size`` each plus a largest-remainder share of the
    rest proportional to k^-s (k = 1..L); deterministic."""
    w = np.arange(1, L + 1, dtype=np.float64) ** (-s)
    return min_size + _largest_remainder(m - min_size * L, w)


def labels_from_sizes(sizes: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)


def mixture_features(sizes: np.ndarray, n: int, d: int, rng: np.random.Generator,
                     mean_var: float = 4.0, shift_var: float = 0.25):
    """Gaussian-mixture source/target features.

    Source row of class l: mu_l + eps, mu_l ~ N(0, mean_var I), eps ~ N(0, I).
    Target: uniform class mix, x = mu_k + delta + eps with one domain shift
    delta ~ N(0, shift_var I)."""
    L = len(sizes)
    mu = rng.normal(0.0, np.sqrt(mean_var), size=(L, d))
    lab = labels_from_sizes(sizes)
    XS = mu[lab] + rng.normal(size=(int(sizes.sum()), d))
    delta = rng.normal(0.0, np.sqrt(shift_var), size=d)
    kt = rng.integers(0, L, size=n)
    XT = mu[kt] + delta + rng.normal(size=(n, d))
    return XS, XT, lab


def cost_matrix(XS: np.ndarray, XT: np.ndarray, device=None) -> np.ndarray:
    """Squared Euclidean cost c_ij = ||xS_i - xT_j||^2 (Sec. 2.1), computed
    in FP64, clamped at 0, scaled to max 1 and rounded once to float32.

    With ``device`` set (a torch device string) the FP64 product runs there;
    the result is returned as a host numpy array either way."""
    if device is None:
        XS = np.asarray(XS, dtype=np.float64)
        XT = np.asarray(XT, dtype=np.float64)
        sq = (XS * XS).sum(1)[:, None] + (XT * XT).sum(1)[None, :] - 2.0 * (XS @ XT.T)
        np.maximum(sq, 0.0, out=sq)
        sq /= sq.max()
        return sq.astype(np.float32)
    import torch
    xs = torch.as_tensor(np.asarray(XS, dtype=np.float64), device=device)
    xt = torch.as_tensor(np.asarray(XT, dtype=np.float64), device=device)
    sq = (xs * xs).sum(1)[:, None] + (xt * xt).sum(1)[None, :] - 2.0 * (xs @ xt.T)
    sq.clamp_(min=0.0)
    sq /= sq.max()
    out = sq.float().cpu().numpy()
    del xs, xt, sq
    return out


def make_problem(XS, XT, labels, L, name="", device=None, keep_features=False) -> Problem:
    C = cost_matrix(XS, XT, device=device)
    m, n = C.shape
    return Problem(C=C, labels=np.ascontiguousarray(labels, dtype=np.int32),
                   a=np.full(m, 1.0 / m), b=np.full(n, 1.0 / n), L=int(L), name=name,
                   XS=XS if keep_features else None, XT=XT if keep_features else None)


def _maybe_shuffle(p: Problem, shuffle_rows: bool, rng: np.random.Generator) -> Problem:
    if not shuffle_rows:
        return p
    perm = rng.permutation(p.m)
    p.C = np.ascontiguousarray(p.C[perm])
    p.labels = np.ascontiguousarray(p.labels[perm])
    if p.XS is not None:
        p.XS = p.XS[perm]
    return p


def tiny(seed: int = 0, shuffle_rows: bool = False, keep_features=False) -> Problem:
    """m=n=200; 10 classes x 20 rows; d=10; source N(mu_l, I) with
    mu_l ~ N(0, 4I); target N(0, 2I)."""
    rng = np.random.default_rng(seed)
    L, g, d = 10, 20, 10
    sizes = np.full(L, g)
    mu = rng.normal(0.0, 2.0, size=(L, d))
    lab = labels_from_sizes(sizes)
    XS = mu[lab] + rng.normal(size=(L * g, d))
    XT = rng.normal(0.0, np.sqrt(2.0), size=(L * g, d))
    p = make_problem(XS, XT, lab, L, name="tiny", keep_features=keep_features)
    return _maybe_shuffle(p, shuffle_rows, rng)


def mid(seed: int = 0, m: int = 4000, n: int = 4000, L: int = 100, d: int = 256,
        shuffle_rows: bool = False, device=None) -> Problem:
    """m=n=4000; 100 classes, sizes 1 + largest-remainder Dirichlet(2); d=256."""
    rng = np.random.default_rng(seed)
    sizes = class_sizes_dirichlet(m, L, 2.0, rng, min_size=1)
    XS, XT, lab = mixture_features(sizes, n, d, rng)
    p = make_problem(XS, XT, lab, L, name="mid", device=device)
    return _maybe_shuffle(p, shuffle_rows, rng)


def large(seed: int = 0, m: int = 20000, n: int = 20000, L: int = 1000, d: int = 512,
          device=None, shuffle_rows: bool = False, keep_features: bool = False) -> Problem:
    """m=n=20000; 1000 classes with Zipf(1.1) sizes (min 2); d=512; C is
    1.6 GB in float32.  Other sizes give smaller members of the same family."""
    rng = np.random.default_rng(seed)
    sizes = class_sizes_zipf(m, L, 1.1, min_size=2)
    XS, XT, lab = mixture_features(sizes, n, d, rng)
    p = make_problem(XS, XT, lab, L, name="large", device=device, keep_features=keep_features)
    return _maybe_shuffle(p, shuffle_rows, rng)


def two_band(seed: int = 0, pairs: int = 64, far_rows: int = 40, near_rows: int = 24, n: int = 8192) -> Problem:
    """Classes alternate between a "far" class of far_rows rows with costs in
    [0.9, 1) and a "near" class of near_rows rows with costs in [0, 0.5)
    (independent uniform draws), labels sorted.  At duals around 0.5 the far
    classes hold no positive part at all, so screening drops them whole."""
    rng = np.random.default_rng(seed)
    sizes = np.tile([far_rows, near_rows], pairs)
    lab = labels_from_sizes(sizes)
    far = np.repeat(np.tile([True, False], pairs), sizes)
    m = int(sizes.sum())
    C = np.where(far[:, None], rng.uniform(0.9, 1.0, (m, n)), rng.uniform(0.0, 0.5, (m, n))).astype(np.float32)
    return Problem(C=C, labels=lab, a=np.full(m, 1.0 / m), b=np.full(n, 1.0 / n), L=int(2 * pairs),
                   name="two_band")


def paper_synthetic(L: int, g: int = 10, seed: int = 0) -> Problem:
    """The paper's synthetic set (Sec. 5.1): d=2, g rows per class, class
    l (1-based) has source mean (5l, -5) and target mean (5l, 5), unit
    Gaussian noise, m = n = L*g.  Target classes only shape the data."""
    rng = np.random.default_rng(seed)
    lab = labels_from_sizes(np.full(L, g))
    ls = (lab + 1).astype(np.float64)
    XS = np.stack([5.0 * ls, np.full_like(ls, -5.0)], 1) + rng.normal(size=(L * g, 2))
    XT = np.stack([5.0 * ls, np.full_like(ls, 5.0)], 1) + rng.normal(size=(L * g, 2))
    return make_problem(XS, XT, lab, L, name=f"paper_synthetic_L{L}_g{g}")


def random_instance(m: int, n: int, L: int, seed: int = 0, d: int = 4,
                    min_size: int = 1, shuffle_rows: bool = True) -> Problem:
    """Small random instance with uneven class sizes (for parity/edge tests)."""
    rng = np.random.default_rng(seed)
    sizes = class_sizes_dirichlet(m, L, 1.0, rng, min_size=min_size)
    XS, XT, lab = mixture_features(sizes, n, d, rng)
    p = make_problem(XS, XT, lab, L, name=f"random_{m}x{n}_L{L}")
    return _maybe_shuffle(p, shuffle_rows, rng)


def batch(seed: int = 0, nprob: int = 512, m_range=(64, 2048), n_range=(64, 2048), L_range=(5, 100),
          d: int = 64, device=None) -> list:
    """Independent problems of uneven shape: m, n uniform in the given
    (inclusive) ranges, L uniform in L_range, class sizes 1 + largest-remainder
    Dirichlet(2) (0 + Dirichlet when m < L), d-dimensional mixture features
    as in :func:`mid`; labels sorted.  Problem k draws from its own stream
    (seed, k), so a prefix of a batch does not depend on nprob."""
    out = []
    for k in range(nprob):
        rng = np.random.default_rng([seed, k])
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        sizes = class_sizes_dirichlet(m, L, 2.0, rng, min_size=1 if m >= L else 0)
        XS, XT, lab = mixture_features(sizes, n, d, rng)
        out.append(make_problem(XS, XT, lab, L, name=f"batch{k}_{m}x{n}_L{L}", device=device))
    return out


def random_duals(m: int, n: int, seed: int = 0, scale: float = 0.5, offset: float = 0.3):
    """Random dual point (alpha, beta) in FP64 where a sizeable fraction of
    f = alpha_i + beta_j - c_ij is positive when C is scaled to [0, 1]."""
    rng = np.random.default_rng(seed)
    alpha = offset + scale * rng.standard_normal(m) * 0.5
    beta = offset + scale * rng.standard_normal(n) * 0.5
    return alpha.astype(np.float64), beta.astype(np.float64)
