"""FP64 CPU oracle of the learned warm start: per-sample input features and
the 3-layer perceptron that maps them to initial duals.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it.  It shares no code with the CUDA path.

The paper has no learned component; this is the definition the project's
own kernels implement (plain numpy, FP64, written for reading).

Features (one row per sample; ``K = 9 + 2 d`` entries, zero-padded to a
multiple of 16 by the caller's choice of ``kpad``):

* source row i of class l:  [0, min_j c_ij, mean_j c_ij, softmin_0.02,
  softmin_0.1, g_l / m, wl_0.5, wl_1, wl_2, x_i (d), mu_l (d)]
* target column j:          [1, min_i c_ij, mean_i c_ij, softmin_0.02,
  softmin_0.1, g_k / m, wl_0.5, wl_1, wl_2, y_j (d), mu_k (d)]

where mu_l is the mean of class l's source features, g_l its size, k the
class whose mean is nearest to y_j (squared distance in FP32, terms added
in index order; ties to the lower class), softmin_tau over values v is
``-tau log(mean exp(-v / tau))`` and the water level wl_s over a row's
(column's) costs v is the L with sum [L - v]_+ = s gamma / m (s gamma / n):
with the other side's duals constant, the dual of a sample whose plan row
sums to its marginal under the squared-L2 regulariser alone.

Second pass (``refine_features``): four more inputs per sample from a first
prediction, the water levels against the other side's predicted duals and
the sample's own prediction.

Network (width H): Z1 = q(X) q(W1)^T + b1, A1 = relu(Z1),
Z2 = q(A1) q(W2)^T + b2, A2 = relu(Z2), y = q(A2) q(w3) + b3, with q the
round-to-nearest-even conversion to bfloat16 (the tensor-core operands) or
the identity (``bf16_ops=False``: exact FP64 arithmetic).  Loss L = mean_b
(y_b - t_b)^2.  Backward pass (the chain rule, with q at the same operand
positions): dy = 2 (y - t) / B, g_w3 = q(A2)^T dy, g_b3 = sum dy,
dZ2 = (dy q(w3)^T) * [Z2 > 0], g_W2 = q(dZ2)^T q(A1), g_b2 = sum_b dZ2,
dZ1 = (q(dZ2) q(W2)) * [Z1 > 0], g_W1 = q(dZ1)^T q(X), g_b1 = sum_b dZ1.
Adam (Kingma & Ba, 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

NSTAT = 9  # flag, min, mean, two softmins, class fraction, three water levels
WL = (0.5, 1.0, 2.0)
TAUS = (0.02, 0.1)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    bfloat16 keeps the upper 16 bits of an IEEE single; the input is first
    rounded to single precision (as the kernels hold it)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16
    nan = np.isnan(f)
    out = (r << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def softmin(v, tau, axis):
    v = np.asarray(v, dtype=np.float64)
    lo = v.min(axis=axis, keepdims=True)
    s = np.mean(np.exp(-(v - lo) / tau), axis=axis, keepdims=True)
    return np.squeeze(lo - tau * np.log(s), axis=axis)


def water_level(v, w):
    """The L with sum_k [L - v_k]_+ = w (w > 0): with v sorted, the level over
    the k smallest values, (w + v_1 + ... + v_k) / k, for the k where it falls
    between v_k and v_(k+1)."""
    v = np.sort(np.asarray(v, dtype=np.float64))
    cs = np.cumsum(v)
    for k in range(1, len(v) + 1):
        lev = (w + cs[k - 1]) / k
        if k == len(v) or lev <= v[k]:
            return lev
    raise AssertionError("unreachable")


def features(C, XS, XT, labels, L, gamma, kpad=None):
    """Per-sample inputs (source rows, then target columns) as float64
    arrays of shape (m, K) and (n, K)."""
    C = np.asarray(C, dtype=np.float64)
    XS = np.asarray(XS, dtype=np.float64)
    XT = np.asarray(XT, dtype=np.float64)
    lab = np.asarray(labels)
    m, n = C.shape
    d = XS.shape[1]
    K = NSTAT + 2 * d
    kp = K if kpad is None else int(kpad)
    assert kp >= K
    g = np.bincount(lab, minlength=L).astype(np.float64)
    mu = np.zeros((L, d))
    for l in range(L):
        if g[l] > 0:
            mu[l] = XS[lab == l].sum(0) / g[l]
    # nearest class mean of each target sample, decided in FP32: the squared
    # differences of the single-precision values added in index order
    mu32 = mu.astype(np.float32)
    xt32 = np.asarray(XT, dtype=np.float32)
    dist = np.full((n, L), np.inf, dtype=np.float32)
    for l in range(L):
        if g[l] > 0:
            acc = np.zeros(n, dtype=np.float32)
            for c in range(d):
                df = xt32[:, c] - mu32[l, c]
                acc = acc + df * df
            dist[:, l] = acc
    near = np.argmin(dist, axis=1)
    S = np.zeros((m, kp))
    S[:, 0] = 0.0
    S[:, 1] = C.min(1)
    S[:, 2] = C.mean(1)
    S[:, 3] = softmin(C, TAUS[0], 1)
    S[:, 4] = softmin(C, TAUS[1], 1)
    S[:, 5] = g[lab] / m
    for q, sc in enumerate(WL):
        S[:, 6 + q] = [water_level(C[i], sc * gamma / m) for i in range(m)]
    S[:, NSTAT:NSTAT + d] = XS
    S[:, NSTAT + d:K] = mu[lab]
    T = np.zeros((n, kp))
    T[:, 0] = 1.0
    T[:, 1] = C.min(0)
    T[:, 2] = C.mean(0)
    T[:, 3] = softmin(C, TAUS[0], 0)
    T[:, 4] = softmin(C, TAUS[1], 0)
    T[:, 5] = g[near] / m
    for q, sc in enumerate(WL):
        T[:, 6 + q] = [water_level(C[:, j], sc * gamma / n) for j in range(n)]
    T[:, NSTAT:NSTAT + d] = XT
    T[:, NSTAT + d:K] = mu[near]
    return S, T


NREF = 4  # second-pass inputs: three water levels against the other side's prediction, the own prediction


def refine_features(C, alpha_hat, beta_hat, gamma):
    """Second-pass inputs of the warm start, given a first prediction
    (alpha_hat, beta_hat): for source row i, the water levels wl_s of the
    values c_ij - beta_hat_j over j (masses s gamma / m, s in 0.5, 1, 2) and
    alpha_hat_i; for target column j, those of c_ij - alpha_hat_i over i
    (masses s gamma / n) and beta_hat_j.  With the other side's duals fixed
    at the prediction and the squared-L2 regulariser alone, wl_1 is the dual
    that makes the sample's plan row (column) sum to its marginal.  Returns
    (m, 4) and (n, 4) float64 arrays.  The differences are formed from the
    single-precision inputs (as the kernels read them) and rounded to single
    precision, as the kernels form them."""
    C32 = np.asarray(C, dtype=np.float32)
    ah = np.asarray(alpha_hat, dtype=np.float32)
    bh = np.asarray(beta_hat, dtype=np.float32)
    m, n = C32.shape
    S = np.zeros((m, NREF))
    T = np.zeros((n, NREF))
    VS = (C32 - bh[None, :]).astype(np.float64)  # FP32 differences, exactly widened
    VT = (C32 - ah[:, None]).astype(np.float64)
    for q, sc in enumerate(WL):
        S[:, q] = [water_level(VS[i], sc * gamma / m) for i in range(m)]
        T[:, q] = [water_level(VT[:, j], sc * gamma / n) for j in range(n)]
    S[:, 3] = ah
    T[:, 3] = bh
    return S, T


def gauge_fix(alpha, beta):
    """The duals shifted along D's invariant direction (alpha + k, beta - k)
    so that mean(alpha) = mean(beta)."""
    k = 0.5 * (np.mean(beta) - np.mean(alpha))
    return alpha + k, beta - k


class MLP:
    """Parameters as float64 arrays: W1 (H, K), b1 (H,), W2 (H, H), b2 (H,),
    w3 (H,), b3 (1,)."""

    def __init__(self, W1, b1, W2, b2, w3, b3, bf16_ops=True):
        self.W1 = np.array(W1, dtype=np.float64)
        self.b1 = np.array(b1, dtype=np.float64)
        self.W2 = np.array(W2, dtype=np.float64)
        self.b2 = np.array(b2, dtype=np.float64)
        self.w3 = np.array(w3, dtype=np.float64)
        self.b3 = np.array(b3, dtype=np.float64).reshape(1)
        self.q = bf16 if bf16_ops else (lambda a: np.asarray(a, dtype=np.float64))

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.w3, self.b3]

    def forward(self, X):
        q = self.q
        Z1 = q(X) @ q(self.W1).T + self.b1
        A1 = np.maximum(Z1, 0.0)
        Z2 = q(A1) @ q(self.W2).T + self.b2
        A2 = np.maximum(Z2, 0.0)
        y = q(A2) @ q(self.w3) + self.b3[0]
        return y, (Z1, A1, Z2, A2)

    def loss_and_grads(self, X, t):
        """Mean squared error and its gradients [W1, b1, W2, b2, w3, b3]."""
        q = self.q
        X = np.asarray(X, dtype=np.float64)
        t = np.asarray(t, dtype=np.float64)
        B = X.shape[0]
        y, (Z1, A1, Z2, A2) = self.forward(X)
        r = y - t
        loss = float(np.mean(r * r))
        dy = 2.0 * r / B
        g_w3 = q(A2).T @ dy
        g_b3 = float(dy.sum())
        dZ2 = np.outer(dy, q(self.w3)) * (Z2 > 0)
        g_W2 = q(dZ2).T @ q(A1)
        g_b2 = dZ2.sum(0)
        dZ1 = (q(dZ2) @ q(self.W2)) * (Z1 > 0)
        g_W1 = q(dZ1).T @ q(X)
        g_b1 = dZ1.sum(0)
        return loss, [g_W1, g_b1, g_W2, g_b2, g_w3, np.array([g_b3])]


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of every array in params, in place;
    m, v are the moment arrays (same shapes, updated in place)."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= b1
        mm += (1.0 - b1) * g
        vv *= b2
        vv += (1.0 - b2) * g * g
        mh = mm / (1.0 - b1 ** t)
        vh = vv / (1.0 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
