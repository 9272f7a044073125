"""Learned warm start for the batched solver (no counterpart in the paper).

The network (:class:`WarmStartMLP`, the library's own kernels) maps each
sample's features (``mlp_features``: cost statistics, its features and its
class-mean embedding) to its dual variable.  Targets are the solver's own
solutions, each side anchored to the mean of its samples' water levels (D
depends on alpha_i + beta_j only, so a common level is not learnable; the
shift search sets it at solve time).  An optional second network also sees
water levels against the first one's prediction (``mlp_refine_features``).
At solve time the prediction is used only when it is better than the zero
start (D above D(0, 0) = 0); otherwise the solve starts from zero, so the
zero-start solver stays the fallback.  Either way the solve runs to the
same stopping rule and reaches the same objective.

Tensors are PyTorch CUDA tensors (plumbing); features, network and solves
run in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import GroupSparseOTBatch, WarmStartMLP, mlp_features, mlp_features_batch, mlp_refine_features

NSTAT = 9


def in_dim_for(d: int) -> int:
    """Feature width for d-dimensional sample features, rounded up to 16."""
    return (NSTAT + 2 * d + 15) // 16 * 16


NREF = 4  # second-pass inputs per sample (three water levels, the own prediction)


def col_refine(d: int) -> int:
    """First feature column of the second-pass inputs."""
    return NSTAT + 2 * d


def in_dim_refine(d: int) -> int:
    """Feature width with room for the second-pass inputs, rounded up to 16."""
    return (NSTAT + 2 * d + NREF + 15) // 16 * 16


def gauge_fix(alpha, beta):
    """alpha + k, beta - k with mean(alpha) = mean(beta) (tensors)."""
    k = 0.5 * (beta.mean() - alpha.mean())
    return alpha + k, beta - k


def problem_features(p, device, in_dim, gamma):
    """Features of a synth.Problem (with XS, XT) on the device: (m + n, in_dim)."""
    import torch
    C = torch.from_numpy(p.C).to(device)
    XS = torch.from_numpy(np.ascontiguousarray(p.XS, dtype=np.float32)).to(device)
    XT = torch.from_numpy(np.ascontiguousarray(p.XT, dtype=np.float32)).to(device)
    lab = torch.from_numpy(p.labels).to(device)
    return mlp_features(C, XS, XT, lab, p.L, gamma, in_dim)


def batch_of(problems, device, gamma, mu):
    import torch
    Cs = [torch.from_numpy(p.C).to(device) for p in problems]
    As = [torch.from_numpy(p.a).to(device) for p in problems]
    Bs = [torch.from_numpy(p.b).to(device) for p in problems]
    Ls = [torch.from_numpy(p.labels).to(device) for p in problems]
    return GroupSparseOTBatch(Cs, As, Bs, Ls, [p.L for p in problems], gamma, mu)


def solve_targets(problems, device, gamma, mu, tol=1e-9, maxit=20000, ftol=1e-14):
    """Solve the problems together; returns the batch handle and per problem
    (alpha, beta) as float64 tensors, gauge-fixed, and D."""
    B = batch_of(problems, device, gamma, mu)
    B.set_params(ftol=ftol)
    B.solve(tol=tol, maxit=maxit)
    r = B.result()
    out = []
    for k in range(len(problems)):
        al, be = gauge_fix(B.split(r["alpha"], k, "alpha"), B.split(r["beta"], k, "beta"))
        out.append((al, be))
    return B, out, r


WL1 = 7  # feature column of the water level wl_1


def dataset(problems, targets, device, in_dim, gamma):
    """Rows of features and their target duals for every sample of every
    problem.  Only alpha + beta enters D, and the start point's common level
    is set by the shift search, so each side's targets are anchored to a
    level the features carry: mean(alpha) = mean of the rows' wl_1, mean(beta)
    = mean of the columns' wl_1.  What is left to learn is each side's shape."""
    import torch
    Xs, ts = [], []
    for p, (al, be) in zip(problems, targets):
        F = problem_features(p, device, in_dim, gamma)
        Xs.append(F)
        ta = al - al.mean() + F[:p.m, WL1].double().mean()
        tb = be - be.mean() + F[p.m:, WL1].double().mean()
        ts.append(torch.cat([ta, tb]).float())
    return torch.cat(Xs), torch.cat(ts)


def dataset_refine(problems, targets, device, in_dim, gamma, net1):
    """Rows for a second network: each problem's features with the
    second-pass inputs (water levels against the other side's prediction,
    the own prediction) from net1's prediction, and the targets of
    :func:`dataset`."""
    import torch
    d = problems[0].XS.shape[1]
    Xs, ts = [], []
    for p, (al, be) in zip(problems, targets):
        F = problem_features(p, device, in_dim, gamma)
        y = net1.forward(F)
        C = torch.from_numpy(p.C).to(device)
        mlp_refine_features([C], y[:p.m].contiguous(), y[p.m:].contiguous(), gamma, col_refine(d), F)
        Xs.append(F)
        ta = al - al.mean() + F[:p.m, WL1].double().mean()
        tb = be - be.mean() + F[p.m:, WL1].double().mean()
        ts.append(torch.cat([ta, tb]).float())
    return torch.cat(Xs), torch.cat(ts)


def train(net: WarmStartMLP, X, t, steps=2000, batch=4096, lr=1e-3, lr_end=1e-4, seed=0):
    """Adam on random minibatches (learning rate decayed geometrically from lr
    to lr_end); returns the loss trace (one value per 50 steps)."""
    import torch
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    batch = min(batch, n, net.max_batch)
    trace = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), device=X.device, generator=g)
        rate = lr * (lr_end / lr) ** (s / max(1, steps - 1))
        loss = net.train_step(X[idx].contiguous(), t[idx].contiguous(), rate)
        if s % 50 == 0 or s == steps - 1:
            trace.append(float(loss.item()))
    return trace


def predict(net: WarmStartMLP, problems, device, in_dim, gamma):
    """Predicted (alpha, beta) per problem, gauge-fixed, float64."""
    out = []
    for p in problems:
        y = net.forward(problem_features(p, device, in_dim, gamma)).double()
        out.append(gauge_fix(y[:p.m], y[p.m:]))
    return out


def predict_batch(net: WarmStartMLP, dev_problems, Ls, in_dim, gamma, timings=None):
    """Predicted (alpha, beta) of many problems in the batch layout, from one
    features launch and one pass of the network over all samples.
    dev_problems: (C, XS, XT, labels) device tensors per problem.  With a
    dict ``timings``, the device is synchronised after each part and the
    features and network times (ms) are recorded there."""
    import time
    import torch
    t0 = time.perf_counter()
    F = mlp_features_batch([q[0] for q in dev_problems], [q[1] for q in dev_problems],
                           [q[2] for q in dev_problems], [q[3] for q in dev_problems], Ls, gamma, in_dim)
    if timings is not None:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        timings["features_ms"] = (t1 - t0) * 1e3
    y = net.forward(F).double()
    if timings is not None:
        torch.cuda.synchronize()
        timings["network_ms"] = (time.perf_counter() - t1) * 1e3
    M = sum(int(q[0].shape[0]) for q in dev_problems)
    return y[:M].contiguous(), y[M:].contiguous()


def predict_batch_refine(net1: WarmStartMLP, net2: WarmStartMLP, dev_problems, Ls, in_dim, gamma):
    """Two passes: net1 on the features, then net2 on the features with the
    second-pass inputs from net1's prediction (the feature width must leave
    room for them: :func:`in_dim_refine`)."""
    F = mlp_features_batch([q[0] for q in dev_problems], [q[1] for q in dev_problems],
                           [q[2] for q in dev_problems], [q[3] for q in dev_problems], Ls, gamma, in_dim)
    M = sum(int(q[0].shape[0]) for q in dev_problems)
    y1 = net1.forward(F)
    d = int(dev_problems[0][1].shape[1])
    mlp_refine_features([q[0] for q in dev_problems], y1[:M].contiguous(), y1[M:].contiguous(), gamma,
                        col_refine(d), F)
    y = net2.forward(F).double()
    return y[:M].contiguous(), y[M:].contiguous()


def warm_state(B: GroupSparseOTBatch, preds, shift_iters=20):
    """Concatenated start point for the batch: each problem's prediction
    when its D beats the zero start's D(0, 0) = 0; if some problem's does
    not, all predictions are first moved to the best point on their line
    (alpha + k, beta) by the library's shift search; a problem whose D still
    does not beat zero starts from zero.  preds: per problem (alpha, beta), or
    the two concatenated vectors.  Returns (alpha, beta, used) with used[k]
    telling which problems start warm."""
    import torch
    if isinstance(preds, tuple) and len(preds) == 2 and preds[0].numel() == B.m:
        al, be = preds[0].clone(), preds[1].clone()
    else:
        al = torch.cat([a for a, _ in preds]).contiguous()
        be = torch.cat([b for _, b in preds]).contiguous()
    D, _ = B.grad(al, be, with_grad=False)
    used = D.cpu().numpy() > 0.0
    if shift_iters > 0 and not used.all():
        B.shift(al, be, shift_iters)
        D, _ = B.grad(al, be, with_grad=False)
        used = D.cpu().numpy() > 0.0
    if not used.all():
        keep_r = torch.from_numpy(np.repeat(used, np.diff(B.row_off))).to(al.device)
        keep_c = torch.from_numpy(np.repeat(used, np.diff(B.col_off))).to(be.device)
        al = torch.where(keep_r, al, torch.zeros_like(al))
        be = torch.where(keep_c, be, torch.zeros_like(be))
    return al, be, used
