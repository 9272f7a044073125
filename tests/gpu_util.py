"""Shared helpers of the GPU tests: seeded problems on the device and the
tolerances the comparisons use."""
import os

import numpy as np
import torch

import paper_2303_07597_gb300 as pk

DEV = "cuda:0"


def to_dev(p):
    C = torch.from_numpy(p.C).to(DEV)
    a = torch.from_numpy(p.a).to(DEV)
    b = torch.from_numpy(p.b).to(DEV)
    lab = torch.from_numpy(p.labels).to(DEV)
    return C, a, b, lab


def solver(p, gamma, mu):
    C, a, b, lab = to_dev(p)
    return pk.GroupSparseOT(C, a, b, lab, p.L, gamma, mu)


# Every checked result's errors against the oracle (listed at the end of the run).
RESULTS = []


def check_grad(out, ref, alpha, beta, a, b, what=""):
    """Objective within 1e-9 relative to |D| (and to the magnitude of its
    terms alpha.a, beta.b, sum psi; where |D| is below 1e-3 of that, a
    cancellation, the terms' scale alone); gradient entries within 1e-5 of
    max(|g_i|, a_i) (marginal scale).  Returns the errors and records them."""
    D, ga, gb = ref
    out = out.cpu().numpy()
    Dg, gag, gbg = out[0], out[1:1 + len(a)], out[1 + len(a):]
    scale = abs(alpha @ a) + abs(beta @ b) + abs(alpha @ a + beta @ b - D)
    dD = abs(Dg - D)
    rel_D = dD / abs(D) if D != 0 else (0.0 if dD == 0 else float("inf"))
    assert dD <= 1e-9 * max(scale, 1e-300), (what, Dg, D, scale)
    assert rel_D <= 1e-9 or abs(D) < 1e-3 * scale, (what, Dg, D, rel_D)
    ea = np.abs(gag - ga) / np.maximum(np.abs(ga), a)
    eb = np.abs(gbg - gb) / np.maximum(np.abs(gb), b)
    assert ea.max() <= 1e-5, (what, ea.max(), int(ea.argmax()))
    assert eb.max() <= 1e-5, (what, eb.max(), int(eb.argmax()))
    res = dict(D_rel_terms=dD / max(scale, 1e-300), D_rel=rel_D, ga_rel=float(ea.max()), gb_rel=float(eb.max()))
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    RESULTS.append(dict(test=test, what=what, **res))
    return res
