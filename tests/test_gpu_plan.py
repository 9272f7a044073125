"""Downstream use of a solution: the transport plan (t = grad psi, Sec. 2.3,
Eq. 5) and the barycentric mapping n T^T X_S (Sec. 2.1) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shuffle", [False, True])
def test_plan_and_barycentric_match_oracle(shuffle):
    p = synth.tiny(seed=2, shuffle_rows=shuffle, keep_features=True)
    gamma, mu = 1.0, 0.1
    o = oracle.Oracle.from_problem(p, gamma, mu)
    r = o.solve(tol=1e-9, maxit=3000)
    s = solver(p, gamma, mu)
    al = torch.from_numpy(r["alpha"]).to(DEV)
    be = torch.from_numpy(r["beta"]).to(DEV)
    T = s.plan(al, be).cpu().numpy()
    To = o.plan(r["alpha"], r["beta"])
    assert np.max(np.abs(T - To)) <= 1e-6 * np.max(To)
    assert np.array_equal(T > 0, To > 0) or np.max(np.abs(T - To)[(T > 0) != (To > 0)]) <= 1e-7 * np.max(To)
    XS = np.asarray(p.XS, dtype=np.float32)
    Xm = s.barycentric(al, be, torch.from_numpy(XS).to(DEV)).cpu().numpy()
    ref = p.n * To.T @ XS.astype(np.float64)
    assert np.allclose(Xm, ref, rtol=1e-4, atol=1e-4 * np.max(np.abs(ref)))


def test_plan_at_random_point_and_strided_output():
    p = synth.random_instance(150, 90, 7, seed=4)
    o = oracle.Oracle.from_problem(p, 0.7, 0.3)
    al, be = synth.random_duals(p.m, p.n, seed=5, scale=0.6, offset=0.35)
    s = solver(p, 0.7, 0.3)
    buf = torch.full((p.m, p.n + 13), -1.0, dtype=torch.float32, device=DEV)
    s.plan(torch.from_numpy(al).to(DEV), torch.from_numpy(be).to(DEV), out=buf[:, :p.n])
    T = buf[:, :p.n].cpu().numpy()
    assert torch.all(buf[:, p.n:] == -1.0)
    To = o.plan(al, be)
    assert np.max(np.abs(T - To)) <= 1e-6 * np.max(To)
