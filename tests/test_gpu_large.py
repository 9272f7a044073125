"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the large workload (m = n = 20000, 1000 Zipf classes,
C = 1.6 GB) at the benchmark's evaluation point, every output against the
FP64 oracle; and the batched workload's 512 problems in one handle, a sample
of problems against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, check_grad

pytestmark = pytest.mark.gpu


def test_large_workload_every_output():
    p = synth.large(seed=0, device=DEV)
    gamma, mu = 1.0, 0.5
    C = torch.from_numpy(p.C).to(DEV)
    # the benchmark's point: alpha = 0, beta_j = 20th smallest c_ij + 1e-3
    beta = (torch.kthvalue(C, 20, dim=0).values.double() + 1e-3).contiguous()
    alpha = torch.zeros(p.m, dtype=torch.float64, device=DEV)
    s = pk.GroupSparseOT(C, torch.from_numpy(p.a).to(DEV), torch.from_numpy(p.b).to(DEV),
                         torch.from_numpy(p.labels).to(DEV), p.L, gamma, mu)
    out = s.grad(alpha, beta)
    torch.cuda.synchronize()
    al, be = alpha.cpu().numpy(), beta.cpu().numpy()
    o = oracle.Oracle.from_problem(p, gamma, mu)
    check_grad(out, o.dual(al, be), al, be, p.a, p.b, what="large")
    s.close()


def test_batched_workload_sampled_problems():
    probs = synth.batch(seed=0, nprob=512, device=DEV)
    gamma, mu = 1.0, 0.1
    devs = [(torch.from_numpy(q.C).to(DEV), torch.from_numpy(q.a).to(DEV), torch.from_numpy(q.b).to(DEV),
             torch.from_numpy(q.labels).to(DEV)) for q in probs]
    B = pk.GroupSparseOTBatch([d[0] for d in devs], [d[1] for d in devs], [d[2] for d in devs],
                              [d[3] for d in devs], [q.L for q in probs], gamma, mu)
    als, bes = [], []
    for k, q in enumerate(probs):
        a_, b_ = synth.random_duals(q.m, q.n, seed=1000 + k, scale=0.3, offset=0.3)
        als.append(a_)
        bes.append(b_)
    D, g = B.grad(torch.from_numpy(np.concatenate(als)).to(DEV), torch.from_numpy(np.concatenate(bes)).to(DEV))
    D, g = D.cpu().numpy(), g.cpu().numpy()
    for k in np.random.default_rng(0).choice(512, size=6, replace=False):
        q = probs[k]
        o = oracle.Oracle.from_problem(q, gamma, mu)
        outk = np.concatenate([[D[k]], g[B.row_off[k]:B.row_off[k + 1]], g[B.m + B.col_off[k]:B.m + B.col_off[k + 1]]])
        check_grad(torch.from_numpy(outk), o.dual(als[k], bes[k]), als[k], bes[k], q.a, q.b, what=q.name)
    B.close()
