"""Column shards (the multi-GPU split of the dual, Eq. 4-5) through the
product path: each shard handle (ot_gs_create_shard) holds C[:, J_p] and
b_Jp and evaluates its part on the GPU; the host combines them the way one
sum across GPUs would (D = sum D_p - (P - 1) alpha.a, grad_alpha = sum of the
shards' - (P - 1) a, grad_beta the shards' own), and the result matches the
FP64 oracle's unsharded evaluation.  One GPU runs the shards one after the
other; the cross-process sum itself is covered by the gloo test."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, check_grad

pytestmark = pytest.mark.gpu


def _shards(p, parts):
    return np.array_split(np.arange(p.n), parts)


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("screened", [False, True])
def test_shards_add_up_to_the_full_evaluation(parts, screened):
    p = synth.random_instance(700, 301, 9, seed=31)  # ragged shards crossing 32-column tiles
    gamma, mu = 1.0, 0.2
    al, be = synth.random_duals(p.m, p.n, seed=32, scale=0.5, offset=0.3)
    a_t = torch.from_numpy(al).to(DEV)
    lab = torch.from_numpy(p.labels).to(DEV)
    a = torch.from_numpy(p.a).to(DEV)
    D = -(parts - 1) * float(al @ p.a)
    ga = -(parts - 1) * p.a
    gb = np.zeros(p.n)
    for J in _shards(p, parts):
        C = torch.from_numpy(np.ascontiguousarray(p.C[:, J])).to(DEV)
        s = pk.GroupSparseOT(C, a, torch.from_numpy(p.b[J]).to(DEV), lab, p.L, gamma, mu, shard=True)
        b_t = torch.from_numpy(np.ascontiguousarray(be[J])).to(DEV)
        if screened:  # a snapshot at a nearby point, then a screened evaluation (Alg. 2) of the shard
            s.snapshot(a_t + 1e-3, b_t - 1e-3, build_N=True)
            out = s.grad_screened(a_t, b_t).cpu().numpy()
        else:
            out = s.grad(a_t, b_t).cpu().numpy()
        D += out[0]
        ga = ga + out[1:1 + p.m]
        gb[J] = out[1 + p.m:]
        s.close()
    ref = oracle.Oracle.from_problem(p, gamma, mu).dual(al, be)
    full = torch.from_numpy(np.concatenate([[D], ga, gb]))
    check_grad(full, ref, al, be, p.a, p.b, what=f"{parts} shards")


def test_a_shard_is_not_solved_alone():
    p = synth.random_instance(200, 60, 4, seed=33)
    J = np.arange(30)
    s = pk.GroupSparseOT(torch.from_numpy(np.ascontiguousarray(p.C[:, J])).to(DEV), torch.from_numpy(p.a).to(DEV),
                         torch.from_numpy(p.b[J]).to(DEV), torch.from_numpy(p.labels).to(DEV), p.L, 1.0, 0.1,
                         shard=True)
    with pytest.raises(pk.OTGSError) as e:
        s.solve(1e-8, 10)
    assert e.value.code == pk.OTGS_EINVAL
    # the same columns as a whole problem are refused (unbalanced marginals)
    with pytest.raises(pk.OTGSError):
        pk.GroupSparseOT(torch.from_numpy(np.ascontiguousarray(p.C[:, J])).to(DEV), torch.from_numpy(p.a).to(DEV),
                         torch.from_numpy(p.b[J]).to(DEV), torch.from_numpy(p.labels).to(DEV), p.L, 1.0, 0.1)
