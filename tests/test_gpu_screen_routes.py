"""The two routes of a screened evaluation (Alg. 2).  After the screen, either
the bound pass streams every needed tile of C and flags the blocks that may
have s > 0, or (few blocks left) the blocks the screen left are read straight
from the transposed copy of C.  The same exact-sum kernels form every block
with s > 0 on both routes, so each equals the dense evaluation bit for bit
(Thm. 2), whichever route the OTGS_DEBUG_SCREEN_ROUTE hook forces.  Checked
on classes of every height (split ones included), against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, check_grad, solver

pytestmark = pytest.mark.gpu


def _giant():
    rng = np.random.default_rng(5)
    sizes = np.array([4500, 30, 2, 300])
    XS, XT, lab = synth.mixture_features(sizes, 70, 3, rng)
    return synth.make_problem(XS, XT, lab, 4)


PROBLEMS = {
    "big_groups": lambda: synth.random_instance(513, 129, 3, seed=1),
    "giant_group": _giant,  # a class split across work items, one just above the slice height
    "many_small": lambda: synth.random_instance(700, 96, 40, seed=4, min_size=0),
    "mid_family": lambda: synth.mid(seed=2, m=1500, n=900, L=30, d=64),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("step", [1e-3, 3e-2])  # the evaluated point near the snapshot, farther away
def test_routes_equal_dense(name, step):
    p = PROBLEMS[name]()
    gamma, mu = 1.0, 0.2
    s = solver(p, gamma, mu)
    al, be = synth.random_duals(p.m, p.n, seed=3, scale=0.5, offset=0.2)
    a0, b0 = torch.from_numpy(al).to(DEV), torch.from_numpy(be).to(DEV)
    rng = np.random.default_rng(4)
    a1 = a0 + torch.from_numpy(rng.normal(scale=step, size=p.m)).to(DEV)
    b1 = b0 + torch.from_numpy(rng.normal(scale=step, size=p.n)).to(DEV)
    s.snapshot(a0, b0, build_N=False)
    s.snapshot(a0, b0, build_N=True)
    dense = s.grad(a1, b1).clone()
    nt = (p.n + 31) // 32
    skips = []
    for route in [1, 2, 0]:
        pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_SCREEN_ROUTE, route)
        skip = torch.empty(p.L * nt, dtype=torch.int32, device=DEV)
        out = s.grad_screened(a1, b1, skip_mask=skip)
        torch.cuda.synchronize()
        assert torch.equal(out, dense), (name, route)
        skips.append(skip.clone())
    assert torch.equal(skips[0], skips[1]) and torch.equal(skips[0], skips[2])
    a1n, b1n = a1.cpu().numpy(), b1.cpu().numpy()
    ref = oracle.Oracle.from_problem(p, gamma, mu).dual(a1n, b1n)
    check_grad(dense, ref, a1n, b1n, p.a, p.b, what=name)


def test_screened_solve_is_the_same_on_both_routes():
    """Alg. 1 with every evaluation on one route, then on the other: the same
    objective trace, bit for bit, as the dense solve."""
    p = synth.random_instance(900, 300, 8, seed=9)
    runs = []
    for screening, route in [(0, 0), (1, 1), (1, 2)]:
        s = solver(p, 1.0, 0.3)
        pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_SCREEN_ROUTE, route)
        s.set_params(use_screening=screening)
        s.solve(0.0, 80)
        D, t, ev = s.trace()
        runs.append(D)
        s.close()
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])


def test_route_switch_is_checked():
    p = synth.tiny()
    s = solver(p, 1.0, 0.1)
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_SCREEN_ROUTE, 3)
