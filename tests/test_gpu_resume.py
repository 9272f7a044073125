"""Checkpoint and resume of the device solver (Alg. 1's loop state): a solve
stopped after k iterations, saved, restored into a fresh handle of the same
problem and resumed follows the iterates of a solve that was never stopped,
bit for bit -- dense, and screened (the snapshot refresh every r iterations
and the set N carry over)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2303_07597_gb300 as pk
import synth
from gpu_util import solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("screening,k", [(0, 37), (1, 40), (1, 23)])
def test_resume_follows_the_uninterrupted_solve(screening, k):
    p = synth.random_instance(600, 400, 12, seed=21)
    gamma, mu, total = 1.0, 0.2, 90
    ref = solver(p, gamma, mu)
    ref.set_params(use_screening=screening)
    ref.solve(0.0, total)
    Dr, _, _ = ref.trace()
    solr = ref.solution()
    first = solver(p, gamma, mu)
    first.set_params(use_screening=screening)
    first.solve(0.0, k)
    buf = first.save_state()
    first.close()
    second = solver(p, gamma, mu)
    second.set_params(use_screening=screening)
    second.restore_state(buf)
    second.solve(0.0, total)
    D2, _, _ = second.trace()
    sol2 = second.solution()
    assert sol2["iters"] == solr["iters"] == total
    assert np.array_equal(D2, Dr[k:])  # entry 0 is the restored iterate
    assert torch.equal(sol2["alpha"], solr["alpha"]) and torch.equal(sol2["beta"], solr["beta"])
    assert sol2["D"] == solr["D"]
    # the optimum the resumed solve heads for is the oracle's
    o = oracle.Oracle.from_problem(p, gamma, mu)
    ro = o.solve(tol=1e-9, maxit=5000)
    assert sol2["D"] <= ro["D"] * (1 + 1e-12)


def test_restore_rejects_another_problem():
    p = synth.random_instance(100, 80, 4, seed=3)
    q = synth.random_instance(100, 81, 4, seed=3)
    a = solver(p, 1.0, 0.1)
    a.solve(0.0, 5)
    buf = a.save_state()
    b = solver(q, 1.0, 0.1)
    with pytest.raises(pk.OTGSError) as e:
        b.restore_state(buf)
    assert e.value.code == pk.OTGS_EINVAL
    c = solver(p, 1.0, 0.3)  # another mu
    with pytest.raises(pk.OTGSError):
        c.restore_state(buf)
