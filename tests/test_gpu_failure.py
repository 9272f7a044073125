"""Failure paths of the library, made without faulting the GPU: invalid
inputs rejected at create, a non-finite start point, a failing evaluation
faked through a test hook (NaN objective from the k-th evaluation on), and
the evaluation kernel's bounded waits running out (a hook stops its consumer
warps from releasing stages; every wait has a limit, the producer waits for
the copies it issued, and the error reaches the result as NaN)."""
import time

import numpy as np
import pytest
import torch

import paper_2303_07597_gb300 as pk
import synth
from gpu_util import DEV, solver, to_dev

pytestmark = pytest.mark.gpu


def _create(C, a, b, lab, L, gamma=1.0, mu=0.1):
    return pk.GroupSparseOT(C, a, b, lab, L, gamma, mu)


def _code(fn):
    with pytest.raises(pk.OTGSError) as e:
        fn()
    return e.value.code


def test_create_rejects_a_nonfinite_cost():
    p = synth.tiny()
    C, a, b, lab = to_dev(p)
    for bad in [float("nan"), float("inf")]:
        C2 = C.clone()
        C2[17, 3] = bad
        assert _code(lambda: _create(C2, a, b, lab, p.L)) == pk.OTGS_ENONFINITE


def test_create_rejects_a_negative_cost():
    p = synth.tiny()
    C, a, b, lab = to_dev(p)
    C[5, 9] = -1e-3
    assert _code(lambda: _create(C, a, b, lab, p.L)) == pk.OTGS_EINVAL


def test_create_rejects_unbalanced_marginals():
    p = synth.tiny()
    C, a, b, lab = to_dev(p)
    assert _code(lambda: _create(C, a, b * 1.001, lab, p.L)) == pk.OTGS_EINVAL
    a2 = a.clone()
    a2[0] = 0.0  # a must be positive
    assert _code(lambda: _create(C, a2, b, lab, p.L)) == pk.OTGS_EINVAL


@pytest.mark.parametrize("bad", [-1, 10, 1 << 20])
def test_create_rejects_labels_out_of_range(bad):
    p = synth.tiny()  # L = 10
    C, a, b, lab = to_dev(p)
    lab[7] = bad
    assert _code(lambda: _create(C, a, b, lab, p.L)) == pk.OTGS_EINVAL


def test_create_rejects_bad_regularisation():
    p = synth.tiny()
    C, a, b, lab = to_dev(p)
    assert _code(lambda: _create(C, a, b, lab, p.L, gamma=0.0)) == pk.OTGS_EINVAL
    assert _code(lambda: _create(C, a, b, lab, p.L, mu=-0.1)) == pk.OTGS_EINVAL


def test_solve_from_a_nonfinite_start_reports_it():
    p = synth.tiny()
    s = solver(p, 1.0, 0.1)
    al = torch.zeros(p.m, dtype=torch.float64, device=DEV)
    al[3] = float("nan")
    s.set_state(al, torch.zeros(p.n, dtype=torch.float64, device=DEV))
    assert _code(lambda: s.solve(1e-8, 100)) == pk.OTGS_ENONFINITE


@pytest.mark.parametrize("screening", [0, 1])
def test_a_failing_evaluation_ends_the_line_search(screening):
    """From the 40th evaluation on the objective reads NaN: no step passes
    the line search, the solve stops with OTGS_ELINESEARCH at the last
    accepted iterate (finite, the trace's last entry) instead of looping."""
    p = synth.tiny()
    s = solver(p, 1.0, 0.1)
    s.set_params(use_screening=screening)
    pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_NAN_EVAL, 40)
    rc = s.solve(1e-12, 500)
    assert rc == pk.OTGS_ELINESEARCH
    sol = s.solution()
    D, t, ev = s.trace()
    assert sol["iters"] >= 1 and ev[-1] < 40
    assert np.isfinite(sol["D"]) and sol["D"] == D[-1]
    assert torch.isfinite(sol["alpha"]).all() and torch.isfinite(sol["beta"]).all()
    # the hook off again: the same handle solves normally from there
    pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_NAN_EVAL, 0)
    assert s.solve(1e-7, 2000) == pk.OTGS_OK


def test_debug_switches_are_checked():
    p = synth.tiny()
    s = solver(p, 1.0, 0.1)
    assert _code(lambda: pk.ot_gs_debug(s.h, 99, 1)) == pk.OTGS_EINVAL
    assert _code(lambda: pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_STALL, 10**11)) == pk.OTGS_EINVAL


def test_stalled_ring_times_out_and_reports():
    """The consumer warps stop releasing stages and the ring's waits give up
    after 2 ms: the kernel returns (the call ends in well under a second of
    device time), D is NaN, and the handle's error word stays set.  Another
    handle of the same problem is unaffected."""
    p = synth.random_instance(2000, 300, 5, seed=3)  # items of many stages
    al, be = synth.random_duals(p.m, p.n, seed=1, scale=0.5, offset=0.3)
    a_t, b_t = torch.from_numpy(al).to(DEV), torch.from_numpy(be).to(DEV)
    good = solver(p, 1.0, 0.1)
    want = good.grad(a_t, b_t).clone()
    s = solver(p, 1.0, 0.1)
    pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_STALL, 2_000_000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = s.grad(a_t, b_t)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert torch.isnan(out[0])
    pk.ot_gs_debug(s.h, pk.OTGS_DEBUG_STALL, 0)
    assert torch.isnan(s.grad(a_t, b_t)[0])  # sticky
    again = good.grad(a_t, b_t)
    torch.cuda.synchronize()
    assert torch.equal(again, want)
