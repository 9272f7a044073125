"""The column-sharded multi-GPU design, simulated with two gloo ranks on CPU.

Target columns are independent blocks of the dual: rank p holds C[:, J_p]
and beta_{J_p} and evaluates its shard; one all-reduce (a sum) of the row
plan sums and of the scalar partials gives the full objective and alpha
gradient, and each rank's beta gradient is local.  Every box here has one
GPU, so the design is checked with the oracle standing in for each rank's
evaluation: the sharded result must equal the unsharded one."""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.random_instance(60, 47, 5, seed=21)
        al, be = synth.random_duals(p.m, p.n, seed=22)
        J = np.array_split(np.arange(p.n), world)[rank]  # this rank's columns
        shard = synth.Problem(C=np.ascontiguousarray(p.C[:, J]), labels=p.labels, a=p.a, b=p.b[J], L=p.L,
                              name=f"shard{rank}")
        o = oracle.Oracle.from_problem(shard, 1.0, 0.1)
        D_p, ga_p, gb_p = o.dual(al, be[J])
        # the shard's own terms: beta_J.b_J - psi_J, and -T_J 1 (alpha.a and a counted once, below)
        part = torch.from_numpy(np.concatenate([[D_p - al @ p.a], ga_p - p.a]))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        D = al @ p.a + float(part[0])
        ga = p.a + part[1:].numpy()
        gb = [None] * world
        dist.all_gather_object(gb, (J.tolist(), gb_p.tolist()))
        if rank == 0:
            G = np.zeros(p.n)
            for cols, vals in gb:
                G[cols] = vals
            q.put((D, ga.tolist(), G.tolist()))
    finally:
        dist.destroy_process_group()


def test_column_shards_add_up_to_the_full_evaluation():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    D, ga, gb = q.get(timeout=10)
    p = synth.random_instance(60, 47, 5, seed=21)
    al, be = synth.random_duals(p.m, p.n, seed=22)
    D0, ga0, gb0 = oracle.Oracle.from_problem(p, 1.0, 0.1).dual(al, be)
    assert abs(D - D0) <= 1e-12 * (abs(al @ p.a) + abs(be @ p.b) + abs(D0))
    assert np.allclose(ga, ga0, rtol=0, atol=1e-13)
    assert np.array_equal(np.asarray(gb), gb0)  # column blocks are independent: bit for bit
