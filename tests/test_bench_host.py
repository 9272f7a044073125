"""Host logic of bench.py on CPU: the multi-process side over two gloo ranks
(the benchmark runs one replica per GPU over NCCL; the timing reduction and
the whole-job throughput are the same host logic), and the clock record."""
import os
import socket
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        slowest = bench.max_over_ranks(times[rank], "cpu")
        dist.barrier()
        q.put((rank, slowest, bench.job_throughput(100, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_every_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 20.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, thr in got:
        assert slowest == 20.0  # both ranks see the slowest rank's time
        assert thr == pytest.approx(100 * 2 / 0.020)  # all ranks' steps over that time


def test_single_process_is_its_own_maximum():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_throughput(10, 1, 500.0) == pytest.approx(20.0)


def test_clock_summary_reads_the_samples_and_the_throttle_reasons(tmp_path):
    """The clocks record of a bench line: median SM clock of the samples, the
    largest max clock seen, and every throttle reason that was Active."""
    sys.path.insert(0, ROOT)
    import bench
    path = tmp_path / "clocks.csv"
    path.write_text("2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    cs = bench.ClockSampler()
    cs.f = open(path)
    got = cs.summary()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()  # the sample file is removed once read
