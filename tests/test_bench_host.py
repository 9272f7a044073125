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


def test_clock_summary_keeps_the_samples_inside_the_timed_region():
    """NVML samples: only those between the marks count; the reason bits map
    to their names (sw_power_cap 0x4, hw_slowdown 0x8)."""
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler()
    cs.samples = [(0.0, 1000.0, 2070.0, 500.0, 0x8)] + \
        [(1.0 + 0.001 * k, 2070.0 - k, 2070.0, 1200.0, 0x4 if k == 2 else 0) for k in range(5)] + \
        [(9.0, 500.0, 2070.0, 300.0, 0x40)]
    cs.window = (0.9, 1.1)
    got = cs.summary()
    assert got["samples"] == 5 and got["sm_mhz"] == 2068.0 and got["reasons"] == ["sw_power_cap"]
    assert got["window"] == "inside the timed region"
    cs.window = (5.0, 5.0001)  # shorter than a sample period: the three nearest
    got = cs.summary()
    assert got["samples"] == 3 and "nearest 3" in got["window"]


def test_screened_needed_bytes_counts_the_unskipped_blocks():
    """C bytes of every block not skipped (rows of its class x 4 bytes), two
    words per unit (tile maximum of z~, word of N), z~ of the columns of the
    units with a block not skipped, and the duals with their snapshot values,
    from a skip mask of L x ceil(n/32) words (bit j % 32 of word j / 32)."""
    np = pytest.importorskip("numpy")
    sys.path.insert(0, ROOT)
    import bench
    L, n = 3, 40
    sizes = [5, 0, 7]
    mask = np.zeros((L, 2), dtype=np.uint32)
    mask[0, 0] = 0xFFFFFFFF          # class 0: columns 0..31 skipped
    mask[0, 1] = 0b101               # and 32, 34
    mask[2, 1] = 0xFFFFFFFF          # class 2: 32..39 skipped (bits past n ignored)
    need, c_need, nskip = bench.screened_needed_bytes(mask.ravel(), sizes, n, L)
    assert nskip == 34 + 8
    assert c_need == 4 * (5 * (40 - 34) + 7 * (40 - 8))
    # units with a block not skipped: (0, tile 1: 8 columns), (2, tile 0: 32)
    assert need == c_need + 4 * (8 + 32) + 8 * L * 2 + 16 * (12 + 40)
