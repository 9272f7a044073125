"""Benchmark: dual gradient evaluations per second of group-sparse OT on GB300.

One step = one evaluation of the dual objective D and its gradient (Eq. 4-5)
over the whole workload, through the library's C ABI.  Default workload: m = n
= 20000, 1000 classes with Zipf(1.1) sizes (min 2), d = 512 Gaussian-mixture
features, C FP32 (1.6 GB) squared-Euclidean scaled to max 1, gamma = 1,
mu = 0.5, synthetic and seeded.  C is larger than L2, so no flush is needed.

Beside the step (1 GPU): the same workload solved from zero to a relative
objective error of 1e-6, dense and screened (Alg. 1), with one dense and one
screened evaluation timed at the iterate where the solve gets there; the
batched workload; the learned warm start.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload on its GPU (the single-problem path is not sharded).
``--impl reference`` times the FP64 CPU oracle on host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "dual grad evals/s"
UNIT = "evals/s"

L2_BYTES = 129 * 1024 * 1024  # GB300's L2

WORKLOADS = {
    "large": dict(m=20000, n=20000, L=1000, d=512, gamma=1.0, mu=0.5),
    # the large generator at a quarter of the size (C = 400 MB, still larger
    # than L2): the case profiles are captured on
    "large10k": dict(m=10000, n=10000, L=500, d=512, gamma=1.0, mu=0.5),
    "mid": dict(m=4000, n=4000, L=100, d=256, gamma=1.0, mu=0.1),
    "tiny": dict(m=200, n=200, L=10, d=10, gamma=1.0, mu=0.1),
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _make_workload(name, seed, device):
    import torch
    cfg = WORKLOADS[name]
    if name == "tiny":
        p = synth.tiny(seed=seed)
    elif name == "mid":
        p = synth.mid(seed=seed, device=device)
    else:
        c = WORKLOADS[name]
        p = synth.large(seed=seed, m=c["m"], n=c["n"], L=c["L"], d=c["d"], device=device)
    C = torch.from_numpy(p.C).to(device)
    return p, C, cfg


def max_over_ranks(x, device):
    """The largest of the ranks' values x (every rank gets it); x itself
    when no process group runs or it has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, slowest_ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (replicas of the same work on every rank)."""
    return units_per_rank * world / (slowest_ms / 1000.0)


def _eval_point(C, k):
    """A dual point like those met mid-solve: alpha = 0 and beta_j just above
    the k-th smallest cost of column j, so about k entries of f are positive
    per column (input construction, not part of the method)."""
    import torch
    beta = torch.kthvalue(C.double(), k, dim=0).values + 1e-3
    alpha = torch.zeros(C.shape[0], dtype=torch.float64, device=C.device)
    return alpha, beta.contiguous()


class _Nvml:
    """Read-only NVML queries through ctypes: SM clock, its maximum, power
    draw and the active clock event reasons of one GPU (by UUID)."""

    # clock event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, uuid):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev)) != 0:
            raise RuntimeError("no NVML device for " + uuid)
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(v)) != 0:
            raise RuntimeError("nvmlDeviceGetMaxClockInfo failed")
        self.max_sm = float(v.value)

    def sample(self):
        c = self.c
        sm, mw, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, c.byref(sm)) != 0:  # NVML_CLOCK_SM
            return None
        self.lib.nvmlDeviceGetPowerUsage(self.dev, c.byref(mw))
        self.reasons_fn(self.dev, c.byref(rs))
        return float(sm.value), self.max_sm, mw.value / 1000.0, int(rs.value)

    def close(self):
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """SM clock and throttle reasons sampled during a region.

    With NVML (read through ctypes), a thread samples every 2 ms and the
    region is marked by ``mark(True)`` / ``mark(False)`` around the timed
    work: the summary keeps the samples inside the marks (at least the three
    nearest to the region when it is shorter than that).  Without NVML,
    ``nvidia-smi -lms 100`` writes the samples to a file that the summary
    reads (CSV: sm, max sm, power, reasons bitmask, then the four reasons
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.002

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.nvml = None
        self.samples = []   # (host time, sm MHz, max sm MHz, W, reasons bitmask)
        self.window = None  # host times of the marks
        self._t0 = None
        self._stop = None
        self.thread = None

    def __enter__(self):
        import threading
        if self.uuid:
            try:
                self.nvml = _Nvml(self.uuid)
            except Exception:
                self.nvml = None
        if self.nvml is not None:
            self._stop = threading.Event()

            def run():
                while not self._stop.is_set():
                    r = self.nvml.sample()
                    if r is not None:
                        self.samples.append((time.perf_counter(),) + r)
                    time.sleep(self.PERIOD_S)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            time.sleep(0.02)
            return self
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def mark(self, start):
        t = time.perf_counter()
        if start:
            self._t0 = t
        else:
            self.window = (self._t0, t)

    def __exit__(self, *a):
        if self.thread is not None:
            time.sleep(0.01)
            self._stop.set()
            self.thread.join(timeout=5)
            self.nvml.close()
            return
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()

    def _summary_nvml(self):
        rows = self.samples
        where = "all samples"
        if self.window:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if len(inside) >= 3:
                rows, where = inside, "inside the timed region"
            else:
                mid = 0.5 * (t0 + t1)
                rows = sorted(rows, key=lambda r: abs(r[0] - mid))[:3]
                where = f"{len(inside)} inside the timed region, nearest 3 used"
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for bit, nm in _Nvml.REASONS.items():
                if r[4] & bit:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "source": "nvml, every 2 ms",
                "window": where, "power_w_median": statistics.median(r[3] for r in rows)}

    def summary(self):
        if self.samples:
            return self._summary_nvml()
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
            os.unlink(self.f.name)
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_for(kernel_src_hash, workload):
    """Per-launch DRAM bytes of the evaluation kernel from a committed ncu
    summary, only when it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
        e = t.get(workload)
        if e and e.get("src_sha1") == kernel_src_hash:
            return e.get("bytes_per_launch")
    except Exception:
        pass
    return None


def _src_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2303_07597_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in ("otgs_eval.cu", "otgs_stream.cu", "otgs_plan.cu", "otgs_internal.cuh"):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()


def cpu_baseline(p, alpha, beta, gamma, mu, budget_s=10.0, ncols=None):
    """FP64 oracle dense evaluation on a column sample (all rows, the first
    ncols columns; the cost is linear in columns), scaled to the workload."""
    import oracle
    n = p.n
    if ncols is None:
        ncols = max(1, min(n, int(4e7 // p.m)))
    o = oracle.Oracle(np.ascontiguousarray(p.C[:, :ncols]), p.labels, p.a, p.b[:ncols], p.L, gamma, mu)
    reps, t0 = 0, time.perf_counter()
    while True:
        o.dual(alpha, beta[:ncols])
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 1000:
            break
    per = el / reps * (n / ncols)
    return {"value": 1.0 / per, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} dense FP64 evaluations on all {p.m} rows x {ncols} of {n} columns "
                      f"({el:.1f} s), scaled by n/{ncols}"}


def _timed(fn, k, stream):
    """Mean device time (ms) of k calls of fn, CUDA events on the launching
    stream, after three untimed calls."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def _stream_timed(h, fn, k, stream):
    """(mean ms of a whole call, mean ms of its k_stream launch)."""
    import paper_2303_07597_gb300 as pk
    fn()
    pk.ot_gs_set_timing(h, True)
    ms = _timed(fn, k, stream)
    pk.ot_gs_set_timing(h, False)
    nl, kms = pk.ot_gs_get_timing(h)
    return ms, kms / max(1, nl)


def screened_needed_bytes(skip_mask, sizes, n, L):
    """Bytes one screened evaluation (Alg. 2 with the tile-level test) must
    read at least: C of every block (l, j) it does not skip (g_l rows x 4
    bytes); per unit (class, 32-column tile) the tile's largest z~ and its
    word of N (4 bytes each); z~ (4 bytes) of every column of the units that
    hold a block it does not skip (the tile test cannot pass there); alpha,
    beta and their snapshot values (FP64).  skip_mask: L x ceil(n/32) words,
    bit j % 32 of word (l, j / 32) set when block (l, j) is skipped; sizes:
    rows per class (an empty class needs nothing)."""
    words = np.asarray(skip_mask, dtype=np.uint32).reshape(L, -1)
    ntiles = words.shape[1]
    bits = np.unpackbits(words.view(np.uint8), bitorder="little").reshape(L, -1)[:, :n]
    sizes = np.asarray(sizes, dtype=np.int64)
    skipped = bits.sum(axis=1).astype(np.int64)
    c_needed = int(np.sum(sizes * (n - skipped))) * 4
    pad = np.ones((L, ntiles * 32), dtype=np.uint8)
    pad[:, :n] = bits
    unit_open = (pad.reshape(L, ntiles, 32) == 0).any(axis=2) & (sizes > 0)[:, None]
    tile_cols = np.minimum(32, n - 32 * np.arange(ntiles))
    z_bytes = 4 * int(np.sum(unit_open * tile_cols[None, :]))
    m = int(np.sum(sizes))
    return c_needed + z_bytes + 8 * L * ntiles + 16 * (m + n), c_needed, int(skipped.sum())


def solve_report(args, dev):
    """Time to a relative objective error of 1e-6 (|D_k - D*| <= 1e-6 |D*|)
    for the plain (dense) and the screened device solver from the zero start
    (Alg. 1), read from the solver's device-time objective trace.  D* is the
    objective of a dense run to stagnation (ftol 1e-14).  The screened solver
    visits the same iterates bit for bit (each screened evaluation equals the
    dense one), so both reach the threshold at the same iteration; only the
    time differs.  At that iterate, with the screened run's own snapshot and
    set N, one dense and one screened evaluation are timed apart (roofline of
    each: the dense one against 4mn + 8(m+n) bytes, the screened one against
    the bytes Alg. 2 must read there)."""
    import torch
    import paper_2303_07597_gb300 as pk
    name = args.solve_workload
    cfg = WORKLOADS[name]
    p, C, _ = _make_workload(name, args.seed, str(dev))
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    lab = torch.from_numpy(p.labels).to(dev)
    stream = torch.cuda.current_stream()
    ref = pk.GroupSparseOT(C, a, b, lab, p.L, cfg["gamma"], cfg["mu"])
    ref.set_params(use_screening=0, ftol=1e-14)
    t0 = time.perf_counter()
    ref.solve(0.0, args.solve_ref_iters)
    ref_s = time.perf_counter() - t0
    D, t, ev = ref.trace()
    sol = ref.solution()
    ref.close()
    Dstar = float(D[-1])
    rel = np.abs(D - Dstar) / abs(Dstar)
    hit = np.nonzero(rel <= 1e-6)[0]
    k = int(hit[0]) if len(hit) and hit[0] < len(D) - 1 else -1
    out = {"workload": f"{name}: m=n={cfg['m']}, L={cfg['L']}, gamma={cfg['gamma']}, mu={cfg['mu']}, from zero",
           "D_star": Dstar, "D_star_iters": int(len(D) - 1), "D_star_grad_inf": sol["grad_inf"],
           "D_star_run_s": ref_s, "iters_to_1e-6": k, "unit": "ms"}
    if k < 0:
        out["note"] = "the reference run did not reach the threshold before its last iterate"
        return out
    out["dense_ms"] = float(t[k])
    out["dense_evals"] = int(ev[k])
    scr = pk.GroupSparseOT(C, a, b, lab, p.L, cfg["gamma"], cfg["mu"])
    scr.set_params(use_screening=1, ftol=0.0)
    scr.solve(0.0, k)
    Ds, ts, evs = scr.trace()
    st = scr.stats()
    out["screened_ms"] = float(ts[k])
    out["screened_evals"] = int(evs[k])
    out["screened_same_iterates"] = bool(len(Ds) > k and np.array_equal(Ds[:k + 1], D[:k + 1]))
    out["screened_units_computed_frac"] = st["units_computed"] / max(1, st["units_total"])
    out["screened_c_bytes_frac"] = st["c_bytes"] / max(1.0, 4.0 * p.m * p.n * st["evals"])
    out["screened_vs_dense"] = out["dense_ms"] / out["screened_ms"]
    # per-iteration time over the last fifth of the run, where the iterates move least
    k0 = int(0.8 * k)
    out["last_fifth_ms_per_iter"] = {"dense": float(t[k] - t[k0]) / (k - k0),
                                     "screened": float(ts[k] - ts[k0]) / (k - k0)}
    # evaluations at the iterate of the crossing
    it = scr.solution()
    al, be = it["alpha"], it["beta"]
    outv = torch.empty(1 + p.m + p.n, dtype=torch.float64, device=dev)
    peak, peak_kind = _peaks()
    reps = args.solve_eval_reps
    dense_bytes = 4.0 * p.m * p.n + 8.0 * (p.m + p.n)
    ms, kms = _stream_timed(scr.h, lambda: pk.ot_gs_grad(scr.h, al, be, outv), reps, stream)
    out["dense_eval_at_iterate"] = {
        "iterate": k, "step_ms": ms, "k_stream_ms": kms, "alg_bytes": dense_bytes,
        "roofline": {"bound": "hbm", "kernel": "k_stream", "achieved": dense_bytes / kms / 1e6, "peak": peak,
                     "unit": "GB/s", "frac": dense_bytes / kms / 1e6 / peak, "peak_kind": peak_kind},
        "step_frac": dense_bytes / ms / 1e6 / peak}
    Dd = float(outv[0].item())
    skip = torch.empty(p.L * ((p.n + 31) // 32), dtype=torch.int32, device=dev)
    pk.ot_gs_grad_screened(scr.h, al, be, outv, skip)
    sizes = np.bincount(p.labels, minlength=p.L)
    need, c_need, nskip = screened_needed_bytes(skip.cpu().numpy().view(np.uint32), sizes, p.n, p.L)
    pk.ot_gs_reset_stats(scr.h)
    ms_s, kms_s = _stream_timed(scr.h, lambda: pk.ot_gs_grad_screened(scr.h, al, be, outv), reps, stream)
    st2 = scr.stats()
    per = max(1, st2["evals"])
    out["screened_eval_at_iterate"] = {
        "iterate": k, "snapshot_iterate": k - (k % scr.params().r or scr.params().r), "step_ms": ms_s, "k_stream_ms": kms_s,
        "blocks_skipped_frac": nskip / (p.L * p.n), "needed_bytes": need, "needed_c_bytes": c_need,
        "streamed_c_bytes": st2["c_bytes"] / per,
        "roofline": {"bound": "hbm", "kernel": "whole screened evaluation", "achieved": need / ms_s / 1e6,
                     "peak": peak, "unit": "GB/s", "frac": need / ms_s / 1e6 / peak, "peak_kind": peak_kind},
        "same_D_as_dense": float(outv[0].item()) == Dd,
        "vs_dense_eval": ms / ms_s}
    scr.close()
    return out


BATCH = dict(nprob=512, m=(64, 2048), n=(64, 2048), L=(5, 100), d=64, gamma=1.0, mu=0.1)


def _batch_on_device(seed, dev, nprob):
    """The batched workload's problems with each C in one device buffer, row
    stride rounded up to 4 floats (the layout the evaluation kernel borrows)."""
    import torch
    probs = synth.batch(seed=seed, nprob=nprob, m_range=BATCH["m"], n_range=BATCH["n"], L_range=BATCH["L"],
                        d=BATCH["d"], device=str(dev))
    lds = [(p.n + 3) // 4 * 4 for p in probs]
    flat = torch.zeros(sum(p.m * ld for p, ld in zip(probs, lds)), dtype=torch.float32, device=dev)
    Cs, off = [], 0
    for p, ld in zip(probs, lds):
        v = flat[off:off + p.m * ld].view(p.m, ld)
        v[:, :p.n].copy_(torch.from_numpy(p.C))
        Cs.append(v[:, :p.n])
        off += p.m * ld
    As = [torch.from_numpy(p.a).to(dev) for p in probs]
    Bs = [torch.from_numpy(p.b).to(dev) for p in probs]
    Ls = [torch.from_numpy(p.labels).to(dev) for p in probs]
    return probs, flat, Cs, As, Bs, Ls


def batch_report(args, dev):
    """Time to a relative objective error of 1e-6 for the batched workload:
    all problems solved together (one evaluation kernel per trial for every
    running problem, trials in CUDA graphs, one L-BFGS state per problem),
    against the plain device solver run on one problem after the other.  D*
    of each problem comes from a longer batched run; both arms start from
    zero and stop a problem once D >= D* - 1e-6 |D*| (the plain solver's
    crossing is read from its device-time objective trace)."""
    import torch
    import paper_2303_07597_gb300 as pk
    g, mu = BATCH["gamma"], BATCH["mu"]
    nprob = args.batch_problems
    probs, flat, Cs, As, Bs, Ls = _batch_on_device(args.seed, dev, nprob)
    out = {"workload": f"batched: {nprob} problems, m, n ~ U[{BATCH['m'][0]}, {BATCH['m'][1]}], "
                       f"L ~ U[{BATCH['L'][0]}, {BATCH['L'][1]}] with Dirichlet(2) sizes, d={BATCH['d']}, "
                       f"gamma={g}, mu={mu}",
           "c_bytes": int(sum(4 * p.m * p.n for p in probs)), "unit": "ms"}
    B = pk.GroupSparseOTBatch(Cs, As, Bs, Ls, [p.L for p in probs], g, mu)
    zero_a = torch.zeros(B.m, dtype=torch.float64, device=dev)
    zero_b = torch.zeros(B.n, dtype=torch.float64, device=dev)
    # reference objectives: until the gradient or the objective stagnates
    # (the FP32 evaluation has a noise floor below which D stops improving)
    B.set_params(ftol=1e-14)
    t0 = time.perf_counter()
    B.solve(tol=1e-10, maxit=args.batch_ref_iters)
    ref = B.result()
    out["ref_s"] = time.perf_counter() - t0
    B.set_params(ftol=0.0)
    Dstar = ref["D"].copy()
    out["ref_iters_mean"] = float(ref["iters"].mean())
    out["ref_status_counts"] = {str(k): int(v) for k, v in zip(*np.unique(ref["status"], return_counts=True))}
    out["ref_iters_max"] = int(ref["iters"].max())

    def timed_batch():
        B.set_state(zero_a, zero_b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = B.solve(tol=0.0, maxit=args.batch_ref_iters, target_D=Dstar, target_rtol=1e-6)
        el = (time.perf_counter() - t0) * 1000.0
        r = B.result(with_iterate=False)
        return st, el, r

    plan0 = B.plan()
    st, el, r = timed_batch()
    out["default_plan"] = plan0
    out["batched_ms"] = el
    out["batched_device_ms"] = float(r["t_ms"].max())
    out["batched_all_reached"] = bool(st == pk.OTGS_OK and np.all(r["status"] == 0))
    out["batched_trials"] = int(r["evals"].sum())
    out["iters_to_1e-6"] = {"mean": float(r["iters"].mean()), "max": int(r["iters"].max())}
    # autotuned plan, tuned at an iterate half way to the target
    B.set_state(zero_a, zero_b)
    B.solve(tol=0.0, maxit=max(1, int(r["iters"].mean()) // 2))
    mid = B.result()
    pk.ot_gs_autotune_clear_cache()
    tune = B.autotune(mid["alpha"], mid["beta"], evals=5)
    st2, el2, r2 = timed_batch()
    out["tuned_plan"] = {**B.plan(), "eval_ms": tune["best_ms"]}
    out["batched_tuned_ms"] = el2
    out["batched_tuned_all_reached"] = bool(st2 == pk.OTGS_OK and np.all(r2["status"] == 0))
    B.close()
    # the plain solver, one problem after the other
    take = list(range(nprob)) if args.batch_plain_sample <= 0 else \
        list(np.random.default_rng(1).choice(nprob, size=min(nprob, args.batch_plain_sample), replace=False))
    plain_ms, plain_wall, missed = 0.0, 0.0, 0
    for k in take:
        s = pk.GroupSparseOT(Cs[k], As[k], Bs[k], Ls[k], probs[k].L, g, mu)
        s.set_params(use_screening=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.solve(0.0, int(r["iters"][k]) + 50)
        plain_wall += time.perf_counter() - t0
        D, t, ev = s.trace()
        s.close()
        hit = np.nonzero(D >= Dstar[k] - 1e-6 * abs(Dstar[k]))[0]
        if len(hit):
            plain_ms += float(t[hit[0]])
        else:
            plain_ms += float(t[-1])
            missed += 1
    scale = nprob / len(take)
    out["plain_problems_timed"] = len(take)
    out["plain_ms"] = plain_ms * scale
    out["plain_wall_ms"] = plain_wall * 1000.0 * scale
    out["plain_missed_target"] = missed
    out["batched_vs_plain"] = out["plain_ms"] / min(out["batched_ms"], out["batched_tuned_ms"])
    del flat
    return out


WARM = dict(m=256, L=13, d=64, gamma=1.0, mu=0.1)


def warm_report(args, dev):
    """Learned warm start: the network is trained (the library's kernels) on
    solutions of args.warm_train problems of the Zipf-class generator family
    (the large workload's generator at m = n = 256, 13 classes, d = 64), then
    the args.warm_test held-out problems are solved together from zero and
    from the network's prediction (features, forward pass, shift search
    included in the warm time), both to D >= D* - 1e-6 |D*| with D* from a
    longer run."""
    import torch
    import paper_2303_07597_gb300 as pk
    from paper_2303_07597_gb300 import warmstart as ws
    c = WARM
    g, mu = c["gamma"], c["mu"]
    K = ws.in_dim_for(c["d"])
    out = {"workload": f"warm start: Zipf(1.1)-class problems m=n={c['m']}, L={c['L']}, d={c['d']}, gamma={g}, "
                       f"mu={mu}; {args.warm_train} training / {args.warm_test} held-out problems",
           "unit": "ms"}
    t0 = time.perf_counter()
    gen = lambda s: synth.large(seed=s, m=c["m"], n=c["m"], L=c["L"], d=c["d"], keep_features=True,
                                device=str(dev))
    train_p = [gen(1000 + s) for s in range(args.warm_train)]
    test_p = [gen(10_000_000 + s) for s in range(args.warm_test)]
    out["generate_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    targets = []
    for c0 in range(0, len(train_p), 512):
        Bt, tg, _ = ws.solve_targets(train_p[c0:c0 + 512], dev, g, mu)
        targets += tg
        Bt.close()
    torch.cuda.synchronize()
    out["solve_targets_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    X, t = ws.dataset(train_p, targets, dev, K, g)
    if args.warm_passes < 2:
        del targets
    net = pk.WarmStartMLP(K, 256, max_batch=8192, seed=1)
    trace = ws.train(net, X, t, steps=args.warm_steps, batch=8192, lr=1e-3, lr_end=1e-4)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    out["train_samples"] = int(X.shape[0])
    out["train_steps"] = args.warm_steps
    out["train_loss_first_last"] = [trace[0], trace[-1]]
    del X, t
    # inference in chunks of 65536 samples (the training handle's buffers hold 8192)
    infer = pk.WarmStartMLP(K, 256, max_batch=65536, seed=1)
    infer.set_params(net.params())
    infer2 = None
    if args.warm_passes >= 2:
        # a second network on the features plus the second-pass inputs from the first one's prediction
        t0 = time.perf_counter()
        X2, t2_ = ws.dataset_refine(train_p, targets, dev, K, g, infer)
        del targets
        net2 = pk.WarmStartMLP(K, 256, max_batch=8192, seed=2)
        trace2 = ws.train(net2, X2, t2_, steps=args.warm_steps, batch=8192, lr=1e-3, lr_end=1e-4)
        del X2, t2_
        infer2 = pk.WarmStartMLP(K, 256, max_batch=65536, seed=2)
        infer2.set_params(net2.params())
        net2.close()
        torch.cuda.synchronize()
        out["train2_s"] = time.perf_counter() - t0
        out["train2_loss_first_last"] = [trace2[0], trace2[-1]]
    # held out
    B, tt, ref = ws.solve_targets(test_p, dev, g, mu)
    Dstar = ref["D"].copy()
    B.set_params(ftol=0.0)
    devp = []
    for p in test_p:
        devp.append((torch.from_numpy(p.C).to(dev),
                     torch.from_numpy(np.ascontiguousarray(p.XS, dtype=np.float32)).to(dev),
                     torch.from_numpy(np.ascontiguousarray(p.XT, dtype=np.float32)).to(dev),
                     torch.from_numpy(p.labels).to(dev)))
    za = torch.zeros(B.m, dtype=torch.float64, device=dev)
    zb = torch.zeros(B.n, dtype=torch.float64, device=dev)
    # one untimed pass of the warm-start preparation (first uses of its kernels)
    ws.warm_state(B, ws.predict_batch(infer, devp, [p.L for p in test_p], K, g))
    B.set_state(za, zb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6)
    cold_ms = (time.perf_counter() - t0) * 1000.0
    cold = B.result(with_iterate=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pal, pbe = ws.predict_batch(infer, devp, [p.L for p in test_p], K, g)
    torch.cuda.synchronize()
    tp = time.perf_counter()
    al, be, used = ws.warm_state(B, (pal, pbe))
    B.set_state(al, be)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st2 = B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6)
    t2 = time.perf_counter()
    warm = B.result(with_iterate=False)
    rmse = []
    for k, (ta, tb) in enumerate(tt):
        a, b = ws.gauge_fix(B.split(pal, k, "alpha"), B.split(pbe, k, "beta"))
        rmse.append(float(torch.cat([a - ta, b - tb]).pow(2).mean().sqrt().item()))
    parts = {}
    ws.predict_batch(infer, devp, [p.L for p in test_p], K, g, timings=parts)  # the parts, timed apart
    if infer2 is not None:
        Ls = [p.L for p in test_p]
        ws.warm_state(B, ws.predict_batch_refine(infer, infer2, devp, Ls, K, g))  # untimed first use
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        pal2, pbe2 = ws.predict_batch_refine(infer, infer2, devp, Ls, K, g)
        al2, be2, used2 = ws.warm_state(B, (pal2, pbe2))
        B.set_state(al2, be2)
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        st3 = B.solve(tol=0.0, maxit=20000, target_D=Dstar, target_rtol=1e-6)
        t5 = time.perf_counter()
        warm2 = B.result(with_iterate=False)
        rmse2 = []
        for k, (ta, tb) in enumerate(tt):
            a, b = ws.gauge_fix(B.split(pal2, k, "alpha"), B.split(pbe2, k, "beta"))
            rmse2.append(float(torch.cat([a - ta, b - tb]).pow(2).mean().sqrt().item()))
        out.update({
            "warm2_ms": (t5 - t3) * 1000.0, "warm2_prepare_ms": (t4 - t3) * 1000.0,
            "warm2_all_reached": bool(st3 == pk.OTGS_OK and np.all(warm2["D"] >= Dstar - 1e-6 * np.abs(Dstar))),
            "warm2_iters_mean": float(warm2["iters"].mean()), "warm2_used_frac": float(np.mean(used2)),
            "warm2_iters_p50_p90_max": [float(np.percentile(warm2["iters"], 50)),
                                        float(np.percentile(warm2["iters"], 90)), int(warm2["iters"].max())],
            "heldout_rmse2_mean": float(np.mean(rmse2)),
            "warm2_vs_cold": cold_ms / ((t5 - t3) * 1000.0),
        })
        infer2.close()
    B.close()
    net.close()
    infer.close()
    out.update({
        "warm_features_ms": parts["features_ms"], "warm_network_ms": parts["network_ms"],
        "cold_ms": cold_ms, "cold_all_reached": bool(st == pk.OTGS_OK),
        "cold_iters_mean": float(cold["iters"].mean()),
        "warm_ms": (t2 - t0) * 1000.0, "warm_predict_ms": (tp - t0) * 1000.0,
        "warm_shift_ms": (t1 - tp) * 1000.0, "warm_solve_ms": (t2 - t1) * 1000.0,
        "warm_all_reached": bool(st2 == pk.OTGS_OK and np.all(warm["D"] >= Dstar - 1e-6 * np.abs(Dstar))),
        "warm_iters_mean": float(warm["iters"].mean()), "warm_used_frac": float(np.mean(used)),
        # spread over the problems: iterations and device time at which each stopped
        "cold_iters_p50_p90_max": [float(np.percentile(cold["iters"], 50)), float(np.percentile(cold["iters"], 90)),
                                   int(cold["iters"].max())],
        "warm_iters_p50_p90_max": [float(np.percentile(warm["iters"], 50)), float(np.percentile(warm["iters"], 90)),
                                   int(warm["iters"].max())],
        "cold_stop_ms_p50_p90_max": [float(np.percentile(cold["t_ms"], 50)), float(np.percentile(cold["t_ms"], 90)),
                                     float(cold["t_ms"].max())],
        "warm_stop_ms_p50_p90_max": [float(np.percentile(warm["t_ms"], 50)), float(np.percentile(warm["t_ms"], 90)),
                                     float(warm["t_ms"].max())],
        "heldout_rmse_mean": float(np.mean(rmse)),
        "warm_vs_cold": cold_ms / ((t2 - t0) * 1000.0),
        # per problem: the median problem's time to the target, cold over warm
        # (the warm one including the preparation), and the slowest problem's
        # iterations if each problem took the better of its two starts
        "warm_vs_cold_median_problem": float(np.percentile(cold["t_ms"], 50))
        / (float(np.percentile(warm["t_ms"], 50)) + (t1 - t0) * 1000.0),
        "min_of_starts_iters_max": int(np.max(np.minimum(cold["iters"], warm["iters"]))),
    })
    return out


def case_report(args, dev):
    """One kernel family in isolation, for profiling under ncu (``--case``).

    batch: ``--case-n`` problems of the batched workload's generator solved
    together from zero for ``--case-iters`` iterations (each trial: k_bgate,
    k_stream, k_split_finish, k_passb, k_bstep), with one evaluation timed at
    zero and one at the final iterate.
    mlp: the warm-start network (input width 144, hidden 256) trained for
    ``--case-iters`` Adam steps on 65536 random samples in batches of 8192,
    then 50 more steps timed (three GEMM kernels forward and five backward
    per step).
    late: a member of the large family (``--case-workload``: the 10k one, m =
    n = 10^4, 500 classes, 400 MB of C, or the full one) solved from zero for ``--case-iters`` iterations (snapshot
    and N taken there, as Alg. 1's refresh), then 10 iterations more (the
    saved state restored and continued); at that iterate 20 dense and 20
    screened evaluations are timed (CUDA events) after 3 of each untimed."""
    import torch
    import paper_2303_07597_gb300 as pk
    out = {"case": args.case}
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    if args.case == "batch":
        probs, flat, Cs, As, Bs, Ls = _batch_on_device(args.seed, dev, args.case_n)
        B = pk.GroupSparseOTBatch(Cs, As, Bs, Ls, [p.L for p in probs], BATCH["gamma"], BATCH["mu"])
        out.update(problems=args.case_n, c_bytes=int(sum(4 * p.m * p.n for p in probs)), plan=B.plan())
        za = torch.zeros(B.m, dtype=torch.float64, device=dev)
        zb = torch.zeros(B.n, dtype=torch.float64, device=dev)

        def eval_ms(a, b, k=10):
            B.grad(a, b)
            torch.cuda.synchronize()
            e0, e1 = ev()
            e0.record()
            for _ in range(k):
                B.grad(a, b, with_grad=False)
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / k

        out["eval_at_zero_ms"] = eval_ms(za, zb)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.solve(tol=0.0, maxit=args.case_iters)
        el = time.perf_counter() - t0
        r = B.result()
        out.update(iters=args.case_iters, solve_s=el, trials=int(r["evals"].max()),
                   trial_ms=el * 1e3 / max(1, int(r["evals"].max())),
                   eval_at_iterate_ms=eval_ms(r["alpha"], r["beta"]))
        B.close()
    elif args.case == "late":
        wl = args.case_workload
        cfg = WORKLOADS[wl]
        p, C, _ = _make_workload(wl, args.seed, str(dev))
        s = pk.GroupSparseOT(C, torch.from_numpy(p.a).to(dev), torch.from_numpy(p.b).to(dev),
                             torch.from_numpy(p.labels).to(dev), p.L, cfg["gamma"], cfg["mu"])
        s.solve(0.0, args.case_iters)
        it0 = s.solution()
        s.restore_state(s.save_state())
        s.solve(0.0, args.case_iters + 10)
        it1 = s.solution()
        s.snapshot(it0["alpha"], it0["beta"], build_N=False)
        s.snapshot(it0["alpha"], it0["beta"], build_N=True)
        outv = torch.empty(1 + p.m + p.n, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        al, be = it1["alpha"], it1["beta"]
        torch.cuda.synchronize()
        torch.cuda.profiler.start()  # (ncu --profile-from-start off captures from here)
        dense_ms = _timed(lambda: pk.ot_gs_grad(s.h, al, be, outv), 20, stream)
        Dd = float(outv[0].item())
        pk.ot_gs_reset_stats(s.h)
        scr_ms = _timed(lambda: pk.ot_gs_grad_screened(s.h, al, be, outv), 20, stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        st = s.stats()
        out.update(workload=f"{wl}: m=n={cfg['m']}, L={cfg['L']}, gamma={cfg['gamma']}, mu={cfg['mu']}",
                   iterate=args.case_iters + 10,
                   snapshot_iterate=args.case_iters, dense_ms=dense_ms, screened_ms=scr_ms,
                   same_D=float(outv[0].item()) == Dd,
                   screened_units_frac=st["units_computed"] / max(1, st["units_total"]),
                   screened_blocks_skipped_frac=st["blocks_skipped"] / max(1, st["blocks_total"]))
        s.close()
    else:
        from paper_2303_07597_gb300 import warmstart as ws
        K, H, nb = 144, 256, 8192
        rng = np.random.default_rng(args.seed)
        X = torch.from_numpy(rng.normal(size=(65536, K)).astype(np.float32)).to(dev)
        t = torch.from_numpy(rng.normal(size=65536).astype(np.float32)).to(dev)
        net = pk.WarmStartMLP(K, H, max_batch=nb, seed=1)
        tr = ws.train(net, X, t, steps=args.case_iters, batch=nb)
        e0, e1 = ev()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(50):
            net.train_step(X[:nb], t[:nb], 1e-4)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 50
        flops = 2 * nb * (K * H + H * H + H) * 3  # forward and the two backward products of each layer
        out.update(steps=args.case_iters, train_step_ms=ms, tflops=flops / ms / 1e9, loss_last=tr[-1])
        net.close()
    return out


def panel_sweep_report(args, dev):
    """Dense evaluations of --workload at the bench point for several panel
    heights (rows of whole class groups per work item): whole step and
    k_stream per launch, CUDA events on the launch stream.  The plan only
    changes how the blocks are tiled, so D is the same for every height."""
    import torch
    import paper_2303_07597_gb300 as pk
    p, C, cfg = _make_workload(args.workload, args.seed, str(dev))
    s = pk.GroupSparseOT(C, torch.from_numpy(p.a).to(dev), torch.from_numpy(p.b).to(dev),
                         torch.from_numpy(p.labels).to(dev), p.L, cfg["gamma"], cfg["mu"])
    alpha, beta = _eval_point(C, 20)
    out = torch.empty(1 + p.m + p.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rows = []
    for pr in [int(x) for x in args.panel_sweep.split(",")]:
        pk.ot_gs_set_plan(s.h, pr, 0, 0)
        plan = pk.ot_gs_get_plan(s.h)
        ms, kms = _stream_timed(s.h, lambda: pk.ot_gs_grad(s.h, alpha, beta, out), args.steps, stream)
        rows.append({"panel_rows": plan["panel_rows"], "n_items": plan["n_items"], "step_ms": ms,
                     "k_stream_ms": kms, "D": float(out[0].item())})
    s.close()
    return {"workload": args.workload, "rows": rows, "same_D": len({r["D"] for r in rows}) == 1}


def grid_report(args, dev):
    """The mid workload (m = n = 4000, 100 Dirichlet(2) classes, d = 256)
    over gamma in {0.1, 1, 10} x mu in {0.01, 0.1, 1}, screening off and on:
    for each pair a dense solve from zero to stagnation (ftol 1e-14) gives D*
    and the dense time to a relative objective error of 1e-6 (from its
    device-time trace); a screened solve (Alg. 1) runs to the same iteration
    and must visit the same iterates bit for bit."""
    import torch
    import paper_2303_07597_gb300 as pk
    p, C, _ = _make_workload("mid", args.seed, str(dev))
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    lab = torch.from_numpy(p.labels).to(dev)
    rows = []
    for gamma in [0.1, 1.0, 10.0]:
        for mu in [0.01, 0.1, 1.0]:
            ref = pk.GroupSparseOT(C, a, b, lab, p.L, gamma, mu)
            ref.set_params(use_screening=0, ftol=1e-14)
            ref.solve(0.0, args.grid_iters)
            D, t, ev = ref.trace()
            ref.close()
            Dstar = float(D[-1])
            hit = np.nonzero(np.abs(D - Dstar) <= 1e-6 * abs(Dstar))[0]
            k = int(hit[0]) if len(hit) else -1
            row = {"gamma": gamma, "mu": mu, "D_star": Dstar, "D_star_iters": int(len(D) - 1), "iters_to_1e-6": k}
            if k > 0:
                scr = pk.GroupSparseOT(C, a, b, lab, p.L, gamma, mu)
                scr.set_params(use_screening=1, ftol=0.0)
                scr.solve(0.0, k)
                Ds, ts, evs = scr.trace()
                st = scr.stats()
                scr.close()
                row.update(dense_ms=float(t[k]), screened_ms=float(ts[k]),
                           screened_vs_dense=float(t[k]) / float(ts[k]),
                           same_iterates=bool(len(Ds) > k and np.array_equal(Ds[:k + 1], D[:k + 1])),
                           blocks_skipped_frac=st["blocks_skipped"] / max(1, st["blocks_total"]))
            rows.append(row)
    return {"workload": "mid: m=n=4000, L=100 (Dirichlet(2) sizes), d=256, from zero", "unit": "ms", "rows": rows}


def sweep_report(args, dev):
    """Paper-shaped trends (Sec. 5, synthetic set with controlled classes):
    time of the screened solver (Alg. 1, with the set N) against the dense
    one, both from zero to ||grad D||_inf <= tol, summed over rho for each
    gamma (the paper's protocol), for growing numbers of classes |L| at g = 10
    (Fig. 2), growing class sizes g at |L| = 10 (appendix), and with / without
    the lower bound (appendix ablation)."""
    import torch
    import paper_2303_07597_gb300 as pk

    def solve_time(p, gamma, rho, screening, lower):
        g2, mu2 = pk.rho_to_gamma_mu(gamma, rho)
        C = torch.from_numpy(p.C).to(dev)
        a = torch.from_numpy(p.a).to(dev)
        b = torch.from_numpy(p.b).to(dev)
        lab = torch.from_numpy(p.labels).to(dev)
        s = pk.GroupSparseOT(C, a, b, lab, p.L, g2, mu2)
        s.set_params(use_screening=int(screening), use_lower_bound=int(lower))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.solve(tol=args.sweep_tol, maxit=args.sweep_maxit)
        el = time.perf_counter() - t0
        sol = s.solution()
        stats = s.stats()
        s.close()
        return el, st, sol["D"], stats

    def gain(p, gammas, rhos, lower=True):
        rows = []
        for gm in gammas:
            td = ts = 0.0
            same = True
            skipped = total = 0
            for rho in rhos:
                e1, st1, D1, _ = solve_time(p, gm, rho, False, True)
                e2, st2, D2, stt = solve_time(p, gm, rho, True, lower)
                td += e1
                ts += e2
                same = same and abs(D1 - D2) <= 1e-9 * max(1.0, abs(D1))
                skipped += stt["blocks_skipped"]
                total += stt["blocks_total"]
            rows.append({"gamma": gm, "dense_s": td, "screened_s": ts, "gain": td / ts, "same_D": same,
                         "skipped_frac": skipped / max(1, total)})
        return rows

    gammas = [float(x) for x in args.sweep_gammas.split(",")]
    rhos = [float(x) for x in args.sweep_rhos.split(",")]
    out = {"protocol": f"tol {args.sweep_tol}, maxit {args.sweep_maxit}, time summed over rho in {rhos}",
           "classes": [], "class_size": [], "lower_bound": []}
    for L in [int(x) for x in args.sweep_classes.split(",")]:
        p = synth.paper_synthetic(L, g=10, seed=args.seed)
        out["classes"].append({"L": L, "m": p.m, "rows": gain(p, gammas, rhos)})
    for gsz in [int(x) for x in args.sweep_sizes.split(",")]:
        p = synth.paper_synthetic(10, g=gsz, seed=args.seed)
        out["class_size"].append({"g": gsz, "m": p.m, "rows": gain(p, gammas, rhos)})
    for L in [int(x) for x in args.sweep_ablation.split(",")]:
        p = synth.paper_synthetic(L, g=10, seed=args.seed)
        out["lower_bound"].append({"L": L, "with": gain(p, gammas, rhos, True),
                                   "without": gain(p, gammas, rhos, False)})
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    if args.workload in ("tiny", "mid"):
        p = {"tiny": synth.tiny, "mid": synth.mid}[args.workload](seed=args.seed)
    else:
        p = synth.large(seed=args.seed, m=cfg["m"], n=cfg["n"], L=cfg["L"], d=cfg["d"])
    Cn = p.C
    k = 20 if args.workload != "tiny" else 5
    beta = np.sort(Cn, axis=0)[k - 1].astype(np.float64) + 1e-3
    alpha = np.zeros(p.m)
    per_step = max(2.0, 30.0 / max(1, args.steps + args.warmup))
    cb = None
    vals = []
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(p, alpha, beta, cfg["gamma"], cfg["mu"], budget_s=per_step)
        if s >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.workload}: m=n={cfg['m']}, L={cfg['L']}, gamma={cfg['gamma']}, "
                                   f"mu={cfg['mu']}", "l2": "inputs > L2"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2303_07597_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, C, cfg = _make_workload(args.workload, args.seed, str(dev))
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    lab = torch.from_numpy(p.labels).to(dev)
    solver = pk.GroupSparseOT(C, a, b, lab, p.L, cfg["gamma"], cfg["mu"])
    k = 20 if args.workload != "tiny" else 5
    alpha, beta = _eval_point(C, k)
    out = torch.empty(1 + p.m + p.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        pk.ot_gs_grad(solver.h, alpha, beta, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    kernels0 = solver.stats()["kernels"]
    pk.ot_gs_set_timing(solver.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid) as cs:
        torch.cuda.synchronize()
        cs.mark(True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        cs.mark(False)
    pk.ot_gs_set_timing(solver.h, False)
    kernels = solver.stats()["kernels"] - kernels0
    launches, kern_ms = pk.ot_gs_get_timing(solver.h)
    el_ms = max_over_ranks(e0.elapsed_time(e1), dev)
    if world > 1:
        dist.barrier()
    clocks = cs.summary()

    # a C that fits in L2 (mid, tiny): the same steps, each after a write of a
    # buffer twice the size of L2, timed one by one with events around the
    # evaluation only
    flushed = None
    if 4.0 * p.m * p.n < L2_BYTES:
        junk = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        pk.ot_gs_set_timing(solver.h, True)
        for a_ev, b_ev in ev:
            junk.fill_(1.0)
            a_ev.record(stream)
            step()
            b_ev.record(stream)
        torch.cuda.synchronize()
        pk.ot_gs_set_timing(solver.h, False)
        fl_launches, fl_kern_ms = pk.ot_gs_get_timing(solver.h)
        fl_ms = max_over_ranks(sum(a_ev.elapsed_time(b_ev) for a_ev, b_ev in ev), dev)
        flushed = {"value": job_throughput(args.steps, world, fl_ms), "unit": UNIT,
                   "ms_per_step": fl_ms / args.steps,
                   "kernel_ms": fl_kern_ms / max(1, fl_launches),
                   "how": "each step after a write of 2x L2 (258 MB); events around each evaluation"}
        del junk

    # end to end: host inputs in pinned memory, copies inside the timed region
    h_alpha = alpha.cpu().pin_memory()
    h_beta = beta.cpu().pin_memory()
    h_out = torch.empty(out.shape, dtype=torch.float64).pin_memory()
    d_alpha, d_beta = torch.empty_like(alpha), torch.empty_like(beta)

    def step_e2e():
        d_alpha.copy_(h_alpha, non_blocking=True)
        d_beta.copy_(h_beta, non_blocking=True)
        pk.ot_gs_grad(solver.h, d_alpha, d_beta, out)
        h_out.copy_(out, non_blocking=True)

    for _ in range(args.warmup):
        step_e2e()
    torch.cuda.synchronize()
    k_e2e = max(1, args.steps // 2)
    e0.record(stream)
    for _ in range(k_e2e):
        step_e2e()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dev)

    if rank == 0:
        m, n = p.m, p.n
        value = job_throughput(args.steps, world, el_ms)
        kern_avg_s = kern_ms / max(1, launches) / 1000.0
        alg_bytes = 4.0 * m * n + 8.0 * (m + n)
        peak, peak_kind = _peaks()
        achieved = alg_bytes / kern_avg_s / 1e9
        cb = None
        if world == 1 and not args.no_cpu_baseline:
            hp = p
            cb = cpu_baseline(hp, alpha.cpu().numpy(), beta.cpu().numpy(), cfg["gamma"], cfg["mu"],
                              budget_s=args.cpu_budget)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: m=n={cfg['m']}, L={cfg['L']} "
                                   f"({'Zipf(1.1) sizes, min 2' if args.workload.startswith('large') else 'classes'}), "
                                   f"d={cfg['d']}, gamma={cfg['gamma']}, mu={cfg['mu']}, dense evaluation",
                       "l2": "inputs > L2 (C is 4mn bytes)" if flushed is None else
                             "C fits in L2: value with C resident (warm), l2_flushed with L2 flushed before each step",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "k_stream", "alg_bytes_per_launch": alg_bytes,
                         "kernel_ms": kern_avg_s * 1000.0,
                         "traffic": _traffic_for(_src_hash(), args.workload)},
            "cpu_baseline": cb,
            "l2_flushed": flushed,
            "e2e": {"value": job_throughput(k_e2e, world, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (m + n), "d2h_bytes_per_step": 8 * (1 + m + n)},
            # the library's own count per evaluation: k_prep, k_stream, k_exact_t,
            # k_reduce, and k_split_finish when a class is split across items
            "gpu_launches": kernels,
            "clocks": clocks,
        }
        if world == 1 and not args.no_solve:
            line["solve"] = solve_report(args, dev)
        if world == 1 and not args.no_batch:
            line["batch"] = batch_report(args, dev)
        if world == 1 and not args.no_warm:
            line["warm_start"] = warm_report(args, dev)
        print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-1e-6 solve measurement")
    ap.add_argument("--solve-workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--solve-ref-iters", type=int, default=65000)
    ap.add_argument("--solve-eval-reps", type=int, default=50,
                    help="evaluations timed at the iterate where the solve reaches 1e-6")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload solve measurement")
    ap.add_argument("--batch-problems", type=int, default=BATCH["nprob"])
    ap.add_argument("--batch-ref-iters", type=int, default=20000)
    ap.add_argument("--batch-plain-sample", type=int, default=64,
                    help="time the plain solver on this many problems and scale (0: all)")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start measurement")
    ap.add_argument("--warm-train", type=int, default=4096)
    ap.add_argument("--warm-test", type=int, default=512)
    ap.add_argument("--warm-steps", type=int, default=8000)
    ap.add_argument("--warm-passes", type=int, default=1, choices=[1, 2],
                    help="2: also a second network on the second-pass inputs (water levels against the first "
                         "prediction), solved from its prediction as well")
    ap.add_argument("--grid", action="store_true",
                    help="only the mid workload over the (gamma, mu) grid, dense and screened time to 1e-6")
    ap.add_argument("--grid-iters", type=int, default=30000)
    ap.add_argument("--panel-sweep", default="",
                    help="only dense evaluations of --workload at these panel heights (comma-separated)")
    ap.add_argument("--sweep", action="store_true",
                    help="only the paper-shaped trends (screened vs dense over classes, class sizes, lower bound)")
    ap.add_argument("--sweep-classes", default="10,40,160,640,1280")
    ap.add_argument("--sweep-sizes", default="10,40,160")
    ap.add_argument("--sweep-ablation", default="10,640")
    ap.add_argument("--sweep-gammas", default="100,1,0.01")
    ap.add_argument("--sweep-rhos", default="0.2,0.8")
    ap.add_argument("--sweep-tol", type=float, default=1e-7)
    ap.add_argument("--sweep-maxit", type=int, default=3000)
    ap.add_argument("--case", choices=["batch", "mlp", "late"],
                    help="only one kernel family in isolation (for profiling): the batched solver, the network, "
                         "or the evaluations at a late solve iterate")
    ap.add_argument("--case-n", type=int, default=128, help="--case batch: problems")
    ap.add_argument("--case-workload", choices=["large10k", "large"], default="large10k",
                    help="--case late: the member of the large family")
    ap.add_argument("--case-iters", type=int, default=300, help="--case batch: iterations; mlp: training steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(case_report(args, torch.device("cuda", 0))))
        return 0
    if args.grid:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"grid": grid_report(args, torch.device("cuda", 0))}))
        return 0
    if args.sweep:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"sweep": sweep_report(args, torch.device("cuda", 0))}))
        return 0
    if args.panel_sweep:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"panel_sweep": panel_sweep_report(args, torch.device("cuda", 0))}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
