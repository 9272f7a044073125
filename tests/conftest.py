import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """The error of every GPU result checked against the oracle: per test the
    largest |D - D*| / |D*|, |D - D*| / (|alpha.a| + |beta.b| + |sum psi|) and
    gradient errors (relative to max(|g|, marginal))."""
    gu = sys.modules.get("gpu_util")
    rows = getattr(gu, "RESULTS", None) if gu else None
    if not rows:
        return
    tr = terminalreporter
    tr.section("errors against the FP64 oracle (max per test)")
    per = {}
    for r in rows:
        k = r["test"]
        q = per.setdefault(k, dict(n=0, D_rel=0.0, D_rel_terms=0.0, ga_rel=0.0, gb_rel=0.0))
        q["n"] += 1
        for f in ("D_rel", "D_rel_terms", "ga_rel", "gb_rel"):
            q[f] = max(q[f], r[f])
    tr.write_line(f"{'test':80s} {'n':>4s} {'|dD|/|D|':>10s} {'|dD|/terms':>10s} {'grad a':>9s} {'grad b':>9s}")
    for k, q in per.items():
        tr.write_line(f"{k[-80:]:80s} {q['n']:4d} {q['D_rel']:10.2e} {q['D_rel_terms']:10.2e} "
                      f"{q['ga_rel']:9.2e} {q['gb_rel']:9.2e}")
    tr.write_line(f"all {len(rows)} results: max |dD|/|D| {max(r['D_rel'] for r in rows):.2e}, "
                  f"max grad error {max(max(r['ga_rel'], r['gb_rel']) for r in rows):.2e}")
