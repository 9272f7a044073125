"""Host-side checks of the C ABI library (no GPU needed): it loads, exports
every entry point declared in include/otgs.h, and its host-side work plan
covers every row of every class exactly once."""
import ctypes

import numpy as np
import pytest

import paper_2303_07597_gb300 as pk
import synth


def test_library_exports_every_header_symbol():
    lib = pk.lib()
    names = pk.header_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert pk.ot_gs_version().startswith("otgs")


def test_create_rejects_null_without_gpu():
    h = ctypes.c_void_p()
    rc = pk.lib().ot_gs_create(ctypes.byref(h), None, 1, None, None, None, 1, 1, 1, 1.0, 0.1, None)
    assert rc == pk.OTGS_EINVAL and not h.value
    assert "NULL" in pk.ot_gs_last_error(None)


ITEM_COLS, STAGE_ROWS = 256, 32


def panel_height(m, n):
    """m * ceil(n / 256) / 2048 rows, clamped to [32, 512]."""
    return min(512, max(32, -(-m * -(-n // ITEM_COLS) // 2048)))


SPLIT_ROWS = 256


def expected_plan(sizes, n):
    """Panels by the packing rule of the plan (consecutive non-empty groups up
    to the panel height; a group of more than 256 rows cut into pieces of 256
    rows, each a panel), items and stages from them."""
    PANEL_ROWS = panel_height(int(np.sum(sizes)), n)
    panels, cur = [], 0
    for g in sizes:
        if g == 0:
            continue
        if g > SPLIT_ROWS:
            if cur:
                panels.append(cur)
                cur = 0
            panels += [min(SPLIT_ROWS, g - k) for k in range(0, g, SPLIT_ROWS)]
            continue
        if cur and cur + g > PANEL_ROWS:
            panels.append(cur)
            cur = 0
        cur += g
        if cur >= PANEL_ROWS:
            panels.append(cur)
            cur = 0
    if cur:
        panels.append(cur)
    nch = -(-n // ITEM_COLS)
    return len(panels), len(panels) * nch, sum(-(-r // STAGE_ROWS) for r in panels) * nch, panels


@pytest.mark.parametrize("sizes,n", [
    ([20] * 10, 200),                        # tiny: equal small groups, one ragged chunk
    ([1, 2, 3, 70, 5, 4100, 0, 9], 77),      # small + giant + empty, ragged n
    ([512, 511, 1, 513, 2, 510], 257),       # groups around the panel height (32 here), two chunks
    ([3] * 4000 + [700], 40000),             # tall panels (512 rows) and one larger group
    ([3] * 400, 1000),                       # many tiny groups: panels close on rows
])
def test_plan_covers_rows(sizes, n):
    lab = synth.labels_from_sizes(np.array(sizes))
    info = pk.ot_gs_plan_info(lab, n, len(sizes))
    n_panels, n_items, n_stages, panels = expected_plan(sizes, n)
    assert sum(panels) == len(lab)  # every row in exactly one panel
    assert (info["n_panels"], info["n_items"], info["n_stages"]) == (n_panels, n_items, n_stages)


def test_plan_zipf_large_shape():
    sizes = synth.class_sizes_zipf(20000, 1000, 1.1, 2)
    lab = synth.labels_from_sizes(sizes)
    info = pk.ot_gs_plan_info(lab, 20000, 1000)
    n_panels, n_items, n_stages, _ = expected_plan(list(sizes), 20000)
    assert (info["n_panels"], info["n_items"], info["n_stages"]) == (n_panels, n_items, n_stages)
    assert panel_height(20000, 20000) == 512
    assert int((np.asarray(sizes) > 512).sum()) < info["n_panels"] < 200
    # streaming one evaluation touches every row once per column chunk, in
    # 32-row stages: at most one partial stage per panel and chunk
    nch = -(-20000 // ITEM_COLS)
    assert info["n_stages"] <= (20000 // STAGE_ROWS + info["n_panels"]) * nch


def test_plan_rejects_bad_labels():
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_plan_info(np.array([0, 3, 1], np.int32), 5, 3)
