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


def test_warm_start_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks of the warm-start entry points run before any device
    call: they fail with OTGS_EINVAL and a message on a machine without a GPU."""
    L = pk.lib()
    P = ctypes.c_void_p
    one = (ctypes.c_int64 * 1)(1)
    ptrs = (P * 1)(P(16))
    fake = P(16)  # never dereferenced: the checks fail first
    # second-pass inputs: no problems; then columns past in_dim
    rc = L.ot_gs_mlp_refine_features(0, ptrs, one, one, one, fake, fake, 1.0, 0, 16, fake, None)
    assert rc == pk.OTGS_EINVAL
    rc = L.ot_gs_mlp_refine_features(1, ptrs, one, one, one, fake, fake, 1.0, 13, 16, fake, None)
    assert rc == pk.OTGS_EINVAL and "col0" in L.ot_gs_mlp_last_error(None).decode()
    # batched features: in_dim below 9 + 2 d
    lab = (P * 1)(P(16))
    Ls = (ctypes.c_int32 * 1)(1)
    rc = L.ot_gs_mlp_features_batch(1, ptrs, one, one, one, ptrs, ptrs, 8, lab, Ls, 1.0, 16, fake, None)
    assert rc == pk.OTGS_EINVAL and "in_dim" in L.ot_gs_mlp_last_error(None).decode()


def test_create_batch_rejects_bad_arguments_without_gpu():
    """ot_gs_create_batch checks its host arrays and scalars before it
    touches a device: no problems, a NULL array, an empty problem, ldc < n and
    a non-positive gamma all fail with OTGS_EINVAL and a message."""
    L = pk.lib()
    P = ctypes.c_void_p
    h = P()
    ptr = (P * 1)(P(16))
    i64 = lambda v: (ctypes.c_int64 * 1)(v)
    i32 = (ctypes.c_int32 * 1)(2)

    def create(nprob=1, C=ptr, ldc=i64(8), m=i64(4), n=i64(8), gamma=1.0):
        return L.ot_gs_create_batch(ctypes.byref(h), nprob, C, ldc, ptr, ptr, ptr, m, n, i32, gamma, 0.1, None)

    for kw, word in [(dict(nprob=0), "nprob"), (dict(C=None), "NULL"), (dict(m=i64(0)), "m, n"),
                     (dict(ldc=i64(4)), "ldc"), (dict(gamma=0.0), "gamma")]:
        assert create(**kw) == pk.OTGS_EINVAL and not h.value, kw
        assert word in pk.ot_gs_last_error(None), (kw, pk.ot_gs_last_error(None))


ITEM_COLS, STAGE_ROWS = 256, 32


def panel_height(m, n):
    """m * ceil(n / 256) / 2048 rows, clamped to [32, 128]."""
    return min(128, max(32, -(-m * -(-n // ITEM_COLS) // 2048)))


SPLIT_ROWS = 256
def panel_stages(groups, piece, fill=0):
    """Stages of a panel whose rows are the given groups (sizes, in order):
    runs of at most 32 rows; with fill > 0 a run ends early at the start of a
    group of at most 32 rows that would straddle its end when that keeps at
    least fill rows (never inside a piece of a split group)."""
    rows = int(sum(groups))
    if piece or fill == 0:
        return -(-rows // STAGE_ROWS)
    starts = np.concatenate([[0], np.cumsum(groups)])
    ra, cnt = 0, 0
    while ra < rows:
        cnt += 1
        nr = min(STAGE_ROWS, rows - ra)
        if ra + nr < rows:
            k = int(np.searchsorted(starts, ra + nr - 1, side="right")) - 1  # group of row ra + nr - 1
            gs, ge = int(starts[k]), int(starts[k + 1])
            if ge > ra + nr and ge - gs <= STAGE_ROWS and gs > ra and gs - ra >= fill:
                nr = gs - ra
        ra += nr
    return cnt


def plan_panels(sizes, panel_rows, split_rows):
    """Panels by the packing rule of the plan (consecutive non-empty groups up
    to the panel height; a group of more than split_rows rows cut into pieces
    of split_rows rows, each a panel) as (group sizes, is a piece)."""
    panels, cur = [], []
    for g in sizes:
        if g == 0:
            continue
        if g > split_rows:
            if cur:
                panels.append((cur, False))
                cur = []
            panels += [([min(split_rows, g - k)], True) for k in range(0, g, split_rows)]
            continue
        if cur and sum(cur) + g > panel_rows:
            panels.append((cur, False))
            cur = []
        cur = cur + [g]
        if sum(cur) >= panel_rows:
            panels.append((cur, False))
            cur = []
    if cur:
        panels.append((cur, False))
    return panels


def expected_plan(sizes, n):
    """Panels, items and stages of one problem."""
    panels = plan_panels(sizes, panel_height(int(np.sum(sizes)), n), SPLIT_ROWS)
    nch = -(-n // ITEM_COLS)
    rows = [int(sum(g)) for g, _ in panels]
    return len(panels), len(panels) * nch, sum(panel_stages(g, pc) for g, pc in panels) * nch, rows


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
    assert panel_height(20000, 20000) == 128
    assert int((np.asarray(sizes) > 128).sum()) < info["n_panels"] < 200
    # streaming one evaluation touches every row once per column chunk, in
    # 32-row stages: at most one partial stage per panel and chunk
    nch = -(-20000 // ITEM_COLS)
    assert info["n_stages"] <= (20000 // STAGE_ROWS + info["n_panels"]) * nch


def test_plan_rejects_bad_labels():
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_plan_info(np.array([0, 3, 1], np.int32), 5, 3)


def expected_plan_batch(sizes_list, ns, panel_rows=0, split_rows=0, fill=0):
    """A batch is planned problem by problem (a panel never holds rows of
    two problems, an item never pairs rows with another problem's columns);
    the default panel height comes from the (row, column chunk) pairs summed
    over the problems."""
    pairs = sum(int(np.sum(s)) * -(-n // ITEM_COLS) for s, n in zip(sizes_list, ns))
    pr = panel_rows or min(128, max(32, -(-pairs // 2048)))
    sr = split_rows or SPLIT_ROWS
    n_panels = n_items = n_stages = 0
    for sizes, n in zip(sizes_list, ns):
        panels = plan_panels(sizes, pr, sr)
        assert sum(int(sum(g)) for g, _ in panels) == int(np.sum(sizes))
        nch = -(-n // ITEM_COLS)
        n_panels += len(panels)
        n_items += len(panels) * nch
        n_stages += sum(panel_stages(g, pc, fill) for g, pc in panels) * nch
    return n_panels, n_items, n_stages


@pytest.mark.parametrize("pr,sr,sf", [(0, 0, 0), (32, 128, 0), (128, 256, 16), (512, 1024, 0), (1024, 64, 16),
                                      (512, 256, 1), (512, 256, 31)])
def test_batch_plan_is_per_problem(pr, sr, sf):
    rng = np.random.default_rng(5)
    sizes_list, ns = [], []
    for k in range(9):
        L = int(rng.integers(1, 30))
        sizes = rng.integers(0, 200, size=L)
        if k == 3:
            sizes[0] = 1300  # a tall group: pieces
        sizes[-1] = max(sizes[-1], 1)
        sizes_list.append(sizes)
        ns.append(int(rng.integers(1, 700)))
    labels = [synth.labels_from_sizes(s) for s in sizes_list]
    info = pk.ot_gs_plan_info_batch(labels, ns, [len(s) for s in sizes_list], pr, sr, sf)
    assert (info["n_panels"], info["n_items"], info["n_stages"]) == expected_plan_batch(sizes_list, ns, pr, sr, sf)


def test_batch_of_one_plans_like_one_problem():
    sizes = [1, 2, 3, 70, 5, 4100, 0, 9]
    lab = synth.labels_from_sizes(np.array(sizes))
    a = pk.ot_gs_plan_info(lab, 77, len(sizes))
    b = pk.ot_gs_plan_info_batch([lab], [77], [len(sizes)])
    assert a == b


def test_batch_plan_rejects_bad_input():
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_plan_info_batch([np.array([0, 1], np.int32), np.array([0, 5], np.int32)], [4, 4], [2, 2])
    h = ctypes.c_void_p()
    rc = pk.lib().ot_gs_create_batch(ctypes.byref(h), 0, None, None, None, None, None, None, None, None,
                                     1.0, 0.1, None)
    assert rc == pk.OTGS_EINVAL and not h.value
    assert "nprob" in pk.ot_gs_last_error(None)
