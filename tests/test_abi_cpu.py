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


@pytest.mark.parametrize("sizes,n", [
    ([20] * 10, 200),                 # tiny: equal small groups
    ([1, 2, 3, 70, 5, 4100, 0, 9], 77),  # small + big + giant + empty, ragged n
    ([64, 65, 1], 33),                # boundary of the small/big split
])
def test_plan_covers_rows(sizes, n):
    lab = synth.labels_from_sizes(np.array(sizes))
    info = pk.ot_gs_plan_info(lab, n, len(sizes))
    assert info["n_panels"] >= 1 and info["n_items"] >= info["n_panels"]
    # every non-empty row appears in exactly one panel per column chunk:
    # rowpart length = sum over panels of rows * chunks, bounded by m * n / 32
    m = len(lab)
    assert m <= info["rowpart_len"] <= m * ((n + 31) // 32)


def test_plan_zipf_large_shape():
    sizes = synth.class_sizes_zipf(20000, 1000, 1.1, 2)
    lab = synth.labels_from_sizes(sizes)
    info = pk.ot_gs_plan_info(lab, 20000, 1000)
    assert 50 < info["n_panels"] < 400
    assert info["n_items"] > 1000


def test_plan_rejects_bad_labels():
    with pytest.raises(pk.OTGSError):
        pk.ot_gs_plan_info(np.array([0, 3, 1], np.int32), 5, 3)
