"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point declared in include/uvc.h, and the binding's host logic."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2103_14137_gb300 as uvc
    uvc.build()
    return uvc.library()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(uvc_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("uvc_build_scene", "uvc_irradiance_matrix", "uvc_fluence", "uvc_fluence_streamed",
                     "uvc_coverage", "uvc_free_scene", "uvc_status_string", "uvc_scene_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    import paper_2103_14137_gb300 as uvc
    assert uvc.status_string(0) == "ok"
    assert "invalid" in uvc.status_string(1)
    assert uvc.status_string(999) == "unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    P = ctypes.c_void_p
    out = P()
    # NULL out pointer and negative counts are rejected on the host
    assert lib.uvc_build_scene(None, 0, None, 0, None, 0, None, None) == 1
    assert lib.uvc_build_scene(None, -1, None, 0, None, 0, None, ctypes.byref(out)) == 1
    assert lib.uvc_irradiance_matrix(None, None, 0, None, None, 0, None, None) == 1
    assert lib.uvc_fluence(None, None, 0, 0, None, 1, None, None) == 1
    assert lib.uvc_coverage(None, None, 1, 1.0, None, None, None) == 1
    assert lib.uvc_scene_status(None, None) == 1
    assert lib.uvc_scene_set_limits(None, 0, 0) == 1
    assert lib.uvc_free_scene(None) == 0
    assert lib.uvc_candidate_features(None, None, 0, None, 66, None) == 1
    assert lib.uvc_probe_features(None, 1, 10, 10, None, None, None, 47, None) == 1      # ldf < 48
    assert lib.uvc_select_top(None, 20000, 1, None, None, None, None) == 1      # n above 16384
    assert lib.uvc_select_top(None, 10, 11, None, None, None, None) == 1        # k > n
    assert lib.uvc_mlp_create(0, 256, 16, 0, ctypes.byref(out)) == 1           # in_dim < 1
    assert lib.uvc_mlp_create(66, 250, 16, 0, ctypes.byref(out)) == 1          # hidden not a multiple of 8
    assert lib.uvc_mlp_create(66, 256, 0, 0, ctypes.byref(out)) == 1           # max_batch < 1
    assert lib.uvc_mlp_forward(None, None, 1, None, None) == 1
    assert lib.uvc_mlp_train_step(None, None, None, None, 1, ctypes.c_float(1e-3), None, None) == 1
    assert lib.uvc_mlp_param_count(None) == -1
    assert lib.uvc_mlp_free(None) == 0


def test_lamp_struct_layout():
    from paper_2103_14137_gb300.uvc import Lamp, _Lamp
    from synth import line_lamp
    assert ctypes.sizeof(_Lamp) == 4 + 4 + 32 * 3 * 4 + 32 * 4
    g = line_lamp(1.2, 8, 120.0)
    c = Lamp(g.offsets, g.weights, g.power)._c()
    assert c.K == 8 and abs(c.power - 120.0) < 1e-6
    assert np.allclose([c.offsets[m][2] for m in range(8)], 1.2 * (np.arange(8) + 0.5) / 8)
    assert np.isclose(sum(c.weight[m] for m in range(8)), 1.0)


def test_vis_unpacking():
    import torch
    from paper_2103_14137_gb300.uvc import vis_to_bool
    w = torch.tensor([[[0b101, -2147483648]]], dtype=torch.int32)   # K=1, nc=1, 2 words
    b = vis_to_bool(w, 40)
    assert b.shape == (1, 40, 1)
    assert b[0, :, 0].nonzero()[0].tolist() == [0, 2]
    w = torch.tensor([[[0, -2147483648]]], dtype=torch.int32)
    assert vis_to_bool(w, 64)[0, :, 0].nonzero()[0].tolist() == [63]


def test_product_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2103_14137_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("no oracle", ""), f


def test_wedge_switch_is_host_only(lib):
    """uvc_set_wedge_traversal returns the previous setting and rejects other values."""
    import paper_2103_14137_gb300 as uvc
    prev = ctypes.c_int32(-1)
    assert lib.uvc_set_wedge_traversal(2, ctypes.byref(prev)) == 1      # UVC_E_INVAL, nothing written
    assert prev.value == -1
    assert uvc.set_wedge_traversal(False) is True and uvc.set_wedge_traversal(True) is False
    assert lib.uvc_set_wedge_traversal(1, ctypes.byref(prev)) == 0 and prev.value == 1
    assert lib.uvc_set_wedge_traversal(1, None) == 0


def test_host_only_entry_points_through_the_package(lib):
    """The package re-exports the host-only calls: the matrix kernel's task
    shape (the counting replay needs it) and the fluence kernel switch."""
    import paper_2103_14137_gb300 as uvc
    assert uvc.irradiance_candidates_per_task() >= 1
    assert uvc.set_fluence_tensor_cores(False) is True      # the default: tensor cores
    assert uvc.set_fluence_tensor_cores(True) is False
    prev = ctypes.c_int32(-1)
    assert lib.uvc_set_fluence_tensor_cores(2, ctypes.byref(prev)) == 1   # UVC_E_INVAL, unchanged
    assert prev.value == -1 and uvc.set_fluence_tensor_cores(True) is True


def test_matrix_row_layouts():
    """The binding passes the library a row stride only for layouts it can
    read and write in bounds: padded rows are fine, too few rows or columns
    and overlapping rows are refused (host logic, no GPU)."""
    from paper_2103_14137_gb300.uvc import _row_layout
    assert _row_layout((4, 10), (10, 1), "A", 4, 10) == 10            # contiguous
    assert _row_layout((4, 10), (16, 1), "A", 4, 10) == 16            # view of a wider buffer
    assert _row_layout((4, 12), (12, 1), "A", 4, 10) == 12            # more columns than written
    assert _row_layout((1, 10), (99, 1), "A", 1, 10) == 10            # one row: its stride is unused
    assert _row_layout((0, 10), (10, 1), "A", 0, 10) == 10            # no rows
    for shape, strides, exc in (((3, 10), (10, 1), ValueError),        # wrong row count
                                ((4, 9), (16, 1), ValueError),         # narrower view than the columns written
                                ((4, 10), (1, 4), ValueError),         # transposed (column stride 4)
                                ((4, 10), (5, 1), ValueError),         # overlapping rows
                                ((4,), (1,), TypeError)):
        with pytest.raises(exc):
            _row_layout(shape, strides, "A", 4, 10)
