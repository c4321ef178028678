"""The C-ABI library loads and exports every symbol include/gs_step.h
declares; plan creation validates its arguments (host only, no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs_step.h")


@pytest.fixture(scope="module")
def gslib():
    from paper_2605_00219_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    build.build()
    from paper_2605_00219_gb300 import gsstep
    return gsstep


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_stage_calls():
    names = _declared()
    for n in ["gs_project_fwd", "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd", "gs_project_bwd_adam"]:
        assert n in names


def test_library_exports_every_declared_symbol(gslib):
    L = ctypes.CDLL(gslib.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(gslib.SYMBOLS) == _declared()


def test_plan_validation(gslib):
    P = gslib.Plan([2000], [(128, 128, 0)])
    assert P.pairs == 2000 and P.tiles == 64 and P.pixels == 128 * 128
    assert P.capacity >= 8 * 2000 and P.capacity % 2048 == 0
    assert P.workspace_bytes() > 0
    P2 = gslib.Plan([10, 20], [(100, 50, 1), (33, 17, 0)], tile=(8, 8))
    assert P2.pairs == 30 and P2.tiles == 13 * 7 + 5 * 3
    for bad in [dict(scene_sizes=[0], views=[(8, 8, 0)]),
                dict(scene_sizes=[5], views=[(8, 8, 1)]),
                dict(scene_sizes=[5], views=[(0, 8, 0)]),
                dict(scene_sizes=[5], views=[(8, 8, 0)], tile=(12, 12)),
                dict(scene_sizes=[5], views=[(8, 8, 0)], bwd_batch=48),
                dict(scene_sizes=[5], views=[(8, 8, 0)] * 65)]:
        with pytest.raises(gslib.GSError):
            gslib.Plan(**bad)


def test_status_strings(gslib):
    L = gslib.lib()
    for code in range(7):
        assert L.gs_status_str(code)
