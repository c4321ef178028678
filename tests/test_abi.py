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
                dict(scene_sizes=[5], views=[(8, 8, 0)], threads_per_tile=100),
                dict(scene_sizes=[5], views=[(8, 8, 0)], tile=(8, 8), threads_per_tile=16),
                dict(scene_sizes=[5], views=[(8, 8, 0)], threads_per_tile=128, bwd_impl=1),
                dict(scene_sizes=[5], views=[(8, 8, 0)], threads_per_tile=64, bwd_impl=2),
                dict(scene_sizes=[5], views=[(8, 8, 0)] * 65)]:
        with pytest.raises(gslib.GSError):
            gslib.Plan(**bad)


def test_threads_per_tile_choices(gslib):
    """One, two or (16-wide tiles) four pixels per raster thread; the
    autotuner's candidates are exactly the accepted combinations."""
    from paper_2605_00219_gb300 import autotune
    for tile in autotune.TILES:
        np_ = tile[0] * tile[1]
        for tpt in (0, np_, np_ // 2, np_ // 4, np_ // 8):
            ok = tpt in (0, np_, np_ // 2) or (tile[0] == 16 and tpt == np_ // 4)
            for impl in (0, 1, 2):
                accept = ok and (impl == 0 or tpt in (0, np_))
                try:
                    gslib.Plan([5], [(40, 40, 0)], tile=tile, bwd_impl=impl, threads_per_tile=tpt)
                    got = True
                except gslib.GSError:
                    got = False
                assert got == accept, (tile, tpt, impl)
    cands = autotune.default_candidates()
    assert len(cands) == len(set(cands)) == 14
    for tile, impl, tpt in cands:
        gslib.Plan([5], [(40, 40, 0)], tile=tile, bwd_impl=impl, threads_per_tile=tpt)


def test_status_strings(gslib):
    L = gslib.lib()
    for code in range(7):
        assert L.gs_status_str(code)
