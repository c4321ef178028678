"""32-bit against 64-bit sort keys (Sec. 4.4), on the oracle (no GPU).

The paper packs the tile id and a truncated depth code into 32 bits and
states that this loses no quality against 64-bit keys.  Here the 64-bit
order (tile, full binary32 depth) is pinned to the depth it sorts by and to
the 32-bit order it refines, and the image difference between compositing in
the two orders is measured on the tiny, mid-size and large workloads (one
view each) and reported.
"""
import numpy as np
import pytest

from paper_2605_00219_gb300 import synth


def _workloads():
    tiny_sc, _, tiny_cams = synth.tiny_workload(0)
    mid_sc, _, mid_cams = synth.mid_workload(0)
    return {"tiny 2k 128x128": (lambda: tiny_sc, tiny_cams[0]),
            "mid 200k 1280x720": (lambda: mid_sc, mid_cams[0]),
            "large 3M 1920x1080": (lambda: synth.large_scene(0),
                                   synth.large_views(1, resolutions=[(1920, 1080)])[0])}


def test_sort64_orders_by_depth_and_refines_the_32bit_order(orc):
    sc, _, cams = synth.tiny_workload(1)
    cam = synth.look_at([3.0, -2.0, 1.5], [0.0, 0.0, 0.0], 160, 120, 140.0)   # 300 tiles: 9 tile bits
    b = orc.bin32(sc, cam)
    b64 = orc.sort64(b, cam)
    TX, TY = orc.tiles_of(cam)
    shift = orc.key_shift(TX * TY)
    tz = b.bin[:, 7]
    for t in range(TX * TY):
        s, e = b.ranges[t]
        g = b64.gidx[s:e].astype(np.int64)
        assert np.all((b64.keys[s:e] >> shift) == t)
        d = tz[g]
        assert np.all(np.diff(d) >= 0)
        same = np.diff(d) == 0
        assert np.all(np.diff(g)[same] > 0)          # equal depths keep index order
    # the truncated codes are monotone in depth: the 32-bit keys, taken in the
    # 64-bit order, are the 32-bit sorted keys
    np.testing.assert_array_equal(b.keys_emit[b64.perm], b.keys)
    assert sorted(b64.gidx.tolist()) == sorted(b.gidx.tolist())


@pytest.mark.parametrize("name", list(_workloads()))
def test_32bit_vs_64bit_key_image_difference(orc, report, name):
    make, cam = _workloads()[name]
    sc = make()
    b = orc.bin32(sc, cam)
    b64 = orc.sort64(b, cam)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    r32 = orc.render64(cam, P, b)
    r64 = orc.render64(cam, P, b64)
    d = np.abs(r32.image - r64.image)
    mse = float((d ** 2).mean())
    psnr = 10.0 * np.log10(1.0 / max(mse, 1e-30))
    TX, TY = orc.tiles_of(cam)
    report(f"keys_32_vs_64 {name}", {"tile_bits": orc.tile_bits(TX * TY), "depth_bits": 32 - orc.tile_bits(TX * TY)
                                     if orc.tile_bits(TX * TY) >= 9 else 23,
                                     "intersections": b.K, "entries_reordered": int((b.gidx != b64.gidx).sum()),
                                     "max_abs_diff": float(d.max()), "mean_abs_diff": float(d.mean()),
                                     "pixels_over_1e-3": int((d.max(-1) > 1e-3).sum()), "psnr_db": psnr})
    if orc.tile_bits(TX * TY) < 9:
        assert np.array_equal(r32.image, r64.image)   # all 23 code bits kept
    assert psnr > 50.0
