"""Host-side facts the CUDA path relies on, checked without a GPU.

- The launch count that bench.py claims per step equals the count in the ncu
  launch list of the 4 x 1920x1080 workload at 16x16 tiles (one graph-replayed
  step launches 17 kernels of this library), whatever the views.
- The compile-time window taps of the L1 + SSIM kernel are the oracle's
  normalised Gaussian window (11 taps, sigma 1.5) rounded to FP32.
- The algorithmic work per stage behind the bench's rooflines, and the
  roofline records built from it.
"""
import os
import re
import types

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _plan(views, tile=(16, 16)):
    return types.SimpleNamespace(views=[(w, h, 0) for (w, h) in views], tile=tile)


def test_launch_count_matches_the_measured_launch_list():
    assert bench.launches_per_step(_plan([(1920, 1080)] * 4)) == 17


def test_launch_count_does_not_depend_on_the_views():
    assert bench.launches_per_step(_plan([(1920, 1080)])) == 17
    assert bench.launches_per_step(_plan([(64, 64)] * 16, tile=(8, 8))) == 17


def test_ssim_window_constants_are_the_oracle_window_in_fp32(orc):
    src = open(os.path.join(ROOT, "paper_2605_00219_gb300", "csrc", "loss_ssim.cu")).read()
    body = src[src.index("constexpr float ssim_w(int k)"):]
    body = body[:body.index("}")]
    # the function lists the taps symmetric about the centre: 0/10, 1/9, ..., 5
    pairs = re.findall(r"\(k == (\d+) \|\| k == (\d+)\)\s*\?\s*([0-9.]+)f", body)
    centre = re.findall(r":\s*([0-9.]+)f;", body)
    assert len(pairs) == 5 and len(centre) == 1
    taps = np.zeros(11, np.float32)
    for a, b, v in pairs:
        taps[int(a)] = taps[int(b)] = np.float32(float(v))
    taps[5] = np.float32(float(centre[0]))
    ref = orc.ssim_window(11, 1.5).astype(np.float32)
    assert np.array_equal(taps, ref), (taps, ref)
    assert abs(float(taps.astype(np.float64).sum()) - 1.0) < 1e-7


def test_stage_work_headline_figures():
    """Algorithmic work of the 3M-Gaussian, 4 x 1920x1080 BF16 step from the
    per-unit figures of the method: 140 B of parameters read per Gaussian and
    48 B written per pair by the projection; 752 B per Gaussian and 36 B per
    intersection for the fused Adam; the raster kernels charged 14 operations
    per evaluated pair and 13 (forward) or 31 (backward) per blended one."""
    K, px, ev, bl, tiles = 17_269_857, 4 * 1920 * 1080, 3_715_163_821, 358_000_000, 4 * 8160
    w = bench.stage_work([3_000_000], [0, 0, 0, 0], K, ev, bl, px, tiles, sh16=True)
    pairs = 12_000_000
    assert w["project_fwd"] == ("hbm", 3_000_000 * 140 + pairs * 48)
    assert w["project_bwd_adam"] == ("hbm", 3_000_000 * 752 + K * 36 + pairs * 8)
    assert w["bin_sort"] == ("hbm", pairs * 16 + K * 16 + tiles * 8)
    assert w["loss_l1"] == ("hbm", px * 36)
    assert w["raster_bwd"] == ("alu", 2.0 * (ev * 14 + bl * 31))
    assert w["raster_fwd"] == ("alu", 2.0 * (ev * 14 + bl * 13))
    # the backward at the recorded 5.28 ms: about 0.30 of the FP32 peak
    r = bench.stage_rooflines(w, {k: 1.0 for k in w} | {"raster_bwd": 5.28}, 6777.0, 80.54784)
    assert abs(r["raster_bwd"]["frac"] - 0.30) < 0.01
    assert set(w) == {"project_fwd", "bin_sort", "raster_fwd", "loss_l1", "raster_bwd", "project_bwd_adam"}


def test_stage_work_counts_each_views_own_scene():
    """Eight scenes with two views each: a view pairs only with the Gaussians
    of its own scene (24M pairs, not 12M x 16)."""
    sizes = [500_000, 500_000, 750_000, 750_000, 1_000_000, 1_250_000, 1_250_000, 6_000_000]
    views = [s for s in range(8) for _ in range(2)]
    w = bench.stage_work(sizes, views, 30_000_000, 1, 1, 1, 1, sh16=True)
    n = sum(sizes)
    assert w["project_fwd"][1] == n * 140 + 2 * n * 48
    assert w["project_bwd_adam"][1] == n * 752 + 30_000_000 * 36 + 2 * n * 8


def test_stage_work_ssim_loss_is_alu_work():
    w = bench.stage_work([1000], [0], 10, 10, 5, 100, 4, sh16=False, loss="l1_ssim")
    assert "loss_l1" not in w and w["loss_l1_ssim"] == ("alu", 100 * 3 * 209 * 2)
    assert w["project_fwd"][1] == 1000 * 236 + 1000 * 48     # FP32 SH
    assert w["project_bwd_adam"][1] == 1000 * 1416 + 10 * 36 + 1000 * 8
    assert w["bin_sort"][1] == 1000 * 16 + 10 * 16 + 4 * 8


def test_stage_rooflines_units_and_fractions():
    work = {"project_fwd": ("hbm", 1.248e9), "raster_bwd": ("alu", 3.7e9 * 90.0)}
    r = bench.stage_rooflines(work, {"project_fwd": 0.729, "raster_bwd": 5.273}, 6777.0, 80.54784)
    assert r["project_fwd"]["unit"] == "GB/s" and abs(r["project_fwd"]["achieved"] - 1.248e9 / 0.729e-3 / 1e9) < 1e-9
    assert abs(r["project_fwd"]["frac"] - r["project_fwd"]["achieved"] / 6777.0) < 1e-12
    assert r["raster_bwd"]["bound"] == "alu" and r["raster_bwd"]["unit"] == "TFLOP/s"
    assert abs(r["raster_bwd"]["achieved"] - 63.15) < 0.01
    assert all(x["traffic"] is None for x in r.values())
