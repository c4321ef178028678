"""Host-side facts the CUDA path relies on, checked without a GPU.

- The launch count that bench.py claims per step equals the count in the ncu
  launch list of the 4 x 1920x1080 workload at 16x16 tiles (one graph-replayed
  step launched 40 kernels of this library; the launch-list profile under
  profiles/).
- The compile-time window taps of the L1 + SSIM kernel are the oracle's
  normalised Gaussian window (11 taps, sigma 1.5) rounded to FP32.
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
    assert bench.launches_per_step(_plan([(1920, 1080)] * 4)) == 40


def test_launch_count_single_view_has_no_view_pass():
    # one view: the view pass of the radix sort (count, 3 scan launches,
    # reorder) is not launched
    assert bench.launches_per_step(_plan([(1920, 1080)])) == 40 - 5


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
