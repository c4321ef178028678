"""Parity at the benchmark's full size and launch configuration (3M
Gaussians, 16x16 tiles, pixel-parallel raster backward): every sorted key and
sorted Gaussian bit-exact against the oracle's FP32 binning (one 1080p view,
and the four-view batch), images and gradients on a sample of tiles that the
FP64 oracle evaluates one by one."""
import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu

N = 3_000_000
TILE_STRIDE = 97   # sampled tiles: every 97th
# Threshold-flag margin for this size: FP32 pixel means near x ~ 1000 px carry
# ~1e-4 px of error, which moves d^2 by up to ~1.1e-3 for the smallest
# footprints (sigma^2 = 0.3 px^2 low-pass), i.e. ~1.2e-4 relative -- above the
# 1e-4 used at 128x128.  1e-3 keeps a factor of about eight.
MARGIN = 1e-3


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep, step
    return gsstep, step, synth.large_scene(0, N)


def test_fullsize_single_view_keys_image_gradients(big, orc, report):
    gsstep, step, scene = big
    cam = synth.large_views(1, resolutions=[(1920, 1080)])[0]
    tr = step.Trainer([scene], [cam], lr=(1e-3,) * 6)
    tr.forward()
    torch.cuda.synchronize()
    st = tr.stats()
    b = orc.bin32(scene, cam)
    assert st.status == 0 and st.k_required == b.K
    np.testing.assert_array_equal(tr.buffer(2, b.K).cpu().numpy().view(np.uint32), b.keys)
    np.testing.assert_array_equal(tr.buffer(3, b.K).cpu().numpy().view(np.uint32), b.gidx)
    # images on sampled tiles
    ntiles = b.ranges.shape[0]
    keep = np.zeros(ntiles, bool)
    keep[::TILE_STRIDE] = True
    bs = orc.Binning(b.count, b.bin, b.mant, b.offset, b.keys_emit, b.gidx_emit, b.keys, b.gidx, b.perm,
                     np.where(keep[:, None], b.ranges, 0))
    p = orc.Params64.from_scene(scene)
    P = orc.project64(p, cam)
    r = orc.render64(cam, P, bs, margin=MARGIN)
    TX = 120
    tiles_px = (np.arange(1080)[:, None] // 16) * TX + (np.arange(1920)[None, :] // 16)
    sampled_px = keep[tiles_px]
    ok = sampled_px & ~r.unstable_px
    img = tr.image.view(1080, 1920, 3).cpu().numpy().astype(np.float64)
    assert ok.sum() > 0.9 * sampled_px.sum()
    assert np.abs(img - r.image)[ok].max() <= 1e-5
    # gradients: per Gaussian, summed over its intersections in sampled tiles
    rng = np.random.default_rng(0)
    dl = (rng.normal(size=(1080, 1920, 3)) / (3 * 1080 * 1920)).astype(np.float32)
    tr.dl.copy_(torch.from_numpy(dl.reshape(-1, 3)))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    torch.cuda.synchronize()
    g2_orc = orc.raster_bwd64(cam, P, bs, dl.astype(np.float64))
    K = b.K
    gr = gsstep.gs_gradient_records(tr.plan, tr.ws, K).cpu().numpy().astype(np.float64)
    slots = tr.buffer(9, K).cpu().numpy().view(np.uint32).astype(np.int64)   # emission slot per sorted entry
    sorted_tile = b.keys >> orc.key_shift(ntiles)
    in_sample = keep[sorted_tile]
    g2_gpu = np.zeros_like(g2_orc)
    np.add.at(g2_gpu, b.gidx[in_sample].astype(np.int64), gr[slots[in_sample]])
    touched = np.zeros(scene.n, bool)
    touched[b.gidx[in_sample]] = True
    bad = r.unstable_g.copy()
    ys, xs = np.nonzero(r.unstable_px & sampled_px)
    for x, y in zip(xs, ys):
        dx, dy = x + 0.5 - P[:, 4], y + 0.5 - P[:, 5]
        d2 = P[:, 9] * dx * dx + 2 * P[:, 10] * dx * dy + P[:, 11] * dy * dy
        bad |= (P[:, 0] > 0) & (d2 <= 9.0 * 1.001)
    good = touched & ~bad
    assert good.sum() > 0.25 * touched.sum() and good.sum() > 5000
    ref, got = g2_orc[good], g2_gpu[good]
    rms = np.sqrt((ref ** 2).mean(0)) + 1e-30
    err = np.abs(got - ref) / np.maximum(np.abs(ref), rms[None, :])
    assert err.max() <= 1e-3, err.max()
    report("config2_1080p_sampled_tiles",
           {"keys": int(K), "keys_bit_exact": True, "image_max_abs_err": float(np.abs(img - r.image)[ok].max()),
            "sampled_pixels": int(sampled_px.sum()), "excluded_pixels": int(sampled_px.sum() - ok.sum()),
            "grad2d_max_rel_err": float(err.max()), "gaussians_touched": int(touched.sum()),
            "excluded_gaussians": int(touched.sum() - good.sum())})


def test_fullsize_four_view_batch_keys(big, orc):
    """The batched workload's four 1080p views: per-view key segments and
    sorted pair indices bit-exact (exercises the view pass at full size)."""
    gsstep, step, scene = big
    cams = synth.large_views(4, resolutions=[(1920, 1080)])
    tr = step.Trainer([scene], cams, lr=(1e-3,) * 6, sh_bf16=True, mom_bf16=True)
    tr.forward()
    torch.cuda.synchronize()
    st = tr.stats()
    bins = [orc.bin32(scene, c) for c in cams]
    K = sum(b.K for b in bins)
    assert st.status == 0 and st.k_required == K
    keys = tr.buffer(2, K).cpu().numpy().view(np.uint32)
    pids = tr.buffer(3, K).cpu().numpy().view(np.uint32)
    o = 0
    for v, b in enumerate(bins):
        np.testing.assert_array_equal(keys[o:o + b.K], b.keys)
        np.testing.assert_array_equal(pids[o:o + b.K], b.gidx + v * scene.n)
        o += b.K


def test_fullsize_uneven_batch_500_fp32_steps(big):
    """The batched configuration's own form: four views of uneven resolution
    (1920x1080, 1600x1064, 1280x720, 960x540), FP32 storage, 500
    graph-replayed steps: status clear, loss falls, parameters finite."""
    gsstep, step, scene = big
    cams = synth.large_views(4)
    tscene = synth.perturbed(scene, 1)
    t = step.Trainer([tscene], cams, lr=(1e-3,) * 6)
    t.forward()
    torch.cuda.synchronize()
    target = t.image.clone()
    del t
    tr = step.Trainer([scene], cams, lr=(1.6e-4 * 30.0, 1e-3, 5e-3, 5e-2, 2.5e-3, 2.5e-3 / 20))
    tr.target.copy_(target)
    tr.step(0)
    first = float(tr.stats().loss)
    tr.capture()
    for _ in range(499):
        tr.replay()
    torch.cuda.synchronize()
    st = tr.stats()
    assert st.status == 0 and st.step == 500
    assert float(st.loss) < 0.5 * first
    assert bool(torch.isfinite(tr.scenes[0].geom).all()) and bool(torch.isfinite(tr.scenes[0].sh).all())
