"""Parity of the CUDA step (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated by the target of the build, applied here):
  - tile counts, keys, sorted lists and tile ranges: bit-exact;
  - images: max |C_gpu - C_fp64| <= 1e-5 on pixels whose decisions are not
    within 1e-4 (relative) of a threshold (1/255, 0.99, 9, 1e-4); the count
    of excluded pixels is reported;
  - gradients: |g_gpu - g_fp64| <= 1e-3 max(|g_fp64|, rms of the component)
    on Gaussians not touching an excluded pixel;
  - post-Adam parameters: |theta_gpu - theta_fp64| <= 1e-5 |theta| + 1e-6
    where the first-step update direction is decided (|g| above 1e-2 rms).
"""
import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu

LR = (1e-3,) * 6


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep, step
    return gsstep, step


def _oracle_all(orc, scene, cam, tile, dl=None, bg=(0.0, 0.0, 0.0)):
    b = orc.bin32(scene, cam, *tile)
    p = orc.Params64.from_scene(scene)
    P = orc.project64(p, cam, *tile)
    r = orc.render64(cam, P, b, bg, 1e-4, *tile)
    return b, p, P, r


def _unstable_gaussians(P, r, cam):
    """Gaussians flagged by the oracle or covering (d^2 <= 9) a flagged pixel."""
    bad = r.unstable_g.copy()
    ys, xs = np.nonzero(r.unstable_px)
    for x, y in zip(xs, ys):
        dx = x + 0.5 - P[:, 4]
        dy = y + 0.5 - P[:, 5]
        d2 = P[:, 9] * dx * dx + 2 * P[:, 10] * dx * dy + P[:, 11] * dy * dy
        bad |= (P[:, 0] > 0) & (d2 <= 9.0 * (1 + 1e-3))
    return bad


def _run_forward(step_mod, scene, cams, tile=(16, 16), bwd_batch=0, bg=None, capacity=0, bwd_impl=0, tpt=0):
    tr = step_mod.Trainer([scene], cams, capacity=capacity, tile=tile, bwd_batch=bwd_batch, bg=bg, lr=LR,
                          bwd_impl=bwd_impl, threads_per_tile=tpt)
    tr.forward()
    torch.cuda.synchronize()
    return tr


def _sum_slots(grad_slots, offset, count):
    n = count.shape[0]
    out = np.zeros((n, 9))
    for g in range(n):
        c = int(count[g])
        if c:
            out[g] = grad_slots[offset[g]:offset[g] + c, :9].astype(np.float64).sum(0)
    return out


def _check_grad(gpu, ref, mask, name, tol=1e-3):
    ref_m, gpu_m = ref[mask], gpu[mask]
    rms = np.sqrt((ref_m ** 2).mean(0)) + 1e-30
    bound = tol * np.maximum(np.abs(ref_m), rms[None, :])
    err = np.abs(gpu_m - ref_m)
    worst = (err / np.maximum(np.abs(ref_m), rms[None, :])).max()
    assert np.all(err <= bound), f"{name}: worst relative error {worst:.3e}"
    return worst


@pytest.mark.parametrize("seed,bwd_impl", [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_tiny_stages(gs, orc, report, seed, bwd_impl):
    """2,000 Gaussians, 128x128: every stage against the oracle (both
    raster-backward implementations)."""
    gsstep, step_mod = gs
    scene, tscene, cams = synth.tiny_workload(seed)
    cam = cams[0]
    b, p, P, r = _oracle_all(orc, scene, cam, (16, 16))
    tr = _run_forward(step_mod, scene, cams, bwd_impl=bwd_impl)
    n = scene.n
    # --- projection: counts bit-exact, means/depth bit-exact, conic/colour close
    count = tr.buffer(0, n).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(count, b.count)
    rec = tr.buffer(7, n * 12, torch.float32).cpu().numpy().reshape(n, 12)
    vis = b.count > 0
    np.testing.assert_array_equal(rec[vis, 0], b.bin[vis, 1])
    np.testing.assert_array_equal(rec[vis, 1], b.bin[vis, 2])
    np.testing.assert_array_equal(rec[vis, 9], b.bin[vis, 7])
    # conic entries relative to the conic's scale (the off-diagonal can be ~0)
    con_g, con_o = rec[vis][:, [2, 3, 4]], P[vis][:, [9, 10, 11]]
    scale = np.abs(con_o).max(1, keepdims=True)
    assert (np.abs(con_g - con_o) / scale).max() <= 1e-4
    np.testing.assert_allclose(rec[vis][:, [6, 7, 8]], P[vis][:, [16, 17, 18]], atol=1e-5)
    # --- binning: sorted keys, sorted Gaussians and ranges bit-exact
    st = tr.stats()
    assert st.status == 0 and st.k_required == b.K
    keys = tr.buffer(2, b.K).cpu().numpy().view(np.uint32)
    pids = tr.buffer(3, b.K).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys, b.keys)
    np.testing.assert_array_equal(pids, b.gidx)
    ranges = tr.buffer(4, 2 * 64).cpu().numpy().view(np.uint32).reshape(64, 2)
    np.testing.assert_array_equal(ranges.astype(np.int64), b.ranges)
    # --- raster forward
    img = tr.image.view(128, 128, 3).cpu().numpy().astype(np.float64)
    ok = ~r.unstable_px
    err = np.abs(img - r.image)[ok].max()
    assert err <= 1e-5, err
    assert r.unstable_px.sum() < 0.01 * ok.size
    nl = tr.buffer(5, 128 * 128).cpu().numpy().reshape(128, 128)
    np.testing.assert_array_equal(nl[ok], r.nlast[ok])
    assert abs(int(st.blended_pairs) - r.blended) <= int(r.unstable_px.sum()) * 8
    # --- raster backward with the oracle's dL/dC (FP32-cast)
    rng = np.random.default_rng(seed + 10)
    dl64 = rng.normal(size=(128, 128, 3)) / (3 * 128 * 128)
    tr.dl.copy_(torch.from_numpy(dl64.astype(np.float32).reshape(-1, 3)))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    g2_orc = orc.raster_bwd64(cam, P, b, dl64.astype(np.float32).astype(np.float64))
    gr = gsstep.gs_gradient_records(tr.plan, tr.ws, b.K).cpu().numpy()
    off = tr.buffer(1, n + 1).cpu().numpy().view(np.uint32).astype(np.int64)
    g2_gpu = _sum_slots(gr, off, count)
    good = vis & ~_unstable_gaussians(P, r, cam)
    assert good.sum() > 0.7 * vis.sum()
    w2 = _check_grad(g2_gpu, g2_orc, good, "grad2d")
    # --- projection backward, gradient-only mode (activated parameters)
    grads = torch.zeros((15, n, 4), dtype=torch.float32, device="cuda")
    gsstep.gs_project_bwd_adam(tr.plan, tr.ws, tr.scenes, tr.cams, None, grads)
    torch.cuda.synchronize()
    g = grads.cpu().numpy()
    gth = orc.project_bwd64(p, cam, P, g2_orc)
    ref = np.concatenate([gth[:, 0:3], gth[:, 3:7], gth[:, 7:10] / p.scales,
                          (gth[:, 10] / (p.opacities * (1 - p.opacities)))[:, None], gth[:, 11:]], axis=1)
    gpu = np.concatenate([g[0, :, :3], g[1], g[2], g[3:].transpose(1, 0, 2).reshape(n, 48)], axis=1)
    w3 = _check_grad(gpu, ref, good, "grad3d")
    report(f"config0_stages_seed{seed}_impl{bwd_impl}",
           {"image_max_abs_err": float(err), "excluded_pixels": int(r.unstable_px.sum()), "pixels": int(ok.size),
            "conic_max_rel_err": float((np.abs(con_g - con_o) / scale).max()),
            "colour_max_abs_err": float(np.abs(rec[vis][:, [6, 7, 8]] - P[vis][:, [16, 17, 18]]).max()),
            "grad2d_max_rel_err": float(w2), "grad3d_max_rel_err": float(w3),
            "excluded_gaussians": int(vis.sum() - good.sum()), "visible_gaussians": int(vis.sum()),
            "keys": int(b.K), "keys_bit_exact": True})


def test_tiny_full_step_adam(gs, orc, report):
    """Whole step (device L1 gradient, fused Adam) vs the oracle's step."""
    gsstep, step_mod = gs
    scene, tscene, cams = synth.tiny_workload(0)
    cam = cams[0]
    tb, tp, tP, tr_ = _oracle_all(orc, tscene, cam, (16, 16))
    target = tr_.image
    res = orc.step(scene, cams, [target], LR, 1)
    tr = step_mod.Trainer([scene], cams, lr=LR)
    tr.set_target([target.astype(np.float32)])
    tr.step(step=1)
    torch.cuda.synchronize()
    st = tr.stats()
    assert st.status == 0
    assert st.loss == pytest.approx(res.loss, rel=1e-4)
    r = res.renders[0]
    img = tr.image.view(128, 128, 3).cpu().numpy()
    # pixels where the loss sign is not decided in FP32 join the excluded set
    undecided = (np.abs(r.image - target) < 1e-5).any(-1)
    r.unstable_px |= undecided
    bad = _unstable_gaussians(res.projs[0], r, cam)
    new = tr.scenes[0].to_scene()
    th_gpu = np.concatenate([new.means, new.quats, np.log(new.scales), np.log(new.opacities / (1 - new.opacities))[:, None],
                             new.sh.reshape(-1, 48)], axis=1).astype(np.float64)
    g = res.grad
    rms = np.sqrt((g[~bad] ** 2).mean(0)) + 1e-30
    decided = (np.abs(g) > 1e-2 * rms[None, :]) & ~bad[:, None]
    zero = (g == 0) & ~bad[:, None]
    assert decided.sum() > 0.5 * g.size
    diff = np.abs(th_gpu - res.theta)
    tol = 1e-5 * np.abs(res.theta) + 1e-6
    assert np.all(diff[decided] <= tol[decided]), diff[decided].max()
    assert np.all(diff[zero] <= tol[zero])
    report("config0_full_step_adam",
           {"loss_rel_err": abs(st.loss - res.loss) / res.loss,
            "post_adam_err_over_bound": float((diff[decided] / tol[decided]).max()),
            "post_adam_max_abs_err": float(diff[decided].max()),
            "decided_values": int(decided.sum()), "values": int(g.size),
            "excluded_gaussians": int(bad.sum()), "gaussians": int(scene.n),
            "excluded_pixels": int(r.unstable_px.sum())})


@pytest.mark.parametrize("tile,bwd_batch,bwd_impl", [((16, 16), 0, 1), ((8, 8), 0, 1), ((16, 32), 0, 1),
                                                     ((16, 16), 32, 1), ((16, 16), 64, 1), ((16, 16), 96, 1),
                                                     ((16, 16), 0, 0), ((8, 8), 0, 0), ((16, 32), 0, 0),
                                                     ((16, 16), 0, 2), ((8, 8), 0, 2), ((16, 32), 0, 2)])
def test_ragged_tiles_and_batches(gs, orc, tile, bwd_batch, bwd_impl):
    """Non-multiple image size (ragged tile tail), all tile shapes, fixed and
    adaptive backward batch sizes: keys bit-exact, images and gradients."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(20000, 16, 3.0, seed=7, log_scale=(-3.5, 0.5), logit_opacity=(0.0, 1.5))
    cam = synth.look_at([0, -6, 2], [0, 0, 0], 203, 149, 180.0)
    b, p, P, r = _oracle_all(orc, scene, cam, tile)
    tr = _run_forward(step_mod, scene, [cam], tile=tile, bwd_batch=bwd_batch, bwd_impl=bwd_impl)
    n = scene.n
    keys = tr.buffer(2, b.K).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys, b.keys)
    np.testing.assert_array_equal(tr.buffer(3, b.K).cpu().numpy().view(np.uint32), b.gidx)
    img = tr.image.view(149, 203, 3).cpu().numpy().astype(np.float64)
    ok = ~r.unstable_px
    assert np.abs(img - r.image)[ok].max() <= 1e-5
    rng = np.random.default_rng(3)
    dl64 = rng.normal(size=(149, 203, 3)).astype(np.float32).astype(np.float64) / (3 * 149 * 203)
    tr.dl.copy_(torch.from_numpy(dl64.astype(np.float32).reshape(-1, 3)))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    g2_orc = orc.raster_bwd64(cam, P, b, dl64, (0, 0, 0), *tile)
    count = tr.buffer(0, n).cpu().numpy().view(np.uint32)
    off = tr.buffer(1, n + 1).cpu().numpy().view(np.uint32).astype(np.int64)
    gr = gsstep.gs_gradient_records(tr.plan, tr.ws, b.K).cpu().numpy()
    g2_gpu = _sum_slots(gr, off, count)
    good = (b.count > 0) & ~_unstable_gaussians(P, r, cam)
    _check_grad(g2_gpu, g2_orc, good, f"grad2d {tile} S={bwd_batch} impl={bwd_impl}")


@pytest.mark.parametrize("tile,tpt,bg", [((16, 16), 128, None), ((16, 16), 64, None), ((8, 8), 32, None),
                                         ((16, 32), 256, None), ((16, 32), 128, None),
                                         ((16, 16), 128, (0.25, 0.5, 0.75)), ((16, 16), 64, (0.3, 0.1, 0.9))])
def test_pixels_per_thread(gs, orc, report, tile, tpt, bg):
    """The pixel-parallel raster backward with 2 or 4 pixels per thread
    (warps of 8 x 8 or 8 x 16 pixels) on a ragged image: the forward is
    unchanged (bit for bit), gradients within 1e-3 of the oracle, with and
    without a background."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(20000, 16, 3.0, seed=7, log_scale=(-3.5, 0.5), logit_opacity=(0.0, 1.5))
    cam = synth.look_at([0, -6, 2], [0, 0, 0], 203, 149, 180.0)
    bgo = bg or (0.0, 0.0, 0.0)
    b, p, P, r = _oracle_all(orc, scene, cam, tile, bg=bgo)
    ref = _run_forward(step_mod, scene, [cam], tile=tile, bg=bg)
    tr = _run_forward(step_mod, scene, [cam], tile=tile, bg=bg, tpt=tpt)
    n = scene.n
    assert torch.equal(tr.image, ref.image)
    assert torch.equal(tr.buffer(5, 149 * 203), ref.buffer(5, 149 * 203))          # n_last
    assert torch.equal(tr.buffer(6, 149 * 203, torch.float32), ref.buffer(6, 149 * 203, torch.float32))
    assert tr.stats().blended_pairs == ref.stats().blended_pairs
    img = tr.image.view(149, 203, 3).cpu().numpy().astype(np.float64)
    ok = ~r.unstable_px
    ierr = np.abs(img - r.image)[ok].max()
    assert ierr <= 1e-5
    rng = np.random.default_rng(4)
    dl64 = rng.normal(size=(149, 203, 3)).astype(np.float32).astype(np.float64) / (3 * 149 * 203)
    tr.dl.copy_(torch.from_numpy(dl64.astype(np.float32).reshape(-1, 3)))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    g2_orc = orc.raster_bwd64(cam, P, b, dl64, bgo, *tile)
    count = tr.buffer(0, n).cpu().numpy().view(np.uint32)
    off = tr.buffer(1, n + 1).cpu().numpy().view(np.uint32).astype(np.int64)
    gr = gsstep.gs_gradient_records(tr.plan, tr.ws, b.K).cpu().numpy()
    good = (b.count > 0) & ~_unstable_gaussians(P, r, cam)
    w = _check_grad(_sum_slots(gr, off, count), g2_orc, good, f"grad2d {tile} tpt={tpt} bg={bg}")
    report(f"pixels_per_thread {tile} tpt={tpt} bg={bg}", {"image_max_abs_err": float(ierr),
                                                          "grad2d_max_rel_err": float(w)})


@pytest.mark.parametrize("bwd_impl", [0, 1, 2])
def test_background_colour(gs, orc, bwd_impl):
    """Non-black background: image, and gradients (the background enters
    every dL/d alpha through the colour still to come)."""
    gsstep, step_mod = gs
    scene, _, cams = synth.tiny_workload(2)
    cam = cams[0]
    bg = (0.25, 0.5, 0.75)
    b, p, P, r = _oracle_all(orc, scene, cam, (16, 16), bg=bg)
    tr = _run_forward(step_mod, scene, cams, bg=bg, bwd_impl=bwd_impl)
    img = tr.image.view(128, 128, 3).cpu().numpy().astype(np.float64)
    ok = ~r.unstable_px
    assert np.abs(img - r.image)[ok].max() <= 1e-5
    rng = np.random.default_rng(4)
    dl64 = rng.normal(size=(128, 128, 3)).astype(np.float32).astype(np.float64) / (3 * 128 * 128)
    tr.dl.copy_(torch.from_numpy(dl64.astype(np.float32).reshape(-1, 3)))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    g2_orc = orc.raster_bwd64(cam, P, b, dl64, bg)
    n = scene.n
    count = tr.buffer(0, n).cpu().numpy().view(np.uint32)
    off = tr.buffer(1, n + 1).cpu().numpy().view(np.uint32).astype(np.int64)
    gr = gsstep.gs_gradient_records(tr.plan, tr.ws, b.K).cpu().numpy()
    good = (b.count > 0) & ~_unstable_gaussians(P, r, cam)
    _check_grad(_sum_slots(gr, off, count), g2_orc, good, f"grad2d bg impl={bwd_impl}")


def test_multi_view_uneven(gs, orc):
    """Three views of uneven resolution in one launch: per-view key segments
    bit-exact, images per view within tolerance."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(30000, 16, 4.0, seed=3, log_scale=(-3.5, 0.5))
    cams = [synth.look_at([0, -7, 2], [0, 0, 0], 160, 96, 150.0),
            synth.look_at([6, 2, 1], [0, 0, 0], 97, 131, 120.0),
            synth.look_at([-5, -5, 3], [0, 0, 0], 256, 144, 220.0)]
    tr = _run_forward(step_mod, scene, cams)
    st = tr.stats()
    bins = [orc.bin32(scene, c) for c in cams]
    K = sum(bb.K for bb in bins)
    assert st.k_required == K and st.status == 0
    keys = tr.buffer(2, K).cpu().numpy().view(np.uint32)
    pids = tr.buffer(3, K).cpu().numpy().view(np.uint32)
    o = 0
    for v, bb in enumerate(bins):
        np.testing.assert_array_equal(keys[o:o + bb.K], bb.keys)
        np.testing.assert_array_equal(pids[o:o + bb.K], bb.gidx + v * scene.n)
        o += bb.K
    p = orc.Params64.from_scene(scene)
    for c, bb, im in zip(cams, bins, tr.image_views()):
        P = orc.project64(p, c)
        r = orc.render64(c, P, bb)
        ok = ~r.unstable_px
        assert np.abs(im.cpu().numpy().astype(np.float64) - r.image)[ok].max() <= 1e-5


def test_long_tile_lists(gs, orc, report):
    """Tile lists far longer than one thread block sorts in shared memory
    (about 20,000 entries per tile on a 64x64 view): the sorted keys and
    Gaussians are the oracle's stable sort bit for bit, and the image matches
    on stable pixels."""
    gsstep, step_mod = gs
    rng = np.random.default_rng(21)
    n = 20000
    scene = synth.Scene(rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32),
                        rng.normal(size=(n, 4)).astype(np.float32),
                        np.exp(rng.normal(-1.5, 0.2, (n, 3))).astype(np.float32),
                        (1.0 / (1.0 + np.exp(-rng.normal(-3.0, 0.5, n)))).astype(np.float32),
                        rng.normal(0.0, 0.3, (n, 16, 3)).astype(np.float32))
    cam = synth.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = 64, 64, 32.0, 32.0
    b, p, P, r = _oracle_all(orc, scene, cam, (16, 16))
    lens = b.ranges[:, 1] - b.ranges[:, 0]
    assert lens.max() > 3 * 4096
    tr = _run_forward(step_mod, scene, [cam], capacity=1 << 20)
    st = tr.stats()
    assert st.status == 0 and st.k_required == b.K
    np.testing.assert_array_equal(tr.buffer(2, b.K).cpu().numpy().view(np.uint32), b.keys)
    np.testing.assert_array_equal(tr.buffer(3, b.K).cpu().numpy().view(np.uint32), b.gidx)
    rg = tr.buffer(4, 2 * 16).cpu().numpy().view(np.uint32).reshape(16, 2).astype(np.int64)
    np.testing.assert_array_equal(rg, b.ranges)
    img = tr.image.view(64, 64, 3).cpu().numpy().astype(np.float64)
    ok = ~r.unstable_px
    err = np.abs(img - r.image)[ok].max()
    assert err <= 1e-5, err
    report("long_tile_lists", {"longest_list": int(lens.max()), "shortest_list": int(lens.min()),
                               "image_max_abs_err": float(err), "keys_bit_exact": True})


def _span_tiles(sp, TX):
    """Tiles of a tile span (one or two bands) in traversal order."""
    nb, rows = (int(sp[0]) >> 24) & 3, (int(sp[0]) >> 26) & 1
    coords = [int(sp[1]) & 0xFFFF, int(sp[1]) >> 16]
    out = []
    for k in range(nb):
        lo, hi = int(sp[2 + k]) & 0xFFFF, int(sp[2 + k]) >> 16
        out += [coords[k] * TX + t if rows else t * TX + coords[k] for t in range(lo, hi + 1)]
    return out


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_tile_spans(gs, orc, report, tile):
    """The projection keeps each pair's traversal as a tile span for the
    emission: for every visible Gaussian the span gives the oracle's tiles in
    the oracle's emission order and its depth code; a Gaussian of more than
    two bands is marked and carries the binning conic, and its tiles (from
    the repeated traversal) are still placed bit-exactly: the sorted keys and
    Gaussians equal the oracle's.  A pair of at most four tiles is ranked:
    the places it took in its tiles' lists are, per tile, each of 0 .. n - 1
    once.  A quarter of the Gaussians are enlarged so that many take the
    other paths."""
    gsstep, step_mod = gs
    scene, _, cams = synth.tiny_workload(2)
    rng = np.random.default_rng(5)
    big = rng.random(scene.n) < 0.25
    scene.scales[big] *= 3.0
    cam = cams[0]
    b = orc.bin32(scene, cam, *tile)
    TX, TY = orc.tiles_of(cam, *tile)
    tiles_emit = (b.keys_emit >> np.uint32(orc.key_shift(TX * TY))).astype(np.int64)
    tr = _run_forward(step_mod, scene, [cam], tile=tile)
    st = tr.stats()
    assert st.status == 0 and st.k_required == b.K
    n = scene.n
    span = tr.buffer(10, 4 * n).cpu().numpy().view(np.uint32).reshape(n, 4)
    rank = tr.buffer(11, 4 * n).cpu().numpy().view(np.uint32).reshape(n, 4)
    ranked_cnt = tr.buffer(12, TX * TY).cpu().numpy().view(np.uint32)
    many, ranked = 0, 0
    ranks_of = [[] for _ in range(TX * TY)]
    for g in range(n):
        c = int(b.count[g])
        if c == 0:
            continue
        sp = span[g]
        assert int(sp[0]) & 0x7FFFFF == int(b.mant[g])
        want = tiles_emit[b.offset[g]:b.offset[g] + c].tolist()
        if (int(sp[0]) >> 24) & 3 == 3:
            many += 1
            np.testing.assert_array_equal(sp[1:4].view(np.float32), b.bin[g, 3:6])
            assert len({t // TX for t in want}) > 2 and len({t % TX for t in want}) > 2
        else:
            assert _span_tiles(sp, TX) == want, g
            # ranked exactly when the pair meets at most four tiles
            assert bool((int(sp[0]) >> 27) & 1) == (c <= 4), g
            if c <= 4:
                ranked += 1
                for t, rk in zip(want, rank[g][:c]):
                    ranks_of[t].append(int(rk))
    assert many >= 10 and ranked > n // 2
    # the ranks a tile handed out are 0 .. (its ranked entries - 1), each once
    for t in range(TX * TY):
        assert sorted(ranks_of[t]) == list(range(int(ranked_cnt[t]))), t
    np.testing.assert_array_equal(tr.buffer(2, b.K).cpu().numpy().view(np.uint32), b.keys)
    np.testing.assert_array_equal(tr.buffer(3, b.K).cpu().numpy().view(np.uint32), b.gidx)
    report(f"tile_spans_{tile[0]}x{tile[1]}", {"visible": int((b.count > 0).sum()), "many_band_pairs": many,
                                                "ranked_pairs": ranked, "keys": int(b.K), "keys_bit_exact": True})


@pytest.mark.parametrize("n", [300, 2500, 6000])
def test_tile_lists_of_every_size_class(gs, orc, report, n):
    """Tile lists in every size class of the per-tile sort -- tiny (<= 254
    entries, four lists per block, one per warp), short (255-1022), medium
    (1023-2046, two lists per block, one per half), long (>= 2047, in shared
    memory up to 4096, chunked beyond) -- on a 64x64 view: the sorted keys
    and Gaussians equal the oracle's stable sort bit for bit."""
    gsstep, step_mod = gs
    rng = np.random.default_rng(30 + n)
    scene = synth.Scene(rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32),
                        rng.normal(size=(n, 4)).astype(np.float32),
                        np.exp(rng.normal(-2.2, 0.5, (n, 3))).astype(np.float32),
                        (1.0 / (1.0 + np.exp(-rng.normal(-2.0, 1.0, n)))).astype(np.float32),
                        rng.normal(0.0, 0.3, (n, 16, 3)).astype(np.float32))
    cam = synth.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = 64, 64, 32.0, 32.0
    b = orc.bin32(scene, cam)
    lens = b.ranges[:, 1] - b.ranges[:, 0]
    tr = _run_forward(step_mod, scene, [cam], capacity=1 << 20)
    st = tr.stats()
    assert st.status == 0 and st.k_required == b.K
    np.testing.assert_array_equal(tr.buffer(2, b.K).cpu().numpy().view(np.uint32), b.keys)
    np.testing.assert_array_equal(tr.buffer(3, b.K).cpu().numpy().view(np.uint32), b.gidx)
    classes = {"tiny": int((lens <= 254).sum()), "short": int(((lens >= 255) & (lens <= 1022)).sum()),
               "medium": int(((lens >= 1023) & (lens <= 2046)).sum()), "long": int((lens >= 2047).sum())}
    report(f"tile_lists_size_classes_n{n}", {**classes, "keys": int(b.K), "keys_bit_exact": True})
    # the inputs reach the classes they are meant for (all four over the three
    # cases, and lists beyond 4096 entries for the chunked path)
    want = {300: ("tiny", "short"), 2500: ("tiny", "short", "long"), 6000: ("short", "medium", "long")}[n]
    assert all(classes[c] > 0 for c in want), classes
    if n == 6000:
        assert lens.max() > 4096


def test_capacity_overflow_sets_status(gs, orc):
    """Too small an intersection capacity is reported, nothing is written
    out of bounds, and a larger capacity then succeeds."""
    gsstep, step_mod = gs
    scene, _, cams = synth.tiny_workload(0)
    tr = _run_forward(step_mod, scene, cams, capacity=2048)
    st = tr.stats()
    assert st.status & gsstep.STATUS_CAPACITY
    assert st.k_required == orc.bin32(scene, cams[0]).K
    tr2 = _run_forward(step_mod, scene, cams, capacity=int(st.k_required))
    assert tr2.stats().status == 0


def test_nonfinite_parameter_sets_status(gs):
    gsstep, step_mod = gs
    scene, _, cams = synth.tiny_workload(0)
    scene.means[5, 1] = np.nan
    tr = _run_forward(step_mod, scene, cams)
    assert tr.stats().status & gsstep.STATUS_NONFINITE


def test_graph_replay_equals_eager(gs):
    """A captured step replays bit-identically to the eager step (two steps)."""
    gsstep, step_mod = gs
    scene, tscene, cams = synth.tiny_workload(0)
    target = np.random.default_rng(0).uniform(0, 0.5, size=(128, 128, 3)).astype(np.float32)
    a = step_mod.Trainer([scene], cams, lr=LR)
    b = step_mod.Trainer([scene], cams, lr=LR)
    for t in (a, b):
        t.set_target([target])
    b.capture()
    b.scenes[0].geom.copy_(a.scenes[0].geom)  # capture ran no kernels
    for _ in range(2):
        a.step(0)
        b.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.scenes[0].geom, b.scenes[0].geom)
    assert torch.equal(a.scenes[0].sh, b.scenes[0].sh)
    assert torch.equal(a.scenes[0].m, b.scenes[0].m)
    assert a.stats().step == b.stats().step == 2


def _bf16_round(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def _bf16_ulp(x):
    """Spacing of bf16 numbers at |x| (8 significant bits)."""
    ax = np.maximum(np.abs(x), np.finfo(np.float32).tiny)
    return 2.0 ** (np.floor(np.log2(ax)) - 7)


def test_bf16_storage_step(gs, orc, report):
    """SH and both Adam moments stored in BF16 (FP32 arithmetic): image and
    post-Adam geometry as in FP32; post-Adam SH and moments within one BF16
    ulp (stochastic rounding) of the FP64 oracle fed the same stored SH."""
    gsstep, step_mod = gs
    scene, tscene, cams = synth.tiny_workload(0)
    cam = cams[0]
    scene.sh = _bf16_round(scene.sh)            # what BF16 storage holds
    tgt = orc.render64(cam, orc.project64(orc.Params64.from_scene(tscene), cam), orc.bin32(tscene, cam)).image
    res = orc.step(scene, cams, [tgt], LR, 1)
    tr = step_mod.Trainer([scene], cams, lr=LR, sh_bf16=True, mom_bf16=True)
    assert tr.scenes[0].sh.dtype == torch.bfloat16 and tr.scenes[0].m.dtype == torch.bfloat16
    tr.set_target([tgt.astype(np.float32)])
    tr.forward()
    torch.cuda.synchronize()
    r = res.renders[0]
    img = tr.image.view(128, 128, 3).cpu().numpy().astype(np.float64)
    assert np.abs(img - r.image)[~r.unstable_px].max() <= 1e-5
    tr.backward_adam(step=1)
    torch.cuda.synchronize()
    assert tr.stats().status == 0
    undecided = (np.abs(r.image - tgt) < 1e-5).any(-1)
    r.unstable_px |= undecided
    bad = _unstable_gaussians(res.projs[0], r, cam)
    g = res.grad
    rms = np.sqrt((g[~bad] ** 2).mean(0)) + 1e-30
    decided = (np.abs(g) > 1e-2 * rms[None, :]) & ~bad[:, None]
    new = tr.scenes[0].to_scene()
    n = scene.n
    # SH parameters: one bf16 ulp of the FP64 result (plus FP32 slack)
    sh_gpu = new.sh.reshape(n, 48).astype(np.float64)
    sh_orc = res.theta[:, 11:]
    tol = _bf16_ulp(sh_orc) + 1e-6
    d = decided[:, 11:]
    assert np.all(np.abs(sh_gpu - sh_orc)[d] <= tol[d])
    sh_ulps = float((np.abs(sh_gpu - sh_orc)[d] / _bf16_ulp(sh_orc)[d]).max())
    # geometry stays FP32
    geo_gpu = np.concatenate([new.means, new.quats, np.log(new.scales)], axis=1).astype(np.float64)
    dg = decided[:, :10]
    assert np.all(np.abs(geo_gpu - res.theta[:, :10])[dg] <= (1e-5 * np.abs(res.theta[:, :10]) + 1e-6)[dg])
    # moments (15 chunks x 4, bf16) against the oracle's m, v in theta order
    def unpack(t):
        a = t.float().cpu().numpy()
        return np.concatenate([a[0, :, :3], a[1], a[2], a[3:].transpose(1, 0, 2).reshape(n, 48)], axis=1)
    for name, gpu_t, orc_a in (("m", tr.scenes[0].m, res.m), ("v", tr.scenes[0].v, res.v)):
        mg = unpack(gpu_t).astype(np.float64)
        ok = decided & (orc_a != 0)
        # one bf16 ulp of rounding plus the FP32 gradient's own 1e-3 (x2 for v)
        bound = _bf16_ulp(orc_a) + 2e-3 * np.abs(orc_a)
        assert np.all(np.abs(mg - orc_a)[ok] <= bound[ok]), name
    report("config0_bf16_storage_step",
           {"image_max_abs_err": float(np.abs(img - r.image)[~r.unstable_px].max()),
            "sh_max_err_bf16_ulps": sh_ulps,
            "geometry_max_abs_err": float(np.abs(geo_gpu - res.theta[:, :10])[dg].max()),
            "decided_values": int(decided.sum()), "excluded_gaussians": int(bad.sum())})


@pytest.mark.parametrize("bf16", [False, True])
def test_multi_view_full_step_adam(gs, orc, bf16):
    """Four views of one scene in one step (loss over all views, one Adam
    update; the fused kernel then spreads each Gaussian over four lanes):
    post-Adam parameters against the oracle's multi-view step."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(8000, 8, 2.5, seed=4, log_scale=(-3.4, 0.4), logit_opacity=(0.0, 1.0))
    if bf16:
        scene.sh = _bf16_round(scene.sh)
    cams = synth.orbit_cameras(4, 5.0, 96, 72, hfov_deg=55.0)
    tscene = synth.perturbed(scene, 9)
    targets = []
    for c in cams:
        targets.append(orc.render64(c, orc.project64(orc.Params64.from_scene(tscene), c), orc.bin32(tscene, c)).image)
    res = orc.step(scene, cams, targets, LR, 1)
    tr = step_mod.Trainer([scene], cams, lr=LR, sh_bf16=bf16, mom_bf16=bf16)
    tr.set_target([t.astype(np.float32) for t in targets])
    tr.step(step=1)
    torch.cuda.synchronize()
    assert tr.stats().status == 0
    bad = np.zeros(scene.n, bool)
    for c, r, P, tg in zip(cams, res.renders, res.projs, targets):
        r.unstable_px |= (np.abs(r.image - tg) < 1e-5).any(-1)
        bad |= _unstable_gaussians(P, r, c)
    g = res.grad
    rms = np.sqrt((g[~bad] ** 2).mean(0)) + 1e-30
    decided = (np.abs(g) > 1e-2 * rms[None, :]) & ~bad[:, None]
    assert decided.sum() > 0.3 * g.size
    new = tr.scenes[0].to_scene()
    th = np.concatenate([new.means, new.quats, np.log(new.scales), np.log(new.opacities / (1 - new.opacities))[:, None],
                         new.sh.reshape(-1, 48)], axis=1).astype(np.float64)
    tol = 1e-5 * np.abs(res.theta) + 1e-6
    if bf16:
        tol[:, 11:] += _bf16_ulp(res.theta[:, 11:])
    assert np.all(np.abs(th - res.theta)[decided] <= tol[decided])
