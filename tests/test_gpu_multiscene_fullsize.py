"""The multi-scene workload at full size through the autograd interface:
eight scenes (0.5 to 6M Gaussians, 12M in all), two views each of mixed
resolution (16 views in one launch per stage), BF16 SH.

- sorted keys and Gaussians of every view bit-exact against the oracle's FP32
  binning;
- images on a sample of tiles of every view against the FP64 oracle;
- the smallest scene's gradients with respect to its stored parameters
  against the oracle's full analytic backward;
- the largest scene's per-intersection gradients on sampled tiles."""
import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu

TILE_STRIDE = 97
MARGIN = 1e-3      # threshold-flag margin at 1-2 MP (see test_gpu_fullsize)


@pytest.fixture(scope="module")
def ms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import autograd, gsstep, step
    scenes, cams = synth.multi_scene_workload()
    for sc in scenes:       # what BF16 storage holds
        sc.sh = torch.from_numpy(np.ascontiguousarray(sc.sh, np.float32)).to(torch.bfloat16).float().numpy()
    R = autograd.Renderer([s.n for s in scenes], cams, sh_bf16=True)
    params = []
    for sc in scenes:
        b = step.SceneBuffers.from_scene(sc, sh_bf16=True, moments=False)
        params += [b.geom.requires_grad_(True), b.sh.requires_grad_(True)]
    img = R.render([(params[2 * k], params[2 * k + 1]) for k in range(len(scenes))])
    total_px = sum(c.width * c.height for c in cams)
    rng = np.random.default_rng(0)
    weights = [(rng.normal(size=(c.height, c.width, 3)) / total_px).astype(np.float32) for c in cams]
    wt = torch.from_numpy(np.concatenate([w.reshape(-1, 3) for w in weights])).cuda()
    (img * wt).sum().backward()
    torch.cuda.synchronize()
    return dict(gsstep=gsstep, R=R, scenes=scenes, cams=cams, params=params, img=img.detach(), weights=weights)


@pytest.fixture(scope="module")
def bins(ms, orc):
    return [orc.bin32(ms["scenes"][c.scene], c) for c in ms["cams"]]


def _segments(ms, bins):
    """Per view: (first sorted entry, pair base) in the plan's order."""
    out, seg, base = [], 0, 0
    for c, b in zip(ms["cams"], bins):
        out.append((seg, base))
        seg += b.K
        base += ms["scenes"][c.scene].n
    return out


def test_keys_every_view(ms, bins):
    gsstep, R = ms["gsstep"], ms["R"]
    st = gsstep.gs_read_stats(R.plan, R.ws)
    K = sum(b.K for b in bins)
    assert st.status == 0 and st.k_required == K
    keys = gsstep.gs_workspace_buffer(R.plan, R.ws, 2, K).cpu().numpy().view(np.uint32)
    pids = gsstep.gs_workspace_buffer(R.plan, R.ws, 3, K).cpu().numpy().view(np.uint32)
    for (seg, base), b in zip(_segments(ms, bins), bins):
        np.testing.assert_array_equal(keys[seg:seg + b.K], b.keys)
        np.testing.assert_array_equal(pids[seg:seg + b.K].astype(np.int64), b.gidx.astype(np.int64) + base)


def _sampled(orc, b):
    keep = np.zeros(b.ranges.shape[0], bool)
    keep[::TILE_STRIDE] = True
    bs = orc.Binning(b.count, b.bin, b.mant, b.offset, b.keys_emit, b.gidx_emit, b.keys, b.gidx, b.perm,
                     np.where(keep[:, None], b.ranges, 0))
    return keep, bs


def _tile_of_pixel(cam):
    TX = (cam.width + 15) // 16
    return (np.arange(cam.height)[:, None] // 16) * TX + (np.arange(cam.width)[None, :] // 16)


def test_images_sampled_tiles_every_view(ms, bins, orc, report):
    views = ms["R"].views(ms["img"])
    worst, excluded, sampled_total = 0.0, 0, 0
    params64 = {}
    for c, b, im in zip(ms["cams"], bins, views):
        if c.scene not in params64:
            params64 = {c.scene: orc.Params64.from_scene(ms["scenes"][c.scene])}
        P = orc.project64(params64[c.scene], c)
        keep, bs = _sampled(orc, b)
        r = orc.render64(c, P, bs, margin=MARGIN)
        sampled = keep[_tile_of_pixel(c)]
        ok = sampled & ~r.unstable_px
        assert ok.sum() > 0.9 * sampled.sum()
        got = im.cpu().numpy().astype(np.float64)
        assert np.abs(got - r.image)[ok].max() <= 1e-5, (c.scene, c.width)
        worst = max(worst, float(np.abs(got - r.image)[ok].max()))
        excluded += int(sampled.sum() - ok.sum())
        sampled_total += int(sampled.sum())
    report("config4_images_sampled_tiles", {"views": len(views), "image_max_abs_err": worst,
                                            "sampled_pixels": sampled_total, "excluded_pixels": excluded})


def _bad_gaussians(r, P, b, cam, mask=None):
    """Gaussians the oracle flags, and every listed Gaussian reaching
    (d^2 <= 9) a flagged pixel -- looked up through the pixel's tile list."""
    bad = r.unstable_g.copy()
    px = r.unstable_px if mask is None else (r.unstable_px & mask)
    ys, xs = np.nonzero(px)
    tiles = (ys // 16) * ((cam.width + 15) // 16) + xs // 16
    for t in np.unique(tiles):
        sel = tiles == t
        s0, e0 = b.ranges[t]
        g = b.gidx[s0:e0].astype(np.int64)
        dx = xs[sel][:, None] + 0.5 - P[g, 4][None, :]
        dy = ys[sel][:, None] + 0.5 - P[g, 5][None, :]
        d2 = P[g, 9] * dx * dx + 2 * P[g, 10] * dx * dy + P[g, 11] * dy * dy
        bad[g[(d2 <= 9.0 * 1.001).any(0)]] = True
    return bad


def test_smallest_scene_gradients_full_backward(ms, bins, orc, report):
    """Scene 0 (500k Gaussians; 1920x1080 and 960x540 views): FP32 gradients
    with respect to the stored parameters against the oracle's analytic
    backward over all its tiles."""
    sc = ms["scenes"][0]
    p = orc.Params64.from_scene(sc)
    g = np.zeros((sc.n, 59))
    bad = np.zeros(sc.n, bool)
    for c, b, w in zip(ms["cams"], bins, ms["weights"]):
        if c.scene != 0:
            continue
        P = orc.project64(p, c)
        r = orc.render64(c, P, b, margin=MARGIN)
        g2 = orc.raster_bwd64(c, P, b, w.astype(np.float64))
        orc.project_bwd64(p, c, P, g2, out=g)
        bad |= _bad_gaussians(r, P, b, c)
    ref = np.concatenate([g[:, 0:3], g[:, 3:7], g[:, 7:10] / p.scales,
                          (g[:, 10] / (p.opacities * (1 - p.opacities)))[:, None], g[:, 11:]], axis=1)
    n = sc.n
    go = _fp32_grads(ms)[:, :n].cpu().numpy()      # scene 0 comes first
    gpu = np.concatenate([go[0, :, :3], go[1], go[2], go[3:15].transpose(1, 0, 2).reshape(n, 48)], axis=1)
    good = ~bad & (np.abs(ref).sum(1) > 0)
    # at 1-2 MP the flags (margin 1e-3 at every threshold) exclude most
    # Gaussians that reach a flagged pixel anywhere in either view
    assert good.sum() > 0.15 * (np.abs(ref).sum(1) > 0).sum() and good.sum() > 20000
    r_, g_ = ref[good], gpu[good]
    rms = np.sqrt((r_ ** 2).mean(0)) + 1e-30
    scale = np.maximum(np.abs(r_), rms[None, :])
    err = np.abs(g_ - r_) / scale
    assert err.max() <= 1e-3, (err[:, :11].max(), err[:, 11:].max())
    report("config4_scene0_full_backward", {"grad_geometry_max_rel_err": float(err[:, :11].max()),
                                            "grad_sh_max_rel_err": float(err[:, 11:].max()),
                                            "gaussians_with_gradient": int((np.abs(ref).sum(1) > 0).sum()),
                                            "excluded_gaussians": int((np.abs(ref).sum(1) > 0).sum() - good.sum())})


def test_largest_scene_records_sampled_tiles(ms, bins, orc, report):
    """Scene 7 (6M Gaussians; 1280x720 and 1600x900): per-Gaussian sums of
    the intersection gradient records in sampled tiles."""
    gsstep, R = ms["gsstep"], ms["R"]
    K = sum(b.K for b in bins)
    gr = gsstep.gs_gradient_records(R.plan, R.ws, K).cpu().numpy()
    slots = gsstep.gs_workspace_buffer(R.plan, R.ws, 9, K).cpu().numpy().view(np.uint32).astype(np.int64)
    sc = ms["scenes"][7]
    p = orc.Params64.from_scene(sc)
    checked = 0
    for (seg, base), c, b, w in zip(_segments(ms, bins), ms["cams"], bins, ms["weights"]):
        if c.scene != 7:
            continue
        P = orc.project64(p, c)
        keep, bs = _sampled(orc, b)
        r = orc.render64(c, P, bs, margin=MARGIN)
        g2_orc = orc.raster_bwd64(c, P, bs, w.astype(np.float64))
        in_sample = keep[b.keys >> orc.key_shift(b.ranges.shape[0])]
        g2_gpu = np.zeros_like(g2_orc)
        np.add.at(g2_gpu, b.gidx[in_sample].astype(np.int64), gr[slots[seg:seg + b.K][in_sample]].astype(np.float64))
        touched = np.zeros(sc.n, bool)
        touched[b.gidx[in_sample]] = True
        good = touched & ~_bad_gaussians(r, P, b, c, keep[_tile_of_pixel(c)])
        assert good.sum() > 0.15 * touched.sum() and good.sum() > 5000
        ref, got = g2_orc[good], g2_gpu[good]
        rms = np.sqrt((ref ** 2).mean(0)) + 1e-30
        err = np.abs(got - ref) / np.maximum(np.abs(ref), rms[None, :])
        assert err.max() <= 1e-3, err.max()
        report(f"config4_scene7_view{checked}_records", {"grad2d_max_rel_err": float(err.max()),
                                                          "gaussians_touched": int(touched.sum()),
                                                          "excluded_gaussians": int(touched.sum() - good.sum())})
        checked += 1
    assert checked == 2


def test_thousand_training_steps_bf16(ms):
    """1,000 graph-replayed training steps of the eight-scene batch with BF16
    storage (fused Adam): the status stays clear, the loss falls, parameters
    stay finite."""
    from paper_2605_00219_gb300 import step as step_mod
    scenes, cams = ms["scenes"], ms["cams"]
    tr = step_mod.Trainer(scenes, cams, sh_bf16=True, mom_bf16=True)
    g = torch.Generator(device="cuda").manual_seed(4)
    tr.target.copy_(torch.rand(tr.target.shape, device="cuda", generator=g) * 0.5)
    tr.step(0)
    first = float(tr.stats().loss)
    tr.capture()
    for _ in range(999):
        tr.replay()
    torch.cuda.synchronize()
    st = tr.stats()
    assert st.status == 0 and st.step == 1000
    tr.forward()
    gsstep = ms["gsstep"]
    gsstep.gs_loss_l1(tr.plan, tr.ws, tr.image, tr.target, tr.dl)
    torch.cuda.synchronize()
    assert float(tr.stats().loss) < 0.7 * first
    for sb in tr.scenes:
        assert bool(torch.isfinite(sb.geom).all()) and bool(torch.isfinite(sb.sh.float()).all())


def _fp32_grads(ms):
    """Gradients of the last render with respect to every scene's stored
    parameters in FP32, from gs_project_bwd_adam in gradient mode (the
    autograd interface returns the SH part in the parameters' bf16 dtype)."""
    import types
    gsstep, R = ms["gsstep"], ms["R"]
    N = sum(sc.n for sc in ms["scenes"])
    go = torch.empty((15, N, 4), dtype=torch.float32, device="cuda")
    bufs = [types.SimpleNamespace(n=sc.n, geom=ms["params"][2 * k], sh=ms["params"][2 * k + 1], m=None, v=None)
            for k, sc in enumerate(ms["scenes"])]
    gsstep.gs_project_bwd_adam(R.plan, R.ws, bufs, R.cams, None, go)
    torch.cuda.synchronize()
    return go


def test_finite_differences_sampled_gaussians(ms, bins, orc, report):
    """Central differences of the FP64 oracle (outer step h = 1e-3 in theta,
    fourth-order stencil) on 64 sampled Gaussians of every scene, 11
    parameters each (every group), against the FP32 gradients of the
    autograd backward: relative error <= 1e-3 with an absolute floor of 1e-3 x
    the RMS of the component over the scene's listed Gaussians, on every evaluation
    that is kept.  Evaluations where a discrete decision of the forward
    changes within +-h are skipped and counted.  The bf16 SH gradients the
    autograd interface returns are the FP32 ones rounded to bf16."""
    import fdcheck
    go = _fp32_grads(ms)
    base = 0
    totals = {"checked": 0, "skipped": 0, "max_err": 0.0}
    per_scene = []
    for si, sc in enumerate(ms["scenes"]):
        n = sc.n
        gsh = go[3:15, base:base + n]
        bf = gsh.reshape(6, 2, n, 4).permute(0, 2, 1, 3).reshape(6, n, 8).to(torch.bfloat16)
        assert torch.equal(bf, ms["params"][2 * si + 1].grad)
        g = go[:, base:base + n].cpu().numpy()
        base += n
        dstored = np.concatenate([g[0, :, :3], g[1], g[2], g[3:15].transpose(1, 0, 2).reshape(n, 48)], axis=1)
        p = orc.Params64.from_scene(sc)
        gth = fdcheck.theta_grads(p, dstored)
        views = [(c, b, orc.project64(p, c), w.astype(np.float64))
                 for c, b, w in zip(ms["cams"], bins, ms["weights"]) if c.scene == si]
        listed = np.zeros(n, bool)
        for _, b, _, _ in views:
            listed |= b.count > 0
        rms = np.sqrt((gth[listed] ** 2).mean(0)) + 1e-30
        picks = np.random.default_rng(100 + si).choice(np.nonzero(listed)[0], size=64, replace=False)
        res = fdcheck.fd_check(orc, sc, views, picks, gth, rms)
        per_scene.append({"scene": si, "n": n, **res})
        totals["checked"] += res["checked"]
        totals["skipped"] += res["skipped"]
        totals["max_err"] = max(totals["max_err"], res["max_err"])
    report("multiscene_fd", {"per_scene": per_scene, **totals})
    for r in per_scene:
        assert r["checked"] >= 300, r
        assert r["max_err"] <= 1e-3, r
