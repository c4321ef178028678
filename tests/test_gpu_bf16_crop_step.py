"""BF16 storage at full size: 3M Gaussians, one 1920x1080 view, SH and both
Adam moments in BF16 (FP32 arithmetic).

- One step with the L1 loss restricted to a 64x64 tile-aligned crop, against
  the FP64 oracle: the image on the crop, the gradients and the post-Adam
  parameters of every Gaussian listed in the crop's tiles.
- The rendered PSNR of BF16 against FP32 storage after 2000 steps of the
  same schedule: |delta| < 0.05 dB on the training view and a held-out view."""
import math

import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu

MARGIN = 1e-3                       # threshold-flag margin at 1080p
LR = (1.6e-4 * 30.0, 1e-3, 5e-3, 5e-2, 2.5e-3, 2.5e-3 / 20)
X0, Y0, CW = 960, 512, 64           # crop: pixels [X0, X0+64) x [Y0, Y0+64), 4x4 tiles of 16


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep, step
    return gsstep, step


def _bf16_round(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def _bf16_ulp(x):
    ax = np.maximum(np.abs(x), np.finfo(np.float32).tiny)
    return 2.0 ** (np.floor(np.log2(ax)) - 7)


def _crop_binning(orc, b):
    TX = b.ranges.shape[0] // 68
    keep = np.zeros(b.ranges.shape[0], bool)
    for ty in range(Y0 // 16, (Y0 + CW) // 16):
        keep[ty * TX + X0 // 16: ty * TX + (X0 + CW) // 16] = True
    bs = orc.Binning(b.count, b.bin, b.mant, b.offset, b.keys_emit, b.gidx_emit, b.keys, b.gidx, b.perm,
                     np.where(keep[:, None], b.ranges, 0))
    return keep, bs


def test_crop_step_against_oracle(mods, orc, report):
    gsstep, step_mod = mods
    scene = synth.large_scene(0)
    scene.sh = _bf16_round(scene.sh)               # what BF16 storage holds
    tscene = synth.perturbed(scene, 1)
    cam = synth.large_views(1, resolutions=[(1920, 1080)])[0]
    # oracle: target on the crop, then the crop-restricted step
    tb = orc.bin32(tscene, cam)
    _, tbs = _crop_binning(orc, tb)
    tgt = orc.render64(cam, orc.project64(orc.Params64.from_scene(tscene), cam), tbs).image
    b = orc.bin32(scene, cam)
    keep, bs = _crop_binning(orc, b)
    p = orc.Params64.from_scene(scene)
    P = orc.project64(p, cam)
    r = orc.render64(cam, P, bs, margin=MARGIN)
    crop = np.zeros((1080, 1920), bool)
    crop[Y0:Y0 + CW, X0:X0 + CW] = True
    dl64 = np.where(crop[..., None], np.sign(r.image - tgt) / (3.0 * CW * CW), 0.0)
    g2 = orc.raster_bwd64(cam, P, bs, dl64)
    grad = orc.project_bwd64(p, cam, P, g2)
    theta = p.theta()
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    orc.adam64(theta, m, v, grad, LR, 1)

    # device: forward, L1 on the crop only, raster backward, fused Adam (t = 1)
    tr = step_mod.Trainer([scene], [cam], lr=LR, sh_bf16=True, mom_bf16=True)
    tr.set_target([tgt.astype(np.float32)])
    tr.forward()
    gsstep.gs_loss_l1(tr.plan, tr.ws, tr.image, tr.target, tr.dl)
    mask = torch.from_numpy(crop.reshape(-1, 1).astype(np.float32)).cuda()
    tr.dl.mul_(mask * float(1920 * 1080) / float(CW * CW))
    gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
    go = torch.empty((15, scene.n, 4), dtype=torch.float32, device="cuda")
    gsstep.gs_project_bwd_adam(tr.plan, tr.ws, tr.scenes, tr.cams, None, go)     # gradient only
    gsstep.gs_project_bwd_adam(tr.plan, tr.ws, tr.scenes, tr.cams, gsstep.make_adam(LR, step=1))
    torch.cuda.synchronize()
    assert tr.stats().status == 0

    img = tr.image.view(1080, 1920, 3).cpu().numpy().astype(np.float64)
    undecided = (np.abs(r.image - tgt) < 1e-5).any(-1) & crop
    stable = crop & ~r.unstable_px
    assert np.abs(img - r.image)[stable].max() <= 1e-5
    r.unstable_px |= undecided
    # Gaussians listed in the crop's tiles; exclude those reaching a flagged pixel
    shift = orc.key_shift(b.ranges.shape[0])
    listed = np.zeros(scene.n, bool)
    listed[b.gidx[keep[b.keys >> shift]]] = True
    bad = r.unstable_g.copy()
    ys, xs = np.nonzero(r.unstable_px & crop)
    for x, y in zip(xs, ys):
        t = (y // 16) * 120 + x // 16
        s0, e0 = b.ranges[t]
        g = b.gidx[s0:e0].astype(np.int64)
        dx, dy = x + 0.5 - P[g, 4], y + 0.5 - P[g, 5]
        d2 = P[g, 9] * dx * dx + 2 * P[g, 10] * dx * dy + P[g, 11] * dy * dy
        bad[g[d2 <= 9.0 * 1.001]] = True
    sel = listed & ~bad
    assert sel.sum() > 0.5 * listed.sum() and sel.sum() > 200
    # gradients with respect to the stored parameters (scales and opacity
    # activated), relative 1e-3 with an absolute floor of 1e-3 x the RMS
    gg = go.cpu().numpy()
    gpu_g = np.concatenate([gg[0, :, :3], gg[1], gg[2], gg[3:15].transpose(1, 0, 2).reshape(-1, 48)], axis=1)[sel]
    ref_g = np.concatenate([grad[:, 0:3], grad[:, 3:7], grad[:, 7:10] / p.scales,
                            (grad[:, 10] / (p.opacities * (1 - p.opacities)))[:, None], grad[:, 11:]], axis=1)[sel]
    grms = np.sqrt((ref_g ** 2).mean(0)) + 1e-30
    gerr = np.abs(gpu_g - ref_g) / np.maximum(np.abs(ref_g), grms[None, :])
    assert gerr.max() <= 1e-3, gerr.max()
    rms = np.sqrt((grad[sel] ** 2).mean(0)) + 1e-30
    decided = (np.abs(grad[sel]) > 1e-2 * rms[None, :])
    new = tr.scenes[0].to_scene()
    th = np.concatenate([new.means, new.quats, np.log(new.scales), np.log(new.opacities / (1 - new.opacities))[:, None],
                         new.sh.reshape(-1, 48)], axis=1).astype(np.float64)[sel]
    ref = theta[sel]
    tol = 1e-5 * np.abs(ref) + 1e-6
    tol[:, 11:] += _bf16_ulp(ref[:, 11:])
    assert decided.sum() > 0.3 * decided.size
    assert np.all(np.abs(th - ref)[decided] <= tol[decided]), np.abs(th - ref)[decided].max()
    sh_ulps = (np.abs(th - ref)[:, 11:] / _bf16_ulp(ref[:, 11:]))[decided[:, 11:]]
    report("config3_bf16_1080p_crop_step",
           {"image_max_abs_err": float(np.abs(img - r.image)[stable].max()), "crop_pixels": int(crop.sum()),
            "excluded_pixels": int((crop & ~stable).sum()), "grad3d_max_rel_err": float(gerr.max()),
            "post_adam_geometry_err_over_bound": float((np.abs(th - ref)[:, :11] / tol[:, :11])[decided[:, :11]].max()),
            "post_adam_sh_max_err_bf16_ulps": float(sh_ulps.max()),
            "listed_gaussians": int(listed.sum()), "excluded_gaussians": int(listed.sum() - sel.sum()),
            "decided_values": int(decided.sum())})
    # Gaussians with no listed intersection in the crop keep their parameters
    far = ~listed
    sh_before = scene.sh.reshape(-1, 48)[far][:1000]
    assert np.array_equal(new.sh.reshape(-1, 48)[far][:1000], sh_before)
    assert np.array_equal(new.means[far][:1000], scene.means[far][:1000])


def _psnr(img, ref):
    mse = float(((img.double() - ref.double()) ** 2).mean().item())
    return 10.0 * math.log10(1.0 / max(mse, 1e-30))


def test_bf16_psnr_after_2000_steps(mods, report):
    """2,000 steps on one 1080p view, FP32 storage against BF16 SH and
    moments, from the same seed.  Quality is PSNR on held-out views (the
    paper evaluates PSNR on test views): |mean difference| < 0.05 dB over three
    held-out views.  The training view is fitted to about 54 dB, where a
    last-ulp change in one rounding moves the FP32 run by ~0.01-0.02 dB, so
    there BF16 must only not fit worse than FP32 by 0.05 dB."""
    gsstep, step_mod = mods
    scene = synth.large_scene(0)
    tscene = synth.perturbed(scene, 1)
    cam = synth.large_views(1, resolutions=[(1920, 1080)])[0]
    held = [synth.large_views(1, resolutions=[(1920, 1080)], phase_deg=d)[0] for d in (45.0, 135.0, -90.0)]

    def render(sc_or_bufs, c, bf16=False):
        t = step_mod.Trainer([sc_or_bufs], [c], lr=LR, sh_bf16=bf16, mom_bf16=bf16)
        t.forward()
        torch.cuda.synchronize()
        return t.image.clone()

    tgt = render(tscene, cam)
    held_tgt = [render(tscene, h) for h in held]
    out = {}
    for bf16 in (False, True):
        tr = step_mod.Trainer([scene], [cam], lr=LR, sh_bf16=bf16, mom_bf16=bf16)
        tr.target.copy_(tgt)
        tr.step(0)
        tr.capture()
        for _ in range(1999):
            tr.replay()
        torch.cuda.synchronize()
        assert tr.stats().status == 0 and tr.stats().step == 2000
        tr.forward()
        torch.cuda.synchronize()
        out[bf16] = (_psnr(tr.image, tgt), [_psnr(render(tr.scenes[0], h, bf16), t) for h, t in zip(held, held_tgt)])
    print("PSNR after 2000 steps (train, held-out): FP32", out[False], "BF16", out[True])
    d_train = out[True][0] - out[False][0]
    d_held = float(np.mean(out[True][1]) - np.mean(out[False][1]))
    report("config3_psnr_2000_steps", {"fp32_train_db": out[False][0], "bf16_train_db": out[True][0],
                                       "fp32_heldout_db": out[False][1], "bf16_heldout_db": out[True][1],
                                       "heldout_mean_delta_db": d_held, "train_delta_db": d_train})
    assert abs(d_held) < 0.05
    assert d_train > -0.05
    assert out[False][0] > _psnr(render(scene, cam), tgt) + 1.0      # training improved the fit
