"""Parity of the fused L1 + SSIM loss kernel (Sec. 4.5, 8-bit RGBA reference)
with the FP64 oracle, through the C ABI.

Tolerances: loss within 1e-5 relative; every pixel's gradient within 1e-3
relative, with an absolute floor of 1e-3 x the RMS of the view's gradient
(the gradient tolerance of the step), pixels whose L1 sign is within 1e-6 of
a tie excluded; lambda = 0 reproduces gs_loss_l1's gradient bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu

# ragged sizes: several 16x16 tiles with partial ones, a view lower than the
# 11-tap window, a single pixel
SHAPES = [(300, 170), (37, 29), (100, 7), (1, 1), (64, 48)]


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep, step
    return gsstep, step


def _plan(gsstep, shapes):
    plan = gsstep.Plan([16], [(w, h, 0) for (w, h) in shapes])
    ws = torch.empty(plan.workspace_bytes(), dtype=torch.uint8, device="cuda")
    gsstep.gs_workspace_init(plan, ws)
    return plan, ws


def _flat(imgs, cols):
    return torch.cat([torch.from_numpy(np.ascontiguousarray(a)).reshape(-1, cols) for a in imgs]).cuda()


def _split(flat, shapes):
    out, o = [], 0
    for (w, h) in shapes:
        out.append(flat[o:o + w * h].reshape(h, w, -1))
        o += w * h
    return out


def _grad_err(got, ref, tie):
    """Per-element error |got - ref| / max(|ref|, RMS of ref), ties excluded."""
    rms = np.sqrt((ref ** 2).mean()) + 1e-30
    return np.where(tie, 0.0, np.abs(got - ref) / np.maximum(np.abs(ref), rms))


def _run(gsstep, plan, ws, img_d, tgt_d, lam):
    dl = torch.full_like(img_d, np.nan)
    gsstep.gs_loss_l1_ssim(plan, ws, img_d, tgt_d, lam, dl)
    torch.cuda.synchronize()
    return gsstep.gs_read_stats(plan, ws).loss, dl.cpu().numpy()


@pytest.mark.parametrize("smooth", [False, True])
@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_l1_ssim_matches_oracle(gs, orc, report, smooth, lam):
    gsstep, _ = gs
    imgs, tgts = synth.loss_images(SHAPES, seed=11 + int(smooth), smooth=smooth)
    plan, ws = _plan(gsstep, SHAPES)
    loss, dl = _run(gsstep, plan, ws, _flat(imgs, 3), _flat(tgts, 4), lam)
    ref_loss, ref_g = orc.l1_ssim_loss_grad(imgs, [orc.rgba8_to_float(t) for t in tgts], lam)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss), (loss, ref_loss)
    worst = 0.0
    for got, ref, img, t in zip(_split(dl, SHAPES), ref_g, imgs, tgts):
        tie = np.abs(img.astype(np.float64) - orc.rgba8_to_float(t)) < 1e-6
        err = _grad_err(got, ref, tie)
        assert np.isfinite(got).all()
        assert err.max() <= 1e-3, err.max()
        worst = max(worst, err.max())
    report(f"l1_ssim_small_lambda{lam}_smooth{int(smooth)}",
           {"loss_rel_err": abs(loss - ref_loss) / abs(ref_loss), "grad_max_err": worst})


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_l1_ssim_alpha_masked_matches_oracle(gs, orc, report, lam):
    """gs_loss_l1_ssim_masked: the reference's alpha (0, 255 and values in
    between) masks render and reference; loss and every pixel's gradient
    against the oracle's masked loss."""
    gsstep, _ = gs
    imgs, tgts = synth.loss_images(SHAPES, seed=21, smooth=True)
    rng = np.random.default_rng(22)
    for t in tgts:
        u = rng.uniform(size=t.shape[:2])
        t[..., 3] = np.where(u < 0.3, 0, np.where(u < 0.6, 255, rng.integers(1, 255, size=u.shape))).astype(np.uint8)
    plan, ws = _plan(gsstep, SHAPES)
    dl = torch.full_like(_flat(imgs, 3), np.nan)
    gsstep.gs_loss_l1_ssim_masked(plan, ws, _flat(imgs, 3), _flat(tgts, 4), lam, dl)
    torch.cuda.synchronize()
    loss, dl = gsstep.gs_read_stats(plan, ws).loss, dl.cpu().numpy()
    masks = [orc.rgba8_alpha(t) for t in tgts]
    ref_loss, ref_g = orc.l1_ssim_loss_grad(imgs, [orc.rgba8_to_float(t) for t in tgts], lam, masks=masks)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss), (loss, ref_loss)
    worst = 0.0
    for got, ref, img, t, m in zip(_split(dl, SHAPES), ref_g, imgs, tgts, masks):
        tie = np.abs(m[..., None] * (img.astype(np.float64) - orc.rgba8_to_float(t))) < 1e-6
        err = _grad_err(got, ref, tie)
        assert np.isfinite(got).all()
        assert not got[m == 0].any()
        assert err.max() <= 1e-3, err.max()
        worst = max(worst, err.max())
    report(f"l1_ssim_alpha_masked_lambda{lam}", {"loss_rel_err": abs(loss - ref_loss) / abs(ref_loss),
                                                  "grad_max_err": worst})


def test_lambda_zero_is_l1(gs):
    gsstep, _ = gs
    imgs, tgts = synth.loss_images(SHAPES, seed=5)
    plan, ws = _plan(gsstep, SHAPES)
    img_d, tgt_d = _flat(imgs, 3), _flat(tgts, 4)
    loss, dl = _run(gsstep, plan, ws, img_d, tgt_d, 0.0)
    tf = (tgt_d[:, :3].float().cpu().numpy() * np.float32(1.0 / 255.0)).astype(np.float32)
    dl1 = torch.full_like(img_d, np.nan)
    gsstep.gs_loss_l1(plan, ws, img_d, torch.from_numpy(tf).cuda(), dl1)
    torch.cuda.synchronize()
    loss1 = gsstep.gs_read_stats(plan, ws).loss
    assert np.array_equal(dl, dl1.cpu().numpy())
    assert abs(loss - loss1) <= 1e-6 * loss1


def test_invalid_arguments(gs):
    gsstep, _ = gs
    plan, ws = _plan(gsstep, [(32, 32)])
    img = torch.zeros((32 * 32, 3), device="cuda")
    tgt = torch.zeros((32 * 32 * 4 + 4,), dtype=torch.uint8, device="cuda")
    dl = torch.zeros_like(img)
    for lam in (-0.1, 1.5, float("nan")):
        with pytest.raises(gsstep.GSError):
            gsstep.gs_loss_l1_ssim(plan, ws, img, tgt, lam, dl)
    with pytest.raises(gsstep.GSError):
        gsstep.gs_loss_l1_ssim(plan, ws, img, tgt[1:], 0.2, dl)   # target not 4-byte aligned
    torch.cuda.synchronize()


def test_trainer_step_with_ssim_loss(gs, orc):
    """The training step with the L1 + SSIM loss: the loss gradient the step
    feeds to the rasterization backward matches the oracle's on the step's
    own render, and the step leaves finite parameters."""
    gsstep, step_mod = gs
    scene, target_scene, cams = synth.tiny_workload(seed=3)
    tr = step_mod.Trainer([scene], cams, lr=(1e-3,) * 6, loss="l1_ssim", ssim_lambda=0.2)
    b = orc.bin32(target_scene, cams[0], 16, 16)
    P = orc.project64(orc.Params64.from_scene(target_scene), cams[0], 16, 16)
    tgt = orc.render64(cams[0], P, b, (0.0, 0.0, 0.0), 1e-4, 16, 16).image
    tr.set_target([tgt])
    tr.forward()
    tr.backward_adam(step=1)
    torch.cuda.synchronize()
    img = tr.image_views()[0].cpu().numpy()
    t8 = tr.target.cpu().numpy().reshape(img.shape[0], img.shape[1], 4)
    ref_loss, ref_g = orc.l1_ssim_loss_grad([img], [orc.rgba8_to_float(t8)], 0.2)
    assert abs(tr.stats().loss - ref_loss) <= 1e-5 * ref_loss
    got = tr.dl.cpu().numpy().reshape(img.shape)
    tie = np.abs(img.astype(np.float64) - orc.rgba8_to_float(t8)) < 1e-6
    assert _grad_err(got, ref_g[0], tie).max() <= 1e-3
    assert torch.isfinite(tr.scenes[0].geom).all() and torch.isfinite(tr.scenes[0].sh).all()


def test_l1_ssim_full_size_four_views(gs, orc, report):
    """The batched workload's size: four 1920x1080 views (smooth images with
    flat regions), loss and every pixel's gradient against the oracle."""
    gsstep, _ = gs
    shapes = [(1920, 1080)] * 4
    imgs, tgts = synth.loss_images(shapes, seed=21, smooth=True)
    plan, ws = _plan(gsstep, shapes)
    loss, dl = _run(gsstep, plan, ws, _flat(imgs, 3), _flat(tgts, 4), 0.2)
    ref_loss, ref_g = orc.l1_ssim_loss_grad(imgs, [orc.rgba8_to_float(t) for t in tgts], 0.2)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss), (loss, ref_loss)
    worst = 0.0
    for got, ref, img, t in zip(_split(dl, shapes), ref_g, imgs, tgts):
        tie = np.abs(img.astype(np.float64) - orc.rgba8_to_float(t)) < 1e-6
        err = _grad_err(got, ref, tie)
        assert err.max() <= 1e-3, err.max()
        worst = max(worst, err.max())
    report("l1_ssim_4x1080p", {"loss_rel_err": abs(loss - ref_loss) / abs(ref_loss), "grad_max_err": worst})
