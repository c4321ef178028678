"""torch.autograd.Function over the CUDA step: several scenes of uneven size,
each with two views of mixed resolution, against the oracle's analytic
gradients and against central finite differences of the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import autograd, step
    return autograd, step


def _scenes():
    s0 = synth.cluster_scene(6000, 8, 2.5, seed=0, log_scale=(-3.5, 0.4), logit_opacity=(0.0, 1.0))
    s1 = synth.cluster_scene(2500, 4, 2.0, seed=1, log_scale=(-3.2, 0.4), logit_opacity=(0.0, 1.0))
    cams = [synth.look_at([0, -5, 1.5], [0, 0, 0], 96, 64, 110.0, scene=0),
            synth.look_at([4, 2, 1], [0, 0, 0], 64, 80, 90.0, scene=0),
            synth.look_at([-3, -3, 2], [0, 0, 0], 80, 48, 80.0, scene=1),
            synth.look_at([0, 4, 2], [0, 0, 0], 48, 48, 70.0, scene=1)]
    return [s0, s1], cams


def _oracle_grads(orc, scenes, cams, weights):
    """Activated-space gradients (n, 59) per scene and per-scene unstable masks."""
    out, bad = [], []
    for si, sc in enumerate(scenes):
        p = orc.Params64.from_scene(sc)
        g = np.zeros((sc.n, 59))
        b_ = np.zeros(sc.n, bool)
        for cam, w in zip(cams, weights):
            if cam.scene != si:
                continue
            b = orc.bin32(sc, cam)
            P = orc.project64(p, cam)
            r = orc.render64(cam, P, b)
            g2 = orc.raster_bwd64(cam, P, b, w)
            orc.project_bwd64(p, cam, P, g2, out=g)
            b_ |= r.unstable_g
            ys, xs = np.nonzero(r.unstable_px)
            for x, y in zip(xs, ys):
                dx, dy = x + 0.5 - P[:, 4], y + 0.5 - P[:, 5]
                d2 = P[:, 9] * dx * dx + 2 * P[:, 10] * dx * dy + P[:, 11] * dy * dy
                b_ |= (P[:, 0] > 0) & (d2 <= 9.0 * 1.001)
        act = np.concatenate([g[:, 0:3], g[:, 3:7], g[:, 7:10] / p.scales,
                              (g[:, 10] / (p.opacities * (1 - p.opacities)))[:, None], g[:, 11:]], axis=1)
        out.append(act)
        bad.append(b_)
    return out, bad


def _gpu_grads(n, dgeom, dsh):
    d = dgeom.cpu().numpy()
    s = dsh.float().cpu().numpy()
    if s.shape[0] == 6:
        s = s.reshape(6, n, 2, 4).transpose(0, 2, 1, 3).reshape(12, n, 4)
    return np.concatenate([d[0, :, :3], d[1], d[2], s.transpose(1, 0, 2).reshape(n, 48)], axis=1)


@pytest.mark.parametrize("bwd_impl", [0, 1, 2])
def test_autograd_multi_scene_vs_oracle(mods, orc, bwd_impl):
    autograd, step = mods
    scenes, cams = _scenes()
    R = autograd.Renderer([s.n for s in scenes], cams, bwd_impl=bwd_impl)
    bufs = [step.SceneBuffers.from_scene(s, moments=False) for s in scenes]
    params = []
    for b in bufs:
        params += [b.geom.clone().requires_grad_(True), b.sh.clone().requires_grad_(True)]
    img = R.render([(params[0], params[1]), (params[2], params[3])])
    rng = np.random.default_rng(0)
    weights = [rng.normal(size=(c.height, c.width, 3)) for c in cams]
    wt = torch.from_numpy(np.concatenate([w.reshape(-1, 3) for w in weights]).astype(np.float32)).cuda()
    loss = (img * wt).sum()
    loss.backward()
    ref, bad = _oracle_grads(orc, scenes, cams, [w.astype(np.float32).astype(np.float64) for w in weights])
    for si, sc in enumerate(scenes):
        gpu = _gpu_grads(sc.n, params[2 * si].grad, params[2 * si + 1].grad)
        good = ~bad[si] & (np.abs(ref[si]).sum(1) > 0)
        assert good.sum() > 0.5 * sc.n
        r_, g_ = ref[si][good], gpu[good]
        rms = np.sqrt((r_ ** 2).mean(0)) + 1e-30
        err = np.abs(g_ - r_) / np.maximum(np.abs(r_), rms[None, :])
        assert err.max() <= 1e-3, (si, err.max())


def test_autograd_bf16_sh_and_finite_differences(mods, orc):
    """BF16 SH storage through autograd, and the FP64 oracle's central finite
    differences (h = 1e-3 in theta) on sampled Gaussians."""
    autograd, step = mods
    scenes, cams = _scenes()
    scenes = [scenes[1]]
    cams = [c for c in cams if c.scene == 1]
    for c in cams:
        c.scene = 0
    sc = scenes[0]
    sc.sh = torch.from_numpy(sc.sh).to(torch.bfloat16).float().numpy()
    R = autograd.Renderer([sc.n], cams, sh_bf16=True)
    b = step.SceneBuffers.from_scene(sc, sh_bf16=True, moments=False)
    geom = b.geom.clone().requires_grad_(True)
    sh = b.sh.clone().requires_grad_(True)
    img = R.render([(geom, sh)])
    rng = np.random.default_rng(1)
    weights = [rng.normal(size=(c.height, c.width, 3)).astype(np.float32).astype(np.float64) for c in cams]
    wt = torch.from_numpy(np.concatenate([w.reshape(-1, 3) for w in weights]).astype(np.float32)).cuda()
    (img * wt).sum().backward()
    assert sh.grad.dtype == torch.bfloat16
    gpu = _gpu_grads(sc.n, geom.grad, sh.grad)
    # finite differences of the oracle in theta; convert GPU grads to theta
    p = orc.Params64.from_scene(sc)
    gth = gpu.copy()
    gth[:, 7:10] *= p.scales
    gth[:, 10] *= p.opacities * (1 - p.opacities)
    theta = p.theta()
    bins = [orc.bin32(sc, c) for c in cams]

    def L(th):
        pp = orc.Params64.from_theta(th)
        tot, sig = 0.0, []
        for c, bb, w in zip(cams, bins, weights):
            r = orc.render64(c, orc.project64(pp, c), bb)
            tot += float((r.image * w).sum())
            sig.append((r.blended, r.nlast.tobytes()))
        return tot, sig

    visible = np.nonzero(np.sum([bb.count for bb in bins], axis=0) > 0)[0]
    pick = rng.choice(visible, size=min(24, visible.size), replace=False)
    h = 1e-3
    checked = agree = 0
    for g in pick:
        for j in (0, 1, 2, 4, 7, 10, 11, 20):
            tp, tm = theta.copy(), theta.copy()
            tp[g, j] += h
            tm[g, j] -= h
            lp, sp = L(tp)
            lm, sm = L(tm)
            if sp != sm:
                continue            # a discrete decision changed within +-h
            fd = (lp - lm) / (2 * h)
            checked += 1
            scale = max(abs(fd), 1e-3 * np.sqrt((gth[visible] ** 2).mean()))
            if abs(gth[g, j] - fd) <= 2e-2 * scale:
                agree += 1
    assert checked >= 40
    assert agree >= 0.9 * checked, (agree, checked)
