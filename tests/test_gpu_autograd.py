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


def test_autograd_bf16_sh_and_finite_differences(mods, orc, report):
    """BF16 SH storage through autograd, and the FP64 oracle's central
    differences (outer step h = 1e-3 in theta, fourth-order stencil) on 64
    sampled Gaussians x 11 parameters against the FP32 gradients: relative
    error <= 1e-3 with an absolute floor of 1e-3 x the component's RMS, on every
    evaluation kept (those where a discrete decision changes within +-h are
    skipped and counted); the bf16 SH gradients are the FP32 ones rounded."""
    import types

    import fdcheck
    from paper_2605_00219_gb300 import gsstep
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
    n = sc.n
    go = torch.empty((15, n, 4), dtype=torch.float32, device="cuda")
    gsstep.gs_project_bwd_adam(R.plan, R.ws, [types.SimpleNamespace(n=n, geom=geom, sh=sh, m=None, v=None)],
                               R.cams, None, go)
    torch.cuda.synchronize()
    bf = go[3:15].reshape(6, 2, n, 4).permute(0, 2, 1, 3).reshape(6, n, 8).to(torch.bfloat16)
    assert torch.equal(bf, sh.grad) and torch.equal(go[0:3], geom.grad)
    g = go.cpu().numpy()
    dstored = np.concatenate([g[0, :, :3], g[1], g[2], g[3:15].transpose(1, 0, 2).reshape(n, 48)], axis=1)
    p = orc.Params64.from_scene(sc)
    gth = fdcheck.theta_grads(p, dstored)
    views = []
    for c, w in zip(cams, weights):
        views.append((c, orc.bin32(sc, c), orc.project64(p, c), w))
    listed = np.zeros(n, bool)
    for _, bb, _, _ in views:
        listed |= bb.count > 0
    rms = np.sqrt((gth[listed] ** 2).mean(0)) + 1e-30
    picks = rng.choice(np.nonzero(listed)[0], size=64, replace=False)
    res = fdcheck.fd_check(orc, sc, views, picks, gth, rms)
    report("autograd_bf16_fd", res)
    assert res["checked"] >= 300, res
    assert res["max_err"] <= 1e-3, res
