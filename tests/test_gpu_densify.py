"""Default densification on the GPU (Sec. 4.6, the 3DGS default strategy)
against the oracle, through the C ABI.

Bars: decisions and counts bit-exact (binary32 comparisons of stored
values); copied rows, split scales and zeroed moments bit-exact; split means
within 2e-6 of the FP64 oracle; the gradient statistic within 1e-3 relative
on Gaussians away from threshold flips, its view count exact."""
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


def _rows(sb):
    """Device SceneBuffers -> the oracle's row layout (float32 copies)."""
    n = sb.n
    geom = sb.geom.float().cpu().numpy()
    sh = sb.sh.float().cpu().numpy().transpose(1, 0, 2).reshape(n, 48)
    m = sb.m.float().cpu().numpy().transpose(1, 0, 2).reshape(n, 60)
    v = sb.v.float().cpu().numpy().transpose(1, 0, 2).reshape(n, 60)
    st = sb.stats.cpu().numpy() if sb.stats is not None else np.zeros((n, 2), np.float32)
    return geom[0, :, :3].copy(), geom[1].copy(), geom[2, :, :3].copy(), geom[2, :, 3].copy(), sh, m, v, st


def _device_scene(step_mod, seed, n, bf16):
    rng = np.random.default_rng(seed)
    sc = synth.uniform_scene(n, seed)
    sc.scales = np.exp(rng.normal(-4.2, 0.9, size=(n, 3))).astype(np.float32)   # both sides of 0.01
    sc.opacities = rng.uniform(0.0, 0.03, size=n).astype(np.float32)           # some below 0.005
    sc.opacities[: n // 2] = rng.uniform(0.01, 0.99, size=n // 2)
    sb = step_mod.SceneBuffers.from_scene(sc, "cuda", bf16, bf16)
    mdt = sb.m.dtype
    sb.m.copy_(torch.from_numpy(rng.normal(size=(15, n, 4)).astype(np.float32)).to(mdt))
    sb.v.copy_(torch.from_numpy(np.abs(rng.normal(size=(15, n, 4))).astype(np.float32)).to(mdt))
    cnt = rng.integers(0, 5, size=n).astype(np.float32)
    stats = np.stack([rng.uniform(0.0, 6e-4, size=n).astype(np.float32) * cnt, cnt], 1)
    sb.stats = torch.from_numpy(stats).cuda()
    return sb


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("prune_big", [False, True])
def test_densify_matches_oracle(gs, orc, bf16, prune_big):
    gsstep, step_mod = gs
    n = 5000
    sb = _device_scene(step_mod, 11 + bf16, n, bf16)
    eps = np.random.default_rng(5).normal(size=(n, 6)).astype(np.float32)
    cfg = gsstep.make_densify_cfg(scene_scale=1.5, prune_big=prune_big)
    scratch = torch.empty(gsstep.gs_densify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    gsstep.gs_densify_count(sb, sb.storage_flags, cfg, scratch)
    counts = gsstep.gs_densify_counts(scratch)
    ref_in = orc.DenseScene(*_rows(sb))
    ref, ref_counts = orc.densify64(ref_in, eps.astype(np.float64), 1.5, prune_big=prune_big)
    assert counts == ref_counts
    assert counts[1] > 10 and counts[2] > 10 and counts[0] + counts[2] < n   # clone, split and prune all occur
    out = step_mod.SceneBuffers.empty_like_layout(sb, counts[3])
    gsstep.gs_densify_apply(sb, sb.storage_flags, cfg, torch.from_numpy(eps).cuda(), scratch, out)
    torch.cuda.synchronize()
    means, quats, scales, opac, sh, m, v, st = _rows(out)
    ns = counts[0] + counts[1]
    assert np.array_equal(means[:ns], ref.means[:ns].astype(np.float32))
    assert np.abs(means[ns:] - ref.means[ns:]).max() <= 2e-6
    for got, want in ((quats, ref.quats), (scales, ref.scales), (opac, ref.opacities), (sh, ref.sh), (m, ref.m),
                      (v, ref.v)):
        assert np.array_equal(got, want.astype(np.float32))
    assert not st.any()


def test_wrong_output_size_writes_nothing(gs):
    gsstep, step_mod = gs
    sb = _device_scene(step_mod, 3, 700, False)
    cfg = gsstep.make_densify_cfg(scene_scale=1.0)
    scratch = torch.empty(gsstep.gs_densify_scratch_bytes(sb.n), dtype=torch.uint8, device="cuda")
    gsstep.gs_densify_count(sb, 0, cfg, scratch)
    total = gsstep.gs_densify_counts(scratch)[3]
    out = step_mod.SceneBuffers.empty_like_layout(sb, total + 1)
    out.geom.fill_(7.0)
    gsstep.gs_densify_apply(sb, 0, cfg, torch.zeros((sb.n, 6), device="cuda"), scratch, out)
    torch.cuda.synchronize()
    assert bool((out.geom == 7.0).all())
    with pytest.raises(gsstep.GSError):
        gsstep.gs_densify_count(sb, 0, gsstep.make_densify_cfg(scene_scale=0.0), scratch)


@pytest.mark.parametrize("bf16", [False, True])
def test_reset_opacity_matches_oracle(gs, orc, bf16):
    gsstep, step_mod = gs
    sb = _device_scene(step_mod, 8, 3000, bf16)
    ref = orc.reset_opacity64(orc.DenseScene(*_rows(sb)), 0.01)
    gsstep.gs_reset_opacity(sb, sb.storage_flags, 0.01)
    torch.cuda.synchronize()
    means, quats, scales, opac, sh, m, v, st = _rows(sb)
    assert np.array_equal(opac, ref.opacities) and np.array_equal(m, ref.m) and np.array_equal(v, ref.v)
    assert np.array_equal(scales, ref.scales) and np.array_equal(sh, ref.sh)


def _unstable_gaussians(P, r, cam):
    bad = r.unstable_g.copy()
    ys, xs = np.nonzero(r.unstable_px)
    for x, y in zip(xs, ys):
        dx = x + 0.5 - P[:, 4]
        dy = y + 0.5 - P[:, 5]
        d2 = P[:, 9] * dx * dx + 2 * P[:, 10] * dx * dy + P[:, 11] * dy * dy
        bad |= (P[:, 0] > 0) & (d2 <= 9.0 * (1 + 1e-3))
    return bad


def test_statistic_accumulated_in_the_step(gs, orc):
    """Two steps over three views of uneven size: the statistic the fused
    kernel accumulates equals the oracle's (summed over both steps' gradients,
    which the first step's Adam update barely moves)."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(6000, 8, 2.5, seed=6, log_scale=(-3.4, 0.4), logit_opacity=(0.0, 1.0))
    cams = [synth.look_at([0, -5, 1.5], [0, 0, 0], 96, 72, 90.0),
            synth.look_at([4, 2, 1], [0, 0, 0], 64, 80, 70.0),
            synth.look_at([-3, -3, 2], [0, 0, 0], 128, 64, 110.0)]
    tscene = synth.perturbed(scene, 9)
    p_t = orc.Params64.from_scene(tscene)
    targets = [orc.render64(c, orc.project64(p_t, c), orc.bin32(tscene, c)).image for c in cams]
    res = orc.step(scene, cams, targets, LR, grad_only=True)
    want = orc.densify_stats64(res, cams)
    tr = step_mod.Trainer([scene], cams, lr=(0.0,) * 6)      # lr 0: parameters stay, statistics add up
    tr.enable_densify_stats()
    tr.set_target([t.astype(np.float32) for t in targets])
    tr.step(step=1)
    tr.step(step=2)
    torch.cuda.synchronize()
    got = tr.scenes[0].stats.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got[:, 1], 2 * want[:, 1])
    bad = np.zeros(scene.n, bool)
    for c, r, P, tg in zip(cams, res.renders, res.projs, targets):
        r.unstable_px |= (np.abs(r.image - tg) < 1e-5).any(-1)
        bad |= _unstable_gaussians(P, r, c)
    ok = ~bad & (want[:, 0] > 1e-3 * np.median(want[want[:, 0] > 0, 0]))
    assert ok.sum() > 0.5 * scene.n
    w2 = 2 * want[ok, 0]
    rel = np.abs(got[ok, 0] - w2) / np.maximum(w2, np.sqrt(np.mean(w2 * w2)))
    assert rel.max() <= 1e-3, rel.max()


def test_trainer_densify_cycle(gs):
    """Training with statistics, one refinement (clone, split and prune all
    happen), an opacity reset and further graph-replayed steps: sizes add
    up, the Adam step counter carries over, parameters stay finite."""
    gsstep, step_mod = gs
    scene = synth.cluster_scene(20000, 8, 2.5, seed=7, log_scale=(-3.0, 0.8), logit_opacity=(-1.0, 2.0))
    cams = synth.orbit_cameras(2, 5.0, 128, 96, hfov_deg=55.0)
    tr = step_mod.Trainer([scene], cams, sh_bf16=True, mom_bf16=True)
    tr.enable_densify_stats()
    g = torch.Generator(device="cuda").manual_seed(0)
    tr.target.copy_(torch.rand(tr.target.shape, device="cuda", generator=g))
    for _ in range(4):
        tr.step(0)
    assert tr.stats().step == 4
    (kept, clones, splits, total), = tr.densify(scene_scale=2.5, generator=g, grow_grad2d=1e-5)
    assert clones > 0 and splits > 0 and kept + splits < scene.n
    assert tr.scenes[0].n == total == kept + clones + 2 * splits
    assert tr.stats().step == 4
    tr.reset_opacity(0.01)
    tr.capture()
    for _ in range(3):
        tr.replay()
    torch.cuda.synchronize()
    st = tr.stats()
    assert st.step == 7 and st.status == 0
    sb = tr.scenes[0]
    assert bool(torch.isfinite(sb.geom).all()) and bool(torch.isfinite(sb.sh.float()).all())
    assert float(sb.stats[:, 1].max()) > 0
