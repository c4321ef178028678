"""Checkpoint and resume: training resumed from a checkpoint repeats the
uninterrupted run bit for bit (deterministic kernels, BF16 rounding keyed by
seed, step and Gaussian), including densification statistics and after a
densification changed the scene size."""
import pytest
import torch

from paper_2605_00219_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def step_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import step
    return step


def _trainer(step_mod, scene, cams, target):
    tr = step_mod.Trainer([scene], cams, sh_bf16=True, mom_bf16=True, seed=7)
    tr.enable_densify_stats()
    tr.target.copy_(target)
    return tr


def _run(tr, n):
    """n steps: one eager, the rest graph replays (device step counter)."""
    tr.step(0)
    tr.capture()
    for _ in range(n - 1):
        tr.replay()
    torch.cuda.synchronize()


def _same(a, b):
    for x, y in zip(a.scenes, b.scenes):
        assert x.n == y.n
        for f in ("geom", "sh", "m", "v", "stats"):
            assert torch.equal(getattr(x, f), getattr(y, f)), f


def test_resume_equals_continuous(step_mod):
    scene = synth.cluster_scene(30000, 8, 2.5, seed=3, log_scale=(-3.0, 0.6), logit_opacity=(-0.5, 1.5))
    cams = synth.orbit_cameras(2, 5.0, 160, 120, hfov_deg=55.0)
    g = torch.Generator(device="cuda").manual_seed(1)
    target = torch.rand((sum(c.width * c.height for c in cams), 3), device="cuda", generator=g)

    full = _trainer(step_mod, scene, cams, target)
    _run(full, 10)
    part = _trainer(step_mod, scene, cams, target)
    _run(part, 4)
    ckpt = part.state_dict()
    assert ckpt["step"] == 4
    resumed = _trainer(step_mod, scene, cams, target)
    resumed.load_state_dict(ckpt)
    _run(resumed, 6)
    assert resumed.stats().step == full.stats().step == 10
    _same(full, resumed)


def test_resume_after_densification(step_mod):
    scene = synth.cluster_scene(30000, 8, 2.5, seed=4, log_scale=(-3.0, 0.8), logit_opacity=(-1.0, 2.0))
    cams = synth.orbit_cameras(2, 5.0, 160, 120, hfov_deg=55.0)
    g = torch.Generator(device="cuda").manual_seed(2)
    target = torch.rand((sum(c.width * c.height for c in cams), 3), device="cuda", generator=g)

    def densified(t):
        _run(t, 3)
        gen = torch.Generator(device="cuda").manual_seed(5)
        t.densify(scene_scale=2.5, generator=gen, grow_grad2d=1e-5)
        return t

    full = densified(_trainer(step_mod, scene, cams, target))
    _run(full, 5)
    part = densified(_trainer(step_mod, scene, cams, target))
    _run(part, 2)
    ckpt = part.state_dict()
    resumed = _trainer(step_mod, scene, cams, target)       # original size: re-plans on load
    resumed.load_state_dict(ckpt)
    assert resumed.scenes[0].n == full.scenes[0].n != scene.n
    _run(resumed, 3)
    assert resumed.stats().step == full.stats().step == 8
    _same(full, resumed)


def test_host_fed_replays_equal_device_steps(step_mod):
    """run_from_host (two graphs over two input buffer sets, host copies
    overlapping the previous step) computes the same steps as plain graph
    replays with the inputs already on the device."""
    scene = synth.cluster_scene(20000, 8, 2.5, seed=5, log_scale=(-3.0, 0.6), logit_opacity=(-0.5, 1.5))
    cams = synth.orbit_cameras(2, 5.0, 160, 120, hfov_deg=55.0)
    g = torch.Generator(device="cuda").manual_seed(3)
    target = torch.rand((sum(c.width * c.height for c in cams), 3), device="cuda", generator=g)
    a = _trainer(step_mod, scene, cams, target)
    a.capture()
    for _ in range(5):
        a.replay()
    torch.cuda.synchronize()
    b = _trainer(step_mod, scene, cams, target)
    host_t = target.cpu().pin_memory()
    host_c = b.cams.cpu().pin_memory()
    losses = b.run_from_host(lambda k: host_t, lambda k: host_c, 5)
    assert len(losses) == 5 and b.stats().step == a.stats().step == 5
    _same(a, b)
