"""Pins of the oracle's default densification (Sec. 4.6, the 3DGS default
strategy) against closed forms and invariants, no GPU."""
import numpy as np
import pytest

from paper_2605_00219_gb300 import synth


def _scene(n, seed, smax=None):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    scales = np.exp(rng.normal(-4.0, 0.5, size=(n, 3)))
    if smax is not None:
        scales = np.tile(np.asarray(smax, np.float64), (n, 1))
    from oracle.oracle import DenseScene
    return DenseScene(rng.uniform(-1, 1, size=(n, 3)).astype(np.float32), q.astype(np.float32),
                      scales.astype(np.float32), rng.uniform(0.05, 0.95, size=n).astype(np.float32),
                      rng.normal(size=(n, 48)).astype(np.float32), rng.normal(size=(n, 60)).astype(np.float32),
                      np.abs(rng.normal(size=(n, 60))).astype(np.float32), np.zeros((n, 2), np.float32))


def test_quiet_scene_is_unchanged(orc):
    sc = _scene(50, 0)
    out, counts = orc.densify64(sc, np.zeros((50, 6)), scene_scale=1.0)
    assert counts == (50, 0, 0, 50)
    for f in ("means", "quats", "scales", "opacities", "sh", "m", "v"):
        assert np.array_equal(getattr(out, f), getattr(sc, f)), f
    assert not out.stats.any()


def test_clone_appends_a_copy_with_zero_moments(orc):
    sc = _scene(10, 1)
    sc.scales[:] = 0.005                      # small: <= 0.01 * scene_scale
    sc.stats[3] = (3e-4 * 4, 4)                # mean 3e-4 > 2e-4
    out, counts = orc.densify64(sc, np.zeros((10, 6)), scene_scale=1.0)
    assert counts == (10, 1, 0, 11)
    assert np.array_equal(out.means[10], sc.means[3]) and np.array_equal(out.sh[10], sc.sh[3])
    assert not out.m[10].any() and not out.v[10].any()
    assert np.array_equal(out.m[3], sc.m[3])  # the original keeps its moments


def test_threshold_directions(orc):
    """Strictly above grow_grad2d is high; a largest scale equal to
    grow_scale3d * scene_scale (binary32 product) counts as small; opacity
    equal to prune_opa survives."""
    f32 = np.float32
    sc = _scene(4, 2)
    thr_small = f32(0.01) * f32(2.0)
    sc.scales[:] = [[thr_small, 0.001, 0.001]] * 4
    sc.stats[0] = (f32(2e-4), 1)              # exactly the threshold: not high
    sc.stats[1] = (np.nextafter(f32(2e-4), f32(1)), 1)
    sc.opacities[2] = f32(0.005)
    sc.opacities[3] = np.nextafter(f32(0.005), f32(0))
    out, counts = orc.densify64(sc, np.zeros((4, 6)), scene_scale=2.0)
    assert counts == (3, 1, 0, 4)             # row 1 cloned (small), row 3 pruned
    assert np.array_equal(out.means[-1], sc.means[1])


def test_split_with_zero_draws(orc):
    sc = _scene(6, 3)
    sc.scales[:] = [[0.3, 0.05, 0.02]] * 6
    sc.stats[[1, 4]] = (1e-3, 1)
    out, counts = orc.densify64(sc, np.zeros((6, 6)), scene_scale=1.0)
    assert counts == (4, 0, 2, 8)
    rest = [0, 2, 3, 5]
    assert np.array_equal(out.means[:4], sc.means[rest])
    for k, src in enumerate([1, 4, 1, 4]):    # first products, then second products
        row = 4 + k
        np.testing.assert_array_equal(out.means[row], sc.means[src].astype(np.float64))
        np.testing.assert_array_equal(out.scales[row], (sc.scales[src] / np.float32(1.6)).astype(np.float32))
        assert np.array_equal(out.quats[row], sc.quats[src]) and np.array_equal(out.sh[row], sc.sh[src])
        assert out.opacities[row] == sc.opacities[src]
        assert not out.m[row].any() and not out.v[row].any()


def test_split_offsets_have_the_gaussian_covariance(orc):
    """The products' offsets mean + R(q)(s * eps) with eps ~ N(0, I) are
    distributed as the Gaussian itself: covariance R diag(s^2) R^T."""
    n = 40000
    rng = np.random.default_rng(4)
    q = np.array([0.8, 0.3, -0.4, 0.33])
    s = np.array([0.3, 0.1, 0.04])
    from oracle.oracle import DenseScene
    sc = DenseScene(np.zeros((n, 3), np.float32), np.tile(q, (n, 1)).astype(np.float32),
                    np.tile(s, (n, 1)).astype(np.float32), np.full(n, 0.5, np.float32), np.zeros((n, 48), np.float32),
                    np.zeros((n, 60), np.float32), np.zeros((n, 60), np.float32),
                    np.tile([1.0, 1.0], (n, 1)).astype(np.float32))
    eps = rng.normal(size=(n, 6))
    out, counts = orc.densify64(sc, eps, scene_scale=1.0)
    assert counts == (0, 0, n, 2 * n)
    qn = q / np.linalg.norm(q)
    w, x, y, z = qn
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    want = R @ np.diag(s * s) @ R.T
    got = np.cov(out.means.T)
    assert np.abs(got - want).max() <= 0.03 * np.abs(want).max()
    # the principal axis of the largest scale is R's first column
    evals, evecs = np.linalg.eigh(got)
    assert abs(abs(evecs[:, -1] @ R[:, 0]) - 1) < 1e-3


def test_prune_big_uses_the_split_scale(orc):
    f32 = np.float32
    sc = _scene(5, 5)
    sc.scales[:] = [[0.05, 0.01, 0.01], [0.12, 0.01, 0.01], [0.2, 0.01, 0.01], [0.12, 0.01, 0.01],
                    [0.05, 0.01, 0.01]]
    sc.stats[[1, 2]] = (1.0, 1)               # split: 0.12 -> 0.075 kept; 0.2 -> 0.125 pruned
    sc.opacities[4] = f32(0.001)              # pruned by opacity
    out, counts = orc.densify64(sc, np.zeros((5, 6)), scene_scale=1.0, prune_big=True)
    # row 3 (0.12, not split) is too big and pruned
    assert counts == (1, 0, 1, 3)
    assert np.array_equal(out.means[0], sc.means[0])
    np.testing.assert_array_equal(out.scales[1], (sc.scales[1] / f32(1.6)))
    out2, counts2 = orc.densify64(sc, np.zeros((5, 6)), scene_scale=1.0, prune_big=False)
    assert counts2 == (2, 0, 2, 6)


def test_grow_off_prunes_only(orc):
    sc = _scene(8, 6)
    sc.stats[:] = (1.0, 1)
    sc.opacities[2] = 0.0
    out, counts = orc.densify64(sc, np.zeros((8, 6)), scene_scale=1.0, grow=False)
    assert counts == (7, 0, 0, 7)


def test_reset_opacity(orc):
    sc = _scene(20, 7)
    out = orc.reset_opacity64(sc, 0.01)
    np.testing.assert_array_equal(out.opacities, np.minimum(sc.opacities, np.float32(0.01)))
    assert not out.m[:, 11].any() and not out.v[:, 11].any()
    keep = [i for i in range(60) if i != 11]
    assert np.array_equal(out.m[:, keep], sc.m[:, keep]) and np.array_equal(out.v[:, keep], sc.v[:, keep])


def test_statistic_counts_views_and_is_per_view_normalised(orc):
    """A view repeated in the batch adds the same per-view statistic again
    (each copy's share of the loss is halved and the P_all / P_view factor
    doubles), and the count of views grows by one per listed view."""
    scene, tgt_scene, cams = synth.tiny_workload(seed=8)
    scene.opacities[:5] = 0.001                # never listed
    cam = cams[0]
    b = orc.bin32(tgt_scene, cam)
    P = orc.project64(orc.Params64.from_scene(tgt_scene), cam)
    target = orc.render64(cam, P, b).image
    r1 = orc.step(scene, [cam], [target], (1e-3,) * 6, grad_only=True)
    r2 = orc.step(scene, [cam, cam], [target, target], (1e-3,) * 6, grad_only=True)
    s1 = orc.densify_stats64(r1, [cam])
    s2 = orc.densify_stats64(r2, [cam, cam])
    vis = r1.binnings[0].count > 0
    assert vis.any() and (~vis).any()
    np.testing.assert_array_equal(s1[:, 1], vis.astype(float))
    np.testing.assert_array_equal(s2[:, 1], 2 * vis.astype(float))
    np.testing.assert_allclose(s2[:, 0], 2 * s1[:, 0], rtol=1e-12, atol=1e-18)
    assert (s1[vis, 0] > 0).mean() > 0.5
