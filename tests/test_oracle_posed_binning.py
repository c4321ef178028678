"""Pins of the oracle's FP32 binning under general camera poses (no GPU).

The binning (Sec. 4.1 culling, Sec. 4.4 keys) re-derives the camera-space
position, the EWA covariance with its field-of-view clamp and the pixel mean
in FP32 before it lists tiles.  These tests look at it through cameras that
are neither axis-aligned nor centred: three elevations and azimuths,
non-square images, fx != fy, principal points off the image centre, and
Gaussians placed beyond 1.3x the half field of view so that the clamp of the
Jacobian is active.  Each quantity is tied to something other than the
binning itself:

- the FP64 projection's covariance equals the push-forward of the 3D
  covariance through the Jacobian of its own (separately pinned) pixel-mean
  map, taken by central differences at the clamped direction;
- the FP32 binning geometry equals the FP64 projection within FP32 rounding;
- every pixel that the FP64 contribution rule admits lies in a listed tile;
- tiled compositing equals a brute-force walk over all Gaussians;
- the listed tiles are exactly those an independent ellipse-rectangle test
  selects.

A transposed camera rotation or a clamp applied to t instead of t / t_z in
the binning fails the geometry, coverage and brute-force tests.
"""
import math

import numpy as np
import pytest

from paper_2605_00219_gb300 import synth

POSES = [(-35.0, 30.0, 144, 96), (15.0, 145.0, 100, 130), (60.0, 250.0, 128, 112)]


def _posed_cam(k):
    el, az, w, h = POSES[k]
    e, a = math.radians(el), math.radians(az)
    eye = 4.0 * np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a), math.sin(e)])
    cam = synth.look_at(eye, (0.1, -0.05, 0.08), w, h, fx=120.0 + 10.0 * k, fy=132.0 - 7.0 * k)
    cam.cx = w / 2.0 + 5.25 - 3.0 * k
    cam.cy = h / 2.0 - 4.125 + 2.0 * k
    return cam


def _limits(cam):
    return 1.3 * (0.5 * cam.width / cam.fx), 1.3 * (0.5 * cam.height / cam.fy)


def _to_world(cam, t_cam):
    """World points whose camera-space coordinates are t_cam (rows)."""
    R = cam.R.astype(np.float64)
    return (np.asarray(t_cam, np.float64) - cam.t.astype(np.float64)) @ R


def _posed_scene(cam, seed, n_inside=150, n_clamped=24):
    """Gaussians around the look-at point, plus large ones whose centres lie
    beyond 1.3x the half field of view (left/right and above/below) at depths
    2-5, so that their clamped footprints still reach into the image."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.4, 1.4, size=(n_inside, 3))
    scales = np.exp(rng.normal(-2.2, 0.8, size=(n_inside, 3)))
    limx, limy = _limits(cam)
    tz = rng.uniform(2.0, 5.0, size=n_clamped)
    side = np.where(rng.uniform(size=n_clamped) < 0.5, -1.0, 1.0)
    over = rng.uniform(1.05, 1.6, size=n_clamped)
    u = np.where(np.arange(n_clamped) % 2 == 0, side * over * limx, rng.uniform(-limx, limx, n_clamped) / 1.3)
    v = np.where(np.arange(n_clamped) % 2 == 1, side * over * limy, rng.uniform(-limy, limy, n_clamped) / 1.3)
    t_cam = np.stack([u * tz, v * tz, tz], axis=1)
    means = np.concatenate([means, _to_world(cam, t_cam)])
    scales = np.concatenate([scales, rng.uniform(0.25, 0.8, size=(n_clamped, 3))])
    n = n_inside + n_clamped
    q = rng.normal(size=(n, 4))
    opac = 10.0 ** rng.uniform(-2.6, 0.0, size=n)
    sh = rng.normal(0.0, 0.3, size=(n, 16, 3))
    f = lambda a: np.asarray(a, np.float32)
    return synth.Scene(f(means), f(q), f(scales), f(opac), f(sh))


def _clamped(cam, P):
    """Gaussians whose direction lies beyond the clamp (either axis)."""
    limx, limy = _limits(cam)
    ok = P[:, 0] > 0
    tz = np.where(ok, P[:, 3], 1.0)
    return ok & ((np.abs(P[:, 1] / tz) > limx) | (np.abs(P[:, 2] / tz) > limy))


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("k", range(len(POSES)))
def test_projection_covariance_is_pushforward_of_mean_map(orc, k):
    """Sigma_2D - 0.3 I of the FP64 projection equals J Sigma J^T, with J the
    central-difference Jacobian of the projection's own pixel mean (pinned by
    the rotated-camera closed form) with respect to the world position,
    evaluated at the point of the same depth along the clamped direction; the
    3D covariance Sigma = R(q) diag(s^2) R(q)^T is formed here from its
    definition."""
    cam = _posed_cam(k)
    sc = _posed_scene(cam, 100 + k)
    p = orc.Params64.from_scene(sc)
    P = orc.project64(p, cam)
    limx, limy = _limits(cam)
    clamped = _clamped(cam, P)
    assert clamped.sum() >= 10
    checked = 0
    for g in np.nonzero(P[:, 0] > 0)[0]:
        t = P[g, 1:4]
        uc = np.clip(t[0] / t[2], -limx, limx)
        vc = np.clip(t[1] / t[2], -limy, limy)
        x0 = _to_world(cam, [[uc * t[2], vc * t[2], t[2]]])[0]
        h = 1e-5 * max(1.0, t[2])
        J = np.zeros((2, 3))
        for j in range(3):
            pts = np.repeat(x0[None, :], 2, axis=0)
            pts[0, j] += h
            pts[1, j] -= h
            one = orc.Params64(pts, np.repeat(p.quats[g:g + 1], 2, 0), np.repeat(p.scales[g:g + 1], 2, 0),
                               np.repeat(p.opacities[g:g + 1], 2, 0), np.repeat(p.sh[g:g + 1], 2, 0))
            Pm = orc.project64(one, cam)
            J[:, j] = (Pm[0, 4:6] - Pm[1, 4:6]) / (2 * h)
        R = _rot(p.quats[g])
        Sig = R @ np.diag(p.scales[g] ** 2) @ R.T
        V = J @ Sig @ J.T
        cov = np.array([[P[g, 6], P[g, 7]], [P[g, 7], P[g, 8]]]) - 0.3 * np.eye(2)
        scale = math.sqrt(V[0, 0] * V[1, 1]) + 1e-12
        assert np.abs(cov - V).max() <= 1e-6 * scale + 1e-9, (g, cov, V)
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("k", range(len(POSES)))
def test_binning_geometry_matches_fp64_projection(orc, k):
    """The FP32 binning's pixel mean, 2D covariance (a, b, c) and depth agree
    with the FP64 projection within FP32 rounding, also for clamped
    Gaussians, and both cull the same Gaussians."""
    cam = _posed_cam(k)
    sc = _posed_scene(cam, 200 + k)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    b = orc.bin32(sc, cam)
    valid32 = b.bin[:, 0] > 0
    listed_op = sc.opacities.astype(np.float64) * 255.0 > 1.0
    np.testing.assert_array_equal(valid32, (P[:, 0] > 0) & listed_op)
    g = np.nonzero(valid32)[0]
    B = b.bin[g].astype(np.float64)
    span = max(cam.width, cam.height)
    err_m = np.abs(B[:, 1:3] - P[g, 4:6]) / (np.abs(P[g, 4:6]) + span)
    assert err_m.max() <= 2e-6, err_m.max()
    scale = np.sqrt(P[g, 6] * P[g, 8])
    err_c = np.abs(B[:, 3:6] - P[g, 6:9]).max(axis=1) / scale
    assert err_c.max() <= 2e-5, err_c.max()
    np.testing.assert_allclose(B[:, 7], P[g, 3], rtol=1e-6)
    assert _clamped(cam, P)[g].sum() >= 5


@pytest.mark.parametrize("k", range(len(POSES)))
def test_no_false_negatives_posed(orc, k):
    """Every pixel where the FP64 rule (d^2 <= 9 and o exp(-d^2/2) >= 1/255)
    holds for a Gaussian lies in a tile that the FP32 binning lists for it."""
    cam = _posed_cam(k)
    sc = _posed_scene(cam, 300 + k)
    b = orc.bin32(sc, cam)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    TX, TY = orc.tiles_of(cam)
    shift = orc.key_shift(TX * TY)
    yy, xx = np.mgrid[0:cam.height, 0:cam.width]
    ys, xs = yy + 0.5, xx + 0.5
    tiles_px = (yy // 16) * TX + (xx // 16)
    clamped_hits = hits = 0
    clamped = _clamped(cam, P)
    for g in np.nonzero(P[:, 0] > 0)[0]:
        dx, dy = xs - P[g, 4], ys - P[g, 5]
        d2 = P[g, 9] * dx * dx + 2 * P[g, 10] * dx * dy + P[g, 11] * dy * dy
        alpha = P[g, 12] * np.exp(-0.5 * d2)
        need = set(np.unique(tiles_px[(d2 <= 9.0) & (alpha >= 1.0 / 255.0)]).tolist())
        listed = set((b.keys_emit[b.offset[g]:b.offset[g + 1]] >> shift).tolist())
        assert need <= listed, g
        hits += bool(need)
        clamped_hits += bool(need) and bool(clamped[g])
    assert hits > 50 and clamped_hits >= 3, (hits, clamped_hits)


def _depth_order(b, n_tiles):
    tb = 0
    while (1 << tb) < n_tiles:
        tb += 1
    drop = tb - 9 if tb >= 9 else 0
    g = np.nonzero(b.bin[:, 0] > 0)[0]
    return g[np.argsort(b.mant[g] >> drop, kind="stable")]


@pytest.mark.parametrize("k", range(len(POSES)))
def test_tiled_equals_bruteforce_posed(orc, k):
    """Tiled compositing over the culled, sorted tile lists equals a per-pixel
    walk over all Gaussians in the same depth order with the same rule."""
    cam = _posed_cam(k)
    sc = _posed_scene(cam, 400 + k, n_inside=400)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    b = orc.bin32(sc, cam)
    TX, TY = orc.tiles_of(cam)
    r = orc.render64(cam, P, b, bg=(0.1, 0.2, 0.3))
    img, tf, bl = orc.render64_brute(cam, P, _depth_order(b, TX * TY), bg=(0.1, 0.2, 0.3))
    assert r.blended == bl and bl > 1000
    assert np.array_equal(r.image, img)
    assert np.array_equal(r.tfinal, tf)


def _rect_meets_ellipse(mx, my, Q, r2, x0, x1, y0, y1):
    """Does the closed ellipse d^T Q d <= r2 meet [x0,x1]x[y0,y1]?  The form
    is convex: its minimum is at the centre if inside, else on an edge."""
    if x0 <= mx <= x1 and y0 <= my <= y1:
        return True
    best = np.inf
    for ey in (y0, y1):
        dy = ey - my
        dx = min(max(-Q[0, 1] * dy / Q[0, 0], x0 - mx), x1 - mx)
        best = min(best, Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy)
    for ex in (x0, x1):
        dx = ex - mx
        dy = min(max(-Q[0, 1] * dx / Q[1, 1], y0 - my), y1 - my)
        best = min(best, Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy)
    return best <= r2


@pytest.mark.parametrize("k,tile", [(0, (16, 16)), (1, (8, 8)), (2, (16, 32))])
def test_scanline_equals_exact_rectangle_test_posed(orc, k, tile):
    """On posed cameras, the tiles listed for each Gaussian are those whose
    pixel-centre rectangle meets its FP64 ellipse d^2 <= r^2(o), sandwiched
    between r^2 (1 -+ 1e-4) to absorb the FP32 geometry."""
    tw, th = tile
    cam = _posed_cam(k)
    sc = _posed_scene(cam, 500 + k)
    b = orc.bin32(sc, cam, tw, th)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    TX, TY = orc.tiles_of(cam, tw, th)
    shift = orc.key_shift(TX * TY)
    checked = 0
    for g in np.nonzero(b.bin[:, 0] > 0)[0]:
        o = float(sc.opacities[g])
        r2 = min(9.0, 2.0 * math.log(255.0 * o)) * (1.0 + 2.0 ** -10) + 2.0 ** -10
        listed = set((b.keys_emit[b.offset[g]:b.offset[g + 1]] >> shift).tolist())
        mx, my = P[g, 4], P[g, 5]
        Q = np.linalg.inv(np.array([[P[g, 6], P[g, 7]], [P[g, 7], P[g, 8]]]))
        inner, outer = set(), set()
        for ty in range(TY):
            for tx in range(TX):
                x0, x1 = tx * tw + 0.5, (tx + 1) * tw - 0.5
                y0, y1 = ty * th + 0.5, (ty + 1) * th - 0.5
                if _rect_meets_ellipse(mx, my, Q, r2 * (1 - 1e-4), x0, x1, y0, y1):
                    inner.add(ty * TX + tx)
                if _rect_meets_ellipse(mx, my, Q, r2 * (1 + 1e-4), x0, x1, y0, y1):
                    outer.add(ty * TX + tx)
        assert inner <= listed <= outer, g
        checked += bool(listed)
    assert checked > 50
