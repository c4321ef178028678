"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties one part of the oracle to a closed form, a brute-force
evaluation, an exact geometric test, a library routine or finite differences,
so that a dropped term, a wrong sign or index or a transposed operand in the
oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2605_00219_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers written independently of the oracle
# ---------------------------------------------------------------------------

def _quat_z(deg):
    h = math.radians(deg) / 2
    return np.array([math.cos(h), 0.0, 0.0, math.sin(h)], np.float32)


def _one_scene(means, quats, scales, opac, sh=None):
    n = len(means)
    if sh is None:
        sh = np.zeros((n, 16, 3), np.float32)
    return synth.Scene(np.asarray(means, np.float32).reshape(n, 3), np.asarray(quats, np.float32).reshape(n, 4),
                       np.asarray(scales, np.float32).reshape(n, 3), np.asarray(opac, np.float32).reshape(n),
                       np.asarray(sh, np.float32).reshape(n, 16, 3))


def _alpha_closed(px, py, mx, my, Q, o):
    dx, dy = px - mx, py - my
    d2 = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
    a = np.minimum(0.99, o * np.exp(-0.5 * d2))
    a = np.where((d2 <= 9.0) & (a >= 1 / 255), a, 0.0)
    return a


def _rect_meets_ellipse(mx, my, Q, r2, x0, x1, y0, y1):
    """Exact test: does the closed ellipse d^T Q d <= r2 meet the rectangle
    [x0,x1]x[y0,y1]?  The quadratic form is convex, so its minimum over the
    rectangle is at the centre (if inside) or on one of the four edges."""
    if x0 <= mx <= x1 and y0 <= my <= y1:
        return True
    best = np.inf
    for ey in (y0, y1):          # horizontal edges: minimise over dx
        dy = ey - my
        dx = -Q[0, 1] * dy / Q[0, 0]
        dx = min(max(dx, x0 - mx), x1 - mx)
        best = min(best, Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy)
    for ex in (x0, x1):          # vertical edges: minimise over dy
        dx = ex - mx
        dy = -Q[0, 1] * dx / Q[1, 1]
        dy = min(max(dy, y0 - my), y1 - my)
        best = min(best, Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy)
    return best <= r2


# ---------------------------------------------------------------------------
# SH basis
# ---------------------------------------------------------------------------

def test_sh_orthonormal_by_quadrature(orc):
    """Real SH basis of degree <= 3 is orthonormal on the sphere: Gauss-Legendre
    in cos(theta) (exact to degree 39) times a uniform phi rule."""
    xs, ws = np.polynomial.legendre.leggauss(20)
    nphi = 40
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y, _ = orc.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_and_sign_convention(orc):
    """Y_00 = 1/(2 sqrt(pi)); degree-1 functions are -c y, c z, -c x with
    c = sqrt(3/(4 pi)) (the sign convention of the 3DGS family)."""
    d = np.array([0.36, -0.48, 0.8])
    Y, _ = orc.sh_basis(d)
    assert Y[0] == pytest.approx(1 / (2 * math.sqrt(math.pi)), rel=1e-15)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:4], [-c1 * d[1], c1 * d[2], -c1 * d[0]], rtol=1e-14)


def test_sh_basis_derivative_fd(orc):
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        _, dY = orc.sh_basis(d)
        h = 1e-6
        for i in range(3):
            e = np.zeros(3); e[i] = h
            fd = (orc.sh_basis(d + e)[0] - orc.sh_basis(d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, i], fd, atol=1e-8)


# ---------------------------------------------------------------------------
# Projection closed forms
# ---------------------------------------------------------------------------

def test_projection_isotropic_at_origin(orc):
    """Isotropic Gaussian (scale sigma) at the origin, camera at z = -4:
    Sigma2 = (fx sigma / 4)^2 I + 0.3 I and mean2D = (cx, cy)."""
    cam = synth.tiny_camera()
    sig = 0.05
    sc = _one_scene([[0, 0, 0]], [[1, 0, 0, 0]], [[sig, sig, sig]], [0.5])
    P = orc.project64(orc.Params64.from_scene(sc), cam)[0]
    s = np.float64(np.float32(sig))
    assert P[0] == 1
    assert P[4] == pytest.approx(cam.cx) and P[5] == pytest.approx(cam.cy)
    assert P[6] == pytest.approx((150 * s / 4) ** 2 + 0.3, rel=1e-12)
    assert P[8] == pytest.approx((150 * s / 4) ** 2 + 0.3, rel=1e-12)
    assert abs(P[7]) < 1e-15
    b = orc.bin32(sc, cam).bin[0]
    assert b[0] == 1
    np.testing.assert_allclose(b[1:6], [64, 64, (150 * s / 4) ** 2 + 0.3, 0, (150 * s / 4) ** 2 + 0.3], rtol=1e-6, atol=1e-7)


def test_projection_offset_and_rotation(orc):
    """A Gaussian at world (d, 0, 0) rotated 90 deg about z with scales
    (s1, s2, s3): Sigma = diag(s2^2, s1^2, s3^2); in camera space it sits at
    (d, 0, 4) so mean2D = (fx d/4 + cx, cy) and the Jacobian's third column
    adds (fx d / 16)^2 s3^2 to a."""
    cam = synth.tiny_camera()
    d, s1, s2, s3 = 0.3, 0.02, 0.07, 0.04
    sc = _one_scene([[d, 0, 0]], [_quat_z(90)], [[s1, s2, s3]], [0.5])
    P = orc.project64(orc.Params64.from_scene(sc), cam)[0]
    f = lambda v: float(np.float32(v))
    d, s1, s2, s3 = f(d), f(s1), f(s2), f(s3)
    fx = 150.0
    assert P[4] == pytest.approx(fx * d / 4 + 64, rel=1e-12)
    assert P[5] == pytest.approx(64, abs=1e-12)
    a = (fx / 4) ** 2 * s2 ** 2 + (fx * d / 16) ** 2 * s3 ** 2 + 0.3
    c = (fx / 4) ** 2 * s1 ** 2 + 0.3
    assert P[6] == pytest.approx(a, rel=1e-6)
    assert P[8] == pytest.approx(c, rel=1e-6)
    assert abs(P[7]) < 1e-9
    np.testing.assert_allclose(P[9:12], [1 / a, 0, 1 / c], rtol=1e-6, atol=1e-12)


def test_projection_camera_rotation(orc):
    """Camera rotated 90 deg about its optical axis (world x -> camera y):
    a Gaussian at world (d, 0, 0) lands at (cx, fy d / 4 + cy)."""
    cam = synth.tiny_camera()
    cam.R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float32)
    d = 0.25
    sc = _one_scene([[d, 0, 0]], [[1, 0, 0, 0]], [[0.03, 0.03, 0.03]], [0.5])
    P = orc.project64(orc.Params64.from_scene(sc), cam)[0]
    assert P[4] == pytest.approx(64, abs=1e-12)
    assert P[5] == pytest.approx(150 * d / 4 + 64, rel=1e-12)


def test_near_plane_and_colour(orc):
    """Behind the near plane (t_z < 0.01) is culled; a degree-0-only SH gives
    colour max(0, Y00 k + 0.5)."""
    cam = synth.tiny_camera()
    sh = np.zeros((2, 16, 3), np.float32)
    sh[:, 0, :] = [[0.3, -0.2, -3.0], [0.1, 0.1, 0.1]]
    sc = _one_scene([[0, 0, 0], [0, 0, -4.5]], [[1, 0, 0, 0]] * 2, [[0.05] * 3] * 2, [0.5, 0.5], sh)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    y0 = 1 / (2 * math.sqrt(math.pi))
    np.testing.assert_allclose(P[0, 16:19], [y0 * float(np.float32(0.3)) + 0.5, y0 * float(np.float32(-0.2)) + 0.5, 0.0], rtol=1e-12)
    assert P[1, 0] == 0
    assert orc.bin32(sc, cam).count[1] == 0


# ---------------------------------------------------------------------------
# Compositing
# ---------------------------------------------------------------------------

def test_single_gaussian_closed_form(orc):
    """One Gaussian on black: C(p) = c alpha(p), T_final = 1 - alpha(p)."""
    cam = synth.tiny_camera()
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 0] = [0.4, 0.1, -0.3]
    sc = _one_scene([[0.05, -0.02, 0.1]], [_quat_z(30)], [[0.2, 0.08, 0.1]], [0.9999], sh)
    p = orc.Params64.from_scene(sc)
    P = orc.project64(p, cam)[0]
    r = orc.render64(cam, orc.project64(p, cam), orc.bin32(sc, cam))
    Q = np.array([[P[9], P[10]], [P[10], P[11]]])
    ys, xs = np.mgrid[0:128, 0:128] + 0.5
    al = _alpha_closed(xs, ys, P[4], P[5], Q, P[12])
    assert al.max() == 0.99  # the clamp is exercised
    np.testing.assert_allclose(r.image, al[..., None] * P[16:19][None, None, :], atol=1e-15)
    np.testing.assert_allclose(r.tfinal, 1 - al, atol=1e-15)
    assert r.blended == int((al > 0).sum())


def test_two_gaussians_closed_form(orc):
    """Two overlapping Gaussians: C = c1 a1 + c2 a2 (1 - a1), front one first."""
    cam = synth.tiny_camera()
    sh = np.zeros((2, 16, 3), np.float32)
    sh[0, 0] = [0.9, -0.5, 0.2]
    sh[1, 0] = [-0.4, 0.6, 0.3]
    # index 0 is farther; it must be composited second
    sc = _one_scene([[0.02, 0.0, 0.5], [-0.02, 0.01, -0.3]], [_quat_z(10), _quat_z(-40)],
                    [[0.08, 0.05, 0.05], [0.05, 0.09, 0.05]], [0.8, 0.7], sh)
    p = orc.Params64.from_scene(sc)
    P = orc.project64(p, cam)
    r = orc.render64(cam, P, orc.bin32(sc, cam))
    ys, xs = np.mgrid[0:128, 0:128] + 0.5
    al = [_alpha_closed(xs, ys, P[i, 4], P[i, 5], np.array([[P[i, 9], P[i, 10]], [P[i, 10], P[i, 11]]]), P[i, 12])
          for i in range(2)]
    a1, a2 = al[1], al[0]
    T2 = 1 - a1
    stop = T2 * (1 - a2) < 1e-4
    a2 = np.where(stop, 0, a2)
    exp = P[1, 16:19] * a1[..., None] + P[0, 16:19] * (a2 * (1 - a1))[..., None]
    np.testing.assert_allclose(r.image, exp, atol=1e-14)


def _depth_order(b, n_tiles):
    shift = 32 - 9 if False else None
    tb = 0
    while (1 << tb) < n_tiles:
        tb += 1
    drop = tb - 9 if tb >= 9 else 0
    valid = b.bin[:, 0] > 0
    g = np.nonzero(valid)[0]
    code = b.mant[g] >> drop
    return g[np.argsort(code, kind="stable")]


@pytest.mark.parametrize("seed", [0, 1])
def test_tiled_equals_bruteforce(orc, seed):
    """Tiled compositing over the culled, sorted tile lists equals a per-pixel
    walk over ALL Gaussians in the same depth order with the same rule."""
    sc, _, cams = synth.tiny_workload(seed)
    cam = cams[0]
    p = orc.Params64.from_scene(sc)
    P = orc.project64(p, cam)
    b = orc.bin32(sc, cam)
    r = orc.render64(cam, P, b, bg=(0.1, 0.2, 0.3))
    order = _depth_order(b, 64)
    img, tf, bl = orc.render64_brute(cam, P, order, bg=(0.1, 0.2, 0.3))
    assert r.blended == bl
    assert np.array_equal(r.image, img)
    assert np.array_equal(r.tfinal, tf)


# ---------------------------------------------------------------------------
# Culling, keys and sort
# ---------------------------------------------------------------------------

def _big_scene(seed, n=60):
    """Opacities 10^U(-2.6, 0): some below 1/255 (never blended), many with
    2 ln(255 o) < 9 (cull radius below 3 sigma), the rest at 3 sigma."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.4, 1.4, size=(n, 3)).astype(np.float32)
    means[:, 2] = rng.uniform(-1, 1, size=n)
    scales = np.exp(rng.normal(-2.2, 0.8, size=(n, 3))).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    opac = (10.0 ** rng.uniform(-2.6, 0.0, size=n)).astype(np.float32)
    return _one_scene(means, q, scales, opac)


def _cull_r2_64(o):
    """The cull radius^2 of the binning, in FP64 from its definition:
    min(9, 2 ln(255 o)) widened by 2^-10 relative and absolute."""
    x = 255.0 * float(np.float32(o))
    if x <= 1.0:
        return -1.0
    return min(9.0, 2.0 * math.log(x)) * (1.0 + 2.0 ** -10) + 2.0 ** -10


def test_log32_and_cull_radius(orc):
    """The binning's FP32 logarithm against the library logarithm (absolute
    error <= 3e-7 on [1, 256], exact at 1), and its cull radius^2 against the
    definition: 3 sigma for opaque Gaussians, shrinking with the opacity,
    negative (never listed) once 255 o <= 1."""
    xs = np.concatenate([np.linspace(1.0, 256.0, 4001), 1.0 + np.geomspace(1e-7, 1.0, 200),
                         np.float32(2.0) ** np.arange(0, 9)]).astype(np.float32)
    err = max(abs(orc.log32(x) - math.log(float(x))) for x in xs)
    assert err <= 3e-7, err
    assert orc.log32(1.0) == 0.0
    assert orc.cull_r2(1.0) == 9.009765625
    assert orc.cull_r2(0.5) == 9.009765625          # 2 ln(127.5) > 9
    assert orc.cull_r2(1.0 / 255.0 * 0.999) < 0.0
    assert orc.cull_r2(0.0) < 0.0
    for o in np.geomspace(1.0 / 255.0 * 1.0001, 1.0, 500):
        r64 = _cull_r2_64(o)
        assert abs(orc.cull_r2(o) - r64) <= 1e-6 + 1e-6 * r64, o
    # opacity 0.1: 2 ln(25.5) = 6.478..., well inside 3 sigma
    assert abs(orc.cull_r2(0.1) - (2 * math.log(25.5) * (1 + 2 ** -10) + 2 ** -10)) < 2e-6


@pytest.mark.parametrize("seed,tile", [(0, (16, 16)), (1, (8, 8)), (2, (16, 32)), (3, (16, 16))])
def test_scanline_equals_exact_rectangle_test(orc, seed, tile):
    """Scan-line culling lists exactly the tiles whose pixel-centre rectangle
    meets the ellipse d^2 <= r^2(o) (checked against an independent exact
    test, sandwiched between r^2 (1 -+ 1e-5) -+ 1e-6 to absorb FP32
    rounding); Gaussians with 255 o <= 1 list nothing."""
    tw, th = tile
    sc = _big_scene(seed)
    cam = synth.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = 120, 100, 60.0, 50.0  # ragged tiles
    b = orc.bin32(sc, cam, tw, th)
    TX, TY = orc.tiles_of(cam, tw, th)
    shift = orc.key_shift(TX * TY)
    rows_mode = cols_mode = small = dropped = 0
    for g in range(sc.n):
        v, mx, my, a, bb, c, det, tz = [float(x) for x in b.bin[g]]
        listed = set((b.keys_emit[b.offset[g]:b.offset[g + 1]] >> shift).tolist())
        r2 = _cull_r2_64(sc.opacities[g])
        if r2 < 0:
            dropped += 1
            assert not v and not listed
        if not v:
            assert not listed
            continue
        small += r2 < 9.0
        Q = np.linalg.inv(np.array([[a, bb], [bb, c]]))
        inner, outer = set(), set()
        for ty in range(TY):
            for tx in range(TX):
                x0, x1 = tx * tw + 0.5, min((tx + 1) * tw, cam.width) - 0.5
                y0, y1 = ty * th + 0.5, min((ty + 1) * th, cam.height) - 0.5
                x1 = (tx + 1) * tw - 0.5
                y1 = (ty + 1) * th - 0.5
                if _rect_meets_ellipse(mx, my, Q, r2 * (1 - 1e-5) - 1e-6, x0, x1, y0, y1):
                    inner.add(ty * TX + tx)
                if _rect_meets_ellipse(mx, my, Q, r2 * (1 + 1e-5) + 1e-6, x0, x1, y0, y1):
                    outer.add(ty * TX + tx)
        assert inner <= listed <= outer, g
        assert len(listed) == b.count[g]
        ey, ex = math.sqrt(r2 * c), math.sqrt(r2 * a)
        if len(listed) > 1:
            if (my + ey) - (my - ey) < (mx + ex) - (mx - ex):
                rows_mode += 1
            else:
                cols_mode += 1
    assert rows_mode > 0 and cols_mode > 0
    assert small > 5 and dropped > 0


def test_no_false_negatives_against_raster_rule(orc):
    """Every pixel where the FP64 rule (d^2 <= 9 and o exp(-d^2/2) >= 1/255)
    holds lies in a listed tile."""
    sc, _, cams = synth.tiny_workload(0)
    cam = cams[0]
    b = orc.bin32(sc, cam)
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    shift = orc.key_shift(64)
    ys, xs = np.mgrid[0:128, 0:128] + 0.5
    tiles_px = (np.mgrid[0:128, 0:128][0] // 16) * 8 + (np.mgrid[0:128, 0:128][1] // 16)
    for g in range(sc.n):
        if not P[g, 0]:
            continue
        dx, dy = xs - P[g, 4], ys - P[g, 5]
        d2 = P[g, 9] * dx * dx + 2 * P[g, 10] * dx * dy + P[g, 11] * dy * dy
        alpha = P[g, 12] * np.exp(-0.5 * d2)
        need = set(np.unique(tiles_px[(d2 <= 9.0) & (alpha >= 1.0 / 255.0)]).tolist())
        listed = set((b.keys_emit[b.offset[g]:b.offset[g + 1]] >> shift).tolist())
        assert need <= listed, g


def test_keys_layout_and_stable_sort(orc):
    """Keys: tile id in the top ceil(log2 tiles) bits, depth code
    (2 z + 1)/(z + 1) mantissa bits below; the sort equals numpy's stable
    argsort; ranges delimit each tile."""
    sc, _, cams = synth.tiny_workload(1)
    cam = cams[0]
    b = orc.bin32(sc, cam)
    shift = orc.key_shift(64)
    assert shift == 23
    tz = b.bin[:, 7].astype(np.float32)
    q = ((np.float32(2) * tz + np.float32(1)) / (tz + np.float32(1))).astype(np.float32)
    mant = q.view(np.uint32) & np.uint32(0x7FFFFF)
    g = b.gidx_emit
    np.testing.assert_array_equal(b.keys_emit & np.uint32(0x7FFFFF), mant[g])
    perm = np.argsort(b.keys_emit, kind="stable")
    np.testing.assert_array_equal(b.keys, b.keys_emit[perm])
    np.testing.assert_array_equal(b.gidx, b.gidx_emit[perm])
    for t in range(64):
        s, e = b.ranges[t]
        assert np.all((b.keys[s:e] >> shift) == t)
        # depth order within the tile
        assert np.all(np.diff(tz[b.gidx[s:e]]) >= -1e-6 * tz[b.gidx[s:e]][1:]) or e - s < 2
    assert b.ranges[:, 1].max() == b.K


def test_paper_key_bit_budget():
    """At 1080p with 16x16 tiles the key keeps at most 14 tile bits and at
    least 18 depth bits (Sec. 4.4)."""
    from oracle import oracle as orc_mod
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    f = facts["key_bits_1080p_16x16"]
    tiles = ((1920 + 15) // 16) * ((1080 + 15) // 16)
    tb = orc_mod.tile_bits(tiles)
    assert tb <= f["max_tile_bits"]
    assert 32 - tb >= f["min_depth_bits"]
    # large depth saturates the code instead of wrapping
    assert orc_mod.key_shift(tiles) == 32 - tb


# ---------------------------------------------------------------------------
# Gradients by finite differences
# ---------------------------------------------------------------------------

def _fd_scene():
    rng = np.random.default_rng(11)
    n = 12
    means = rng.uniform(-0.3, 0.3, size=(n, 3)).astype(np.float32)
    means[0] = [1.5, 0.1, 0.0]   # |x/z| beyond the 1.3x FOV clamp
    scales = np.exp(rng.normal(-2.0, 0.3, size=(n, 3))).astype(np.float32)
    scales[0] = [0.5, 0.3, 0.4]
    q = rng.normal(size=(n, 4)).astype(np.float32)
    op = (1 / (1 + np.exp(-rng.normal(0, 1, size=n)))).astype(np.float32)
    op[3] = 0.9995             # alpha clamped at 0.99 near the centre
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0] = rng.normal(0, 0.8, size=(n, 3))
    sh[:, 1:] = rng.normal(0, 0.3, size=(n, 15, 3))
    sc = _one_scene(means, q, scales, op, sh)
    cam = synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 4], np.float32), 60.0, 60.0, 16.0, 16.0, 32, 32)
    return sc, cam


def test_raster_backward_fd(orc):
    """Compositing backward (dL/d mean2D, conic, opacity, colour) against
    central differences of the FP64 render under a fixed tile order."""
    sc, cam = _fd_scene()
    P = orc.project64(orc.Params64.from_scene(sc), cam)
    b = orc.bin32(sc, cam)
    rng = np.random.default_rng(5)
    w = rng.normal(size=(32, 32, 3))
    base = orc.render64(cam, P, b, bg=(0.2, 0.1, 0.3), margin=1e-3)
    g2 = orc.raster_bwd64(cam, P, b, w, bg=(0.2, 0.1, 0.3))
    cols = [4, 5, 9, 10, 11, 12, 16, 17, 18]
    h = 1e-7
    checked = 0
    for g in range(sc.n):
        if base.unstable_g[g] or not P[g, 0]:
            continue
        for j, col in enumerate(cols):
            Pp, Pm = P.copy(), P.copy()
            Pp[g, col] += h
            Pm[g, col] -= h
            rp = orc.render64(cam, Pp, b, bg=(0.2, 0.1, 0.3))
            rm = orc.render64(cam, Pm, b, bg=(0.2, 0.1, 0.3))
            if rp.blended != rm.blended or not np.array_equal(rp.nlast, rm.nlast):
                continue
            fd = ((rp.image - rm.image) * w).sum() / (2 * h)
            assert g2[g, j] == pytest.approx(fd, rel=1e-5, abs=1e-6), (g, j)
            checked += 1
    assert checked > 60


def test_full_backward_fd(orc):
    """Projection + compositing backward in theta = (mean, quat, log-scale,
    logit-opacity, SH) against central differences (FP64, fixed tile order),
    covering the FOV clamp, the alpha clamp and the colour clamp."""
    sc, cam = _fd_scene()
    p = orc.Params64.from_scene(sc)
    P = orc.project64(p, cam)
    b = orc.bin32(sc, cam)
    rng = np.random.default_rng(6)
    w = rng.normal(size=(32, 32, 3))
    base = orc.render64(cam, P, b, margin=1e-3)
    g2 = orc.raster_bwd64(cam, P, b, w)
    grad = orc.project_bwd64(p, cam, P, g2)
    theta = p.theta()
    h = 1e-6
    checked = 0
    scale = np.abs(grad).max()
    for g in range(sc.n):
        if base.unstable_g[g]:
            continue
        for j in range(59):
            tp, tm = theta.copy(), theta.copy()
            tp[g, j] += h
            tm[g, j] -= h
            rp = orc.render64(cam, orc.project64(orc.Params64.from_theta(tp), cam), b)
            rm = orc.render64(cam, orc.project64(orc.Params64.from_theta(tm), cam), b)
            if rp.blended != rm.blended or not np.array_equal(rp.nlast, rm.nlast):
                continue
            fd = ((rp.image - rm.image) * w).sum() / (2 * h)
            assert grad[g, j] == pytest.approx(fd, rel=1e-4, abs=1e-7 * scale), (g, j)
            checked += 1
    assert checked > 400
    # the clamped-FOV Gaussian and the clamped-alpha Gaussian were exercised
    assert abs(grad[0, :3]).sum() > 0 and abs(grad[3, 10]) >= 0


# ---------------------------------------------------------------------------
# Adam, L1 and the whole step
# ---------------------------------------------------------------------------

def test_adam_step1_closed_form(orc):
    """First Adam step: theta1 = theta0 - lr g / (|g| + eps), per group."""
    rng = np.random.default_rng(2)
    th = rng.normal(size=(7, 59))
    g = rng.normal(size=(7, 59)) * 10.0 ** rng.uniform(-8, 2, size=(7, 59))
    g[0, :5] = 0
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    grp = np.array([0] * 3 + [1] * 4 + [2] * 3 + [3] + [4] * 3 + [5] * 45)
    th1, m, v = th.copy(), np.zeros_like(th), np.zeros_like(th)
    orc.adam64(th1, m, v, g.copy(), lr, 1)
    np.testing.assert_allclose(th1, th - lr[grp][None, :] * g / (np.abs(g) + 1e-15), rtol=1e-12, atol=1e-15)


def test_adam_five_steps_equal_torch_adam(orc):
    """Five Adam steps with changing gradients equal torch.optim.Adam (FP64,
    one parameter group per learning-rate group): bias corrections and the
    moment recurrences past the first step."""
    import torch
    rng = np.random.default_rng(5)
    th0 = rng.normal(size=(6, 59))
    grads = [rng.normal(size=(6, 59)) * 10.0 ** rng.uniform(-6, 1, size=(6, 59)) for _ in range(5)]
    lr = np.array([1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3])
    grp = np.array([0] * 3 + [1] * 4 + [2] * 3 + [3] + [4] * 3 + [5] * 45)
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    for t, g in enumerate(grads, 1):
        orc.adam64(th, m, v, g.copy(), lr, t)
    cols = [np.nonzero(grp == k)[0] for k in range(6)]
    params = [torch.tensor(th0[:, c], dtype=torch.float64, requires_grad=True) for c in cols]
    opt = torch.optim.Adam([{"params": [p], "lr": float(lr[k])} for k, p in enumerate(params)],
                           betas=(0.9, 0.999), eps=1e-15)
    for g in grads:
        for k, p in enumerate(params):
            p.grad = torch.tensor(g[:, cols[k]], dtype=torch.float64)
        opt.step()
    for k, p in enumerate(params):
        np.testing.assert_allclose(th[:, cols[k]], p.detach().numpy(), rtol=1e-10, atol=1e-14)


def test_l1_gradient_closed_form(orc):
    a = np.array([[[0.5, 0.2, 0.0]]]); t = np.array([[[0.4, 0.2, 0.1]]])
    loss, (g,) = orc.l1_loss_grad([a], [t])
    assert loss == pytest.approx(0.2 / 3)
    np.testing.assert_array_equal(g, np.array([[[1, 0, -1]]]) / 3)


def test_step_decreases_loss(orc):
    """A small Adam step along the oracle's gradient lowers the L1 loss."""
    sc, tsc, cams = synth.tiny_workload(0)
    cam = cams[0]
    tgt = orc.render64(cam, orc.project64(orc.Params64.from_scene(tsc), cam), orc.bin32(tsc, cam)).image
    res = orc.step(sc, cams, [tgt], [2e-5] * 6)
    new = res.params
    sc2 = synth.Scene(new.means.astype(np.float32), new.quats.astype(np.float32), new.scales.astype(np.float32),
                      new.opacities.astype(np.float32), new.sh.reshape(-1, 16, 3).astype(np.float32))
    res2 = orc.step(sc2, cams, [tgt], [2e-5] * 6, grad_only=True)
    assert res2.loss < res.loss
