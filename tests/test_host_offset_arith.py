"""FP32 arithmetic of the raster kernels' pixel offset and exponent, emulated
with numpy float32 (each operation rounded to nearest, as the kernels'
__fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn do) against float64.

The raster kernels stage a Gaussian's mean relative to the tile's first pixel
o, rounded once, m_t = (m_hi - o) + m_lo, and form a pixel's offset as one
subtraction from its tile-relative centre.  These tests check the error bound
the kernels' comments state (about one ulp of the tile-relative mean), that
it is of the same order as the former (p - m_hi) - m_lo, and that the
exponent's two groupings agree to a few ulp.
"""
import numpy as np

f32 = np.float32


def _ulp(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


def _cases(seed, n=200_000):
    rng = np.random.default_rng(seed)
    # means over a 1080p-wide view and beyond it, residuals below half an ulp
    m_hi = rng.uniform(-200.0, 2200.0, n).astype(f32)
    m_lo = (rng.uniform(-0.5, 0.5, n) * _ulp(m_hi)).astype(f32)
    # a 16-px tile within 300 px of the mean, and a pixel centre inside it
    o = (np.floor((m_hi.astype(np.float64) + rng.uniform(-300, 300, n)) / 16) * 16).astype(np.int64)
    px = rng.integers(0, 16, n)
    return m_hi, m_lo, o, px


def test_tile_relative_offset_error_bound():
    m_hi, m_lo, o, px = _cases(0)
    pc_rel = (px.astype(f32) + f32(0.5))                         # exact
    m_t = (m_hi - o.astype(f32)) + m_lo                          # two float32 roundings
    dx_new = (pc_rel - m_t).astype(np.float64)
    truth = (o + px + 0.5) - (m_hi.astype(np.float64) + m_lo.astype(np.float64))
    err = np.abs(dx_new - truth)
    rel_mean = np.abs(m_hi.astype(np.float64) - o)
    bound = _ulp(rel_mean) + 0.5 * _ulp(truth) + 1e-12
    assert np.all(err <= bound), float((err / bound).max())
    # within 16 px of the tile the error stays near 1e-6 px
    near = rel_mean <= 16.0
    assert err[near].max() <= 2.5e-6


def test_tile_relative_offset_matches_former_form():
    m_hi, m_lo, o, px = _cases(1)
    pc_abs = (o.astype(f32) + px.astype(f32)) + f32(0.5)         # exact below 2^23
    dx_old = ((pc_abs - m_hi) - m_lo).astype(np.float64)
    dx_new = ((px.astype(f32) + f32(0.5)) - ((m_hi - o.astype(f32)) + m_lo)).astype(np.float64)
    truth = (o + px + 0.5) - (m_hi.astype(np.float64) + m_lo.astype(np.float64))
    e_old = np.abs(dx_old - truth)
    e_new = np.abs(dx_new - truth)
    # the same order of error: neither form is more than a few ulp of the
    # offset's scale worse than the other on these cases
    scale = _ulp(np.abs(truth) + 16.0)
    assert e_new.max() <= 2.0 * scale.max()
    assert e_old.max() <= 2.0 * scale.max()
    assert np.mean(e_new) <= 4.0 * np.mean(e_old) + 1e-9


def test_exponent_groupings_agree():
    rng = np.random.default_rng(2)
    n = 200_000
    # conics of footprints 0.5-50 px across, prescaled to base 2 (A, C < 0)
    sx = rng.uniform(0.5, 50.0, n)
    sy = rng.uniform(0.5, 50.0, n)
    rho = rng.uniform(-0.9, 0.9, n)
    det = (sx * sy) ** 2 * (1 - rho ** 2)
    ca, cb, cc = (sy ** 2) / det, -(rho * sx * sy) / det, (sx ** 2) / det
    k = -1.4426950408889634
    A, B, C = (f32(0.5 * k) * ca.astype(f32)), (f32(k) * cb.astype(f32)), (f32(0.5 * k) * cc.astype(f32))
    dx = (rng.uniform(-3, 3, n) * sx).astype(f32)
    dy = (rng.uniform(-3, 3, n) * sy).astype(f32)

    def fma(a, b, c):   # one rounding of a*b + c
        return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)

    old = fma(dx, fma(A, dx, B * dy), (C * dy) * dy)
    new = fma(dy, fma(C, dy, B * dx), (A * dx) * dx)
    truth = (A.astype(np.float64) * dx.astype(np.float64) ** 2 + B.astype(np.float64) * dx.astype(np.float64)
             * dy.astype(np.float64) + C.astype(np.float64) * dy.astype(np.float64) ** 2)
    # the quadratic form is negative definite: no cancellation beyond a few ulp
    tol = 8.0 * _ulp(np.abs(A * dx * dx) + np.abs(B * dx * dy) + np.abs(C * dy * dy))
    assert np.all(np.abs(new.astype(np.float64) - truth) <= tol)
    assert np.all(np.abs(old.astype(np.float64) - truth) <= tol)


def test_opacity_test_before_clamp_is_the_same_decision():
    # alpha = min(0.99, o G) >= 1/255 exactly when o G >= 1/255, for finite o G
    rng = np.random.default_rng(3)
    araw = np.concatenate([rng.uniform(0, 1.5, 100_000), np.float32(1 / 255) + np.arange(-64, 64) * 1e-9]).astype(f32)
    amin = f32(1.0 / 255.0)
    assert np.array_equal(np.minimum(f32(0.99), araw) >= amin, araw >= amin)
