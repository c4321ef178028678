"""Pins of the oracle's L1 + SSIM loss and gradient (no GPU)."""
import numpy as np
import pytest


def test_ssim_constant_images_closed_form(orc):
    """Constant images a, b: away from the border (window inside the image)
    SSIM = (2ab + C1) / (a^2 + b^2 + C1) per channel."""
    H, W = 40, 48
    x = np.full((H, W, 3), 0.6)
    y = np.full((H, W, 3), 0.25)
    g = orc.ssim_window()
    from scipy.ndimage import correlate1d

    def f(img):
        return correlate1d(correlate1d(img, g, axis=0, mode="constant"), g, axis=1, mode="constant")
    mx, my = f(x[..., 0]), f(y[..., 0])
    s = (2 * mx * my + orc.SSIM_C1) * (2 * (f(x[..., 0] * y[..., 0]) - mx * my) + orc.SSIM_C2) / (
        (mx * mx + my * my + orc.SSIM_C1) * (f(x[..., 0] ** 2) - mx * mx + f(y[..., 0] ** 2) - my * my + orc.SSIM_C2))
    expect = (2 * 0.6 * 0.25 + orc.SSIM_C1) / (0.6 ** 2 + 0.25 ** 2 + orc.SSIM_C1)
    assert s[10:-10, 10:-10] == pytest.approx(expect, rel=1e-12)
    # the loss with lam = 1 averages exactly these maps
    loss, _ = orc.l1_ssim_loss_grad([x], [y], lam=1.0)
    assert loss == pytest.approx(1 - s.mean(), rel=1e-12)


def test_ssim_identical_images():
    """x = y: SSIM = 1 everywhere and the SSIM term has zero gradient."""
    from oracle import oracle as orc
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(20, 24, 3))
    loss, (g,) = orc.l1_ssim_loss_grad([x], [x.copy()], lam=1.0)
    assert loss == pytest.approx(0.0, abs=1e-12)
    assert np.abs(g).max() < 1e-12


def test_ssim_symmetric():
    from oracle import oracle as orc
    rng = np.random.default_rng(1)
    x, y = rng.uniform(size=(2, 16, 18, 3))
    l1, _ = orc.l1_ssim_loss_grad([x], [y], lam=1.0)
    l2, _ = orc.l1_ssim_loss_grad([y], [x], lam=1.0)
    assert l1 == pytest.approx(l2, rel=1e-13)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_l1_ssim_gradient_fd(orc, lam):
    """Analytic gradient against central differences (two views, border
    pixels included, zero padding)."""
    rng = np.random.default_rng(2)
    xs = [rng.uniform(0.1, 0.9, size=(13, 11, 3)), rng.uniform(0.1, 0.9, size=(9, 15, 3))]
    ys = [rng.uniform(0.1, 0.9, size=x.shape) for x in xs]
    loss, grads = orc.l1_ssim_loss_grad(xs, ys, lam=lam)
    h = 1e-6
    for v in range(2):
        for idx in [(0, 0, 0), (6, 5, 1), (12, 10, 2), (3, 0, 2), (8, 14, 0)][: (5 if v else 3)]:
            if v == 0 and (idx[0] >= 13 or idx[1] >= 11):
                continue
            if v == 1 and (idx[0] >= 9 or idx[1] >= 15):
                continue
            xp = [x.copy() for x in xs]
            xm = [x.copy() for x in xs]
            xp[v][idx] += h
            xm[v][idx] -= h
            fd = (orc.l1_ssim_loss_grad(xp, ys, lam)[0] - orc.l1_ssim_loss_grad(xm, ys, lam)[0]) / (2 * h)
            assert grads[v][idx] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_rgba8_target():
    from oracle import oracle as orc
    t = np.array([[[255, 0, 51, 7]]], np.uint8)
    np.testing.assert_allclose(orc.rgba8_to_float(t), [[[1.0, 0.0, 0.2]]])


def test_loss_equals_direct_window_sums():
    """The loss against SSIM written out with plain loops: per pixel and
    channel, sums over the 11x11 window of w_a w_b times x, y, x^2, y^2, xy
    with zero outside the image, w_k = exp(-(k - 5)^2 / (2 * 1.5^2)) / sum;
    SSIM = (2 mx my + C1)(2 cov + C2) / ((mx^2 + my^2 + C1)(vx + vy + C2));
    the mean over 3 x all pixels of two ragged views."""
    import math
    from oracle import oracle as orc
    rng = np.random.default_rng(7)
    xs = [rng.uniform(0, 1, size=(9, 7, 3)), rng.uniform(0, 1, size=(5, 12, 3))]
    ys = [rng.uniform(0, 1, size=x.shape) for x in xs]
    e = [math.exp(-(k - 5) ** 2 / (2 * 1.5 ** 2)) for k in range(11)]
    w = [v / sum(e) for v in e]
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim_sum = l1_sum = 0.0
    cnt = 0
    for x, y in zip(xs, ys):
        H, W, _ = x.shape
        for c in range(3):
            for i in range(H):
                for j in range(W):
                    m = [0.0] * 5
                    for a in range(11):
                        for b in range(11):
                            ii, jj = i + a - 5, j + b - 5
                            if 0 <= ii < H and 0 <= jj < W:
                                ww = w[a] * w[b]
                                xv, yv = float(x[ii, jj, c]), float(y[ii, jj, c])
                                m[0] += ww * xv
                                m[1] += ww * yv
                                m[2] += ww * xv * xv
                                m[3] += ww * yv * yv
                                m[4] += ww * xv * yv
                    mx, my = m[0], m[1]
                    vx, vy, cov = m[2] - mx * mx, m[3] - my * my, m[4] - mx * my
                    ssim_sum += (2 * mx * my + C1) * (2 * cov + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
                    l1_sum += abs(float(x[i, j, c]) - float(y[i, j, c]))
                    cnt += 1
    for lam in (0.0, 0.2, 1.0):
        loss, _ = orc.l1_ssim_loss_grad(xs, ys, lam)
        assert loss == pytest.approx((1 - lam) * l1_sum / cnt + lam * (1 - ssim_sum / cnt), rel=1e-12)


def test_alpha_mask_of_ones_is_the_unmasked_loss(orc):
    rng = np.random.default_rng(5)
    x, y = rng.uniform(size=(2, 14, 17, 3))
    l0, (g0,) = orc.l1_ssim_loss_grad([x], [y], 0.2)
    l1, (g1,) = orc.l1_ssim_loss_grad([x], [y], 0.2, masks=[np.ones((14, 17))])
    assert l1 == l0 and np.array_equal(g1, g0)


def test_alpha_mask_of_zeros_gives_no_loss(orc):
    """Everything masked out: both masked images are 0, SSIM of two zero
    images is 1 and the L1 term 0, so the loss and its gradient vanish."""
    rng = np.random.default_rng(6)
    x, y = rng.uniform(size=(2, 12, 12, 3))
    loss, (g,) = orc.l1_ssim_loss_grad([x], [y], 0.2, masks=[np.zeros((12, 12))])
    assert loss == pytest.approx(0.0, abs=1e-15) and not g.any()


def test_alpha_mask_excludes_masked_pixels(orc):
    """A 0/1 mask: the render's values under m = 0 change neither the loss
    nor any gradient, and their own gradient is 0."""
    rng = np.random.default_rng(7)
    x, y = rng.uniform(size=(2, 16, 15, 3))
    m = (rng.uniform(size=(16, 15)) > 0.4).astype(float)
    l0, (g0,) = orc.l1_ssim_loss_grad([x], [y], 0.2, masks=[m])
    x2 = x.copy()
    x2[m == 0] = rng.uniform(size=((m == 0).sum(), 3))
    l2, (g2,) = orc.l1_ssim_loss_grad([x2], [y], 0.2, masks=[m])
    assert l2 == pytest.approx(l0, rel=1e-13)
    assert np.allclose(g2, g0, rtol=0, atol=1e-15)
    assert not g0[m == 0].any()


def test_alpha_masked_gradient_fd(orc):
    """Fractional mask: the analytic gradient (with the factor m) against
    central differences of the masked loss."""
    rng = np.random.default_rng(8)
    x = rng.uniform(0.1, 0.9, size=(11, 13, 3))
    y = rng.uniform(0.1, 0.9, size=x.shape)
    m = rng.uniform(size=(11, 13))
    m[0, 0] = 0.0
    _, (g,) = orc.l1_ssim_loss_grad([x], [y], 0.2, masks=[m])
    h = 1e-6
    for idx in [(0, 0, 0), (5, 6, 1), (10, 12, 2), (3, 0, 2), (7, 9, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (orc.l1_ssim_loss_grad([xp], [y], 0.2, masks=[m])[0] -
              orc.l1_ssim_loss_grad([xm], [y], 0.2, masks=[m])[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), idx
