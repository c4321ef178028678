"""Central finite differences of the FP64 oracle on sampled Gaussians (test
infrastructure for the gradient tests; no GPU code).

The step is differentiated with its tile lists and depth order held fixed
(Sec. 4.2: the backward runs over the lists the forward used), so each
evaluation perturbs one parameter of one Gaussian g in theta = (mean,
quaternion, log-scale, logit-opacity, SH), re-projects g alone, and
re-renders only the tiles that list it, on a crop of the view that covers
them.  The loss is a fixed weighting of the rendered pixels, sum w * C.

An evaluation pair (theta +- h) is skipped only when a discrete decision of
the forward differs between its two ends, since a central difference across
a jump or a kink is not a derivative:
- the blended pair count and every crop pixel's last blended list position
  (covers the stop test T (1 - alpha) < 1e-4 of every pair behind g);
- the pixels where g itself contributes (d^2 <= 9 and alpha >= 1/255), where
  its alpha is clamped at 0.99, its colour channels clamped at 0, and whether
  its direction lies beyond the field-of-view clamp of the Jacobian.
"""
from __future__ import annotations

import copy

import numpy as np

H_STEP = 1e-3
# mean x, y, z; quaternion w, y; log-scale x, z; logit-opacity; SH degree 0
# (red); a degree-2 and a degree-3 coefficient
COMPONENTS = (0, 1, 2, 3, 5, 7, 9, 10, 11, 20, 47)


class CropView:
    """One view of one Gaussian g: the tiles that list g, on the crop of the
    image that covers them, with every Gaussian those tiles list."""

    def __init__(self, orc, cam, b, P, w, g):
        TX = (cam.width + 15) // 16
        shift = orc.key_shift(b.ranges.shape[0])
        tiles = np.unique(b.keys_emit[b.offset[g]:b.offset[g + 1]] >> shift).astype(np.int64)
        tx, ty = tiles % TX, tiles // TX
        tx0, ty0 = int(tx.min()), int(ty.min())
        self.x0, self.y0 = 16 * tx0, 16 * ty0
        TXc, TYc = int(tx.max()) - tx0 + 1, int(ty.max()) - ty0 + 1
        Wc = min(16 * (tx0 + TXc), cam.width) - self.x0
        Hc = min(16 * (ty0 + TYc), cam.height) - self.y0
        ents = [b.gidx[b.ranges[t, 0]:b.ranges[t, 1]].astype(np.int64) for t in tiles]
        glob = np.unique(np.concatenate(ents))
        ranges = np.zeros((TXc * TYc, 2), np.int64)
        start = 0
        for t, e in zip(tiles, ents):
            lt = (int(t // TX) - ty0) * TXc + (int(t % TX) - tx0)
            ranges[lt] = (start, start + e.size)
            start += e.size
        gl = np.searchsorted(glob, np.concatenate(ents)).astype(np.uint32)
        z = np.zeros(1, np.uint32)
        self.bin = orc.Binning(z, None, z, None, z, z, z, gl, z, ranges)
        self.P = P[glob].copy()
        self.P[:, 4] -= self.x0
        self.P[:, 5] -= self.y0
        self.gl = int(np.searchsorted(glob, g))
        self.base_row = self.P[self.gl].copy()
        self.cam_full = cam
        self.cam = copy.copy(cam)
        self.cam.width, self.cam.height = Wc, Hc
        self.w = w[self.y0:self.y0 + Hc, self.x0:self.x0 + Wc]
        tp = (np.arange(Hc)[:, None] // 16) * TXc + (np.arange(Wc)[None, :] // 16)
        listed = np.zeros(TXc * TYc, bool)
        listed[ranges[:, 1] > ranges[:, 0]] = True
        self.mask = listed[tp]
        ys, xs = np.nonzero(self.mask)
        self.px, self.py = xs + 0.5, ys + 0.5
        self.limx = 1.3 * 0.5 * cam.width / cam.fx
        self.limy = 1.3 * 0.5 * cam.height / cam.fy
        self.orc = orc

    def evaluate(self, pp):
        """(sum w C over the listed tiles, signature of discrete decisions)
        with g's parameters replaced by the one-Gaussian Params64 pp."""
        orc = self.orc
        Pg = orc.project64(pp, self.cam_full)[0]
        row = Pg.copy()
        row[4] -= self.x0
        row[5] -= self.y0
        self.P[self.gl] = row
        r = orc.render64(self.cam, self.P, self.bin)
        self.P[self.gl] = self.base_row
        value = float((r.image * self.w)[self.mask].sum())
        if Pg[0]:
            dx, dy = self.px - row[4], self.py - row[5]
            d2 = row[9] * dx * dx + 2 * row[10] * dx * dy + row[11] * dy * dy
            araw = row[12] * np.exp(-0.5 * d2)
            inside = d2 <= 9.0
            contrib = inside & (np.minimum(araw, 0.99) >= 1.0 / 255.0)
            clamp = inside & (araw > 0.99)
            fov = (abs(Pg[1] / Pg[3]) > self.limx, abs(Pg[2] / Pg[3]) > self.limy)
            own = (contrib.tobytes(), clamp.tobytes(), tuple(Pg[13:16] < 0), fov)
        else:
            own = None
        return value, (r.blended, r.nlast[self.mask].tobytes(), own)


def fd_check(orc, scene, views, picks, grad_theta, rms, components=COMPONENTS, h=H_STEP):
    """Central differences for Gaussians `picks` of `scene` over `views`
    (list of (cam, binning, FP64 projection, weights)), against grad_theta
    (n x 59, d/d theta).

    The derivative is the fourth-order central stencil whose outer points are
    theta +- h and inner points theta +- h/2,
        D = (8 (L(+h/2) - L(-h/2)) - (L(+h) - L(-h))) / (6 h).
    The two-point difference (L(+h) - L(-h)) / (2 h) carries a truncation
    error of h^2/6 times the third derivative, which reaches 1e-2 relative
    for footprints below a pixel (it falls 4x per halving of h); the
    stencil's leading error is of order h^4.  An evaluation is skipped when a
    discrete decision differs between any of the four points.
    Error = |g - D| / max(|D|, rms[j]): relative to D, with an absolute
    floor of (bound) x the component's RMS, as in every gradient parity test
    of the step.  Returns a dict: checked,
    skipped, the largest error and the worst (g, component, gradient, D),
    and the largest error of the two-point difference at h, for reference."""
    p = orc.Params64.from_scene(scene)
    theta = p.theta()
    checked = skipped = 0
    worst, worst2 = (0.0, None), 0.0
    for g in picks:
        crops = [CropView(orc, c, b, P, w, int(g)) for c, b, P, w in views if b.count[g] > 0]
        for j in components:
            vals, sigs = [], []
            for step in (h, h / 2, -h / 2, -h):
                t = theta[g].copy()
                t[j] += step
                ev = [cv.evaluate(orc.Params64.from_theta(t[None, :])) for cv in crops]
                vals.append(sum(v for v, _ in ev))
                sigs.append([s for _, s in ev])
            if any(s != sigs[0] for s in sigs[1:]):
                skipped += 1
                continue
            lp, lph, lmh, lm = vals
            d4 = (8.0 * (lph - lmh) - (lp - lm)) / (6.0 * h)
            d2 = (lp - lm) / (2.0 * h)
            floor = rms[j]
            err = abs(grad_theta[g, j] - d4) / max(abs(d4), floor)
            worst2 = max(worst2, abs(grad_theta[g, j] - d2) / max(abs(d2), floor))
            checked += 1
            if err > worst[0]:
                worst = (err, (int(g), j, float(grad_theta[g, j]), d4))
    return {"checked": checked, "skipped": skipped, "max_err": float(worst[0]), "worst": worst[1],
            "two_point_max_err": float(worst2)}


def theta_grads(p, dstored):
    """d/d theta from gradients with respect to the stored (activated)
    parameters (n x 59: mean, quaternion, scales, opacity, SH): scales and
    opacity through s = exp(theta_s) and o = sigmoid(theta_o)."""
    g = np.array(dstored, np.float64, copy=True)
    g[:, 7:10] *= p.scales
    g[:, 10] *= p.opacities * (1 - p.opacities)
    return g
