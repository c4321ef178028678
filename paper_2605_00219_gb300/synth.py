"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random scenes and builds camera poses.  It holds none
of the method's arithmetic (no projection, culling, compositing, gradients or
optimiser), so both the CUDA path and the CPU oracle can take their inputs
from it.

Parameters are stored the way the step consumes them (Sec. 4.3 of the paper
keeps scale and opacity in activated form): per-axis scales s > 0 and opacity
o in (0, 1), both drawn in log / logit space.  SH coefficients are degree 3,
16 x 3 per Gaussian.

The paper trains on Mip-NeRF 360 scenes (about 3M Gaussians after
densification, 1-2 MP views), which are not available here; the cluster
scenes below stand in for them at that scale.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    means: np.ndarray      # (n, 3) float32, world space
    quats: np.ndarray      # (n, 4) float32, (w, x, y, z), not normalised
    scales: np.ndarray     # (n, 3) float32, activated (> 0)
    opacities: np.ndarray  # (n,)   float32, activated, in (0, 1)
    sh: np.ndarray         # (n, 16, 3) float32, degree-3 SH

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.quats.copy(), self.scales.copy(),
                     self.opacities.copy(), self.sh.copy())


@dataclass
class Camera:
    R: np.ndarray          # (3, 3) float32, world -> camera rotation (x right, y down, z forward)
    t: np.ndarray          # (3,) float32, world -> camera translation
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    scene: int = 0         # index of the scene this view renders

    def pose_params(self) -> np.ndarray:
        """R (row-major 9), t (3), fx, fy, cx, cy packed as 16 float32."""
        return np.concatenate([self.R.reshape(-1), self.t.reshape(-1),
                               np.array([self.fx, self.fy, self.cx, self.cy], np.float32)]).astype(np.float32)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh(rng: np.random.Generator, n: int, dc_sigma: float, rest_sigma: float) -> np.ndarray:
    sh = np.empty((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.normal(0.0, dc_sigma, size=(n, 3))
    sh[:, 1:, :] = rng.normal(0.0, rest_sigma, size=(n, 15, 3))
    return sh


def uniform_scene(n: int, seed: int) -> Scene:
    """Tiny-scene recipe: means U[-1,1]^3, log-scales N(-3.5, 0.5) per axis,
    random unit quaternions, opacity logits N(0, 1), SH DC N(0, 0.5) and the
    higher bands N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    scales = np.exp(rng.normal(-3.5, 0.5, size=(n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n)).astype(np.float32)
    sh = _sh(rng, n, 0.5, 0.05)
    return Scene(means, quats, scales, opac, sh)


def cluster_scene(n: int, n_clusters: int, box: float, seed: int,
                  log_scale=(-4.0, 0.7), logit_opacity=(-1.0, 1.5)) -> Scene:
    """Clustered-scene recipe: means from `n_clusters` anisotropic clusters
    (centres uniform in a `box`-metre cube centred on the origin, per-cluster
    covariance diag U(0.1, 1.5) m^2 randomly rotated), log-scales
    N(-4, 0.7), opacity logits N(-1, 1.5), SH as in the tiny scene."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-box / 2, box / 2, size=(n_clusters, 3))
    var = rng.uniform(0.1, 1.5, size=(n_clusters, 3))
    rot = np.empty((n_clusters, 3, 3))
    for i in range(n_clusters):
        a = rng.normal(size=(3, 3))
        qm, rm = np.linalg.qr(a)
        rot[i] = qm * np.sign(np.diag(rm))
    which = rng.integers(0, n_clusters, size=n)
    z = rng.normal(size=(n, 3)) * np.sqrt(var[which])
    means = (np.einsum("nij,nj->ni", rot[which], z) + centres[which]).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], size=(n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(logit_opacity[0], logit_opacity[1], size=n)).astype(np.float32)
    sh = _sh(rng, n, 0.5, 0.05)
    return Scene(means, quats, scales, opac, sh)


def perturbed(scene: Scene, seed: int, mean_sigma: float = 0.02, colour_sigma: float = 0.1) -> Scene:
    """Copy of `scene` with means + N(0, mean_sigma) m and the SH DC
    coefficients (the view-independent colour) + N(0, colour_sigma)."""
    rng = np.random.default_rng(seed)
    s = scene.copy()
    s.means += rng.normal(0.0, mean_sigma, size=s.means.shape).astype(np.float32)
    s.sh[:, 0, :] += rng.normal(0.0, colour_sigma, size=(s.n, 3)).astype(np.float32)
    return s


def tiny_camera() -> Camera:
    """128 x 128 pinhole, fx = fy = 150, at (0, 0, -4) looking at the origin."""
    return Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 4], np.float32),
                  150.0, 150.0, 64.0, 64.0, 128, 128)


def look_at(eye, target, width: int, height: int, fx: float, fy: float | None = None,
            up=(0.0, 0.0, 1.0), scene: int = 0) -> Camera:
    """Pinhole camera at `eye` looking at `target` (OpenCV axes: x right,
    y down, z forward), principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-R.astype(np.float64) @ eye).astype(np.float32)
    fy = fx if fy is None else fy
    return Camera(R, t, float(fx), float(fy), width / 2.0, height / 2.0, width, height, scene)


def orbit_cameras(n_views: int, radius: float, width: int, height: int,
                  elevation_deg: float = 20.0, hfov_deg: float = 60.0,
                  centre=(0.0, 0.0, 0.0), scene: int = 0, phase_deg: float = 0.0) -> list[Camera]:
    """`n_views` cameras on a z-up orbit, evenly spaced in azimuth, looking
    at `centre`; focal length from the horizontal field of view
    (fx = W / (2 tan(hfov / 2)), 0.866 W for 60 degrees)."""
    fx = width / (2.0 * math.tan(math.radians(hfov_deg) / 2.0))
    el = math.radians(elevation_deg)
    cams = []
    for i in range(n_views):
        az = math.radians(phase_deg + 360.0 * i / n_views)
        eye = np.asarray(centre) + radius * np.array(
            [math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams.append(look_at(eye, centre, width, height, fx, scene=scene))
    return cams


# Workload presets (sizes and seeds only).
TINY_N = 2000
MID_N = 200_000
LARGE_N = 3_000_000
BATCH_RESOLUTIONS = [(1920, 1080), (1600, 1064), (1280, 720), (960, 540)]


def tiny_workload(seed: int = 0):
    """2,000 Gaussians and one 128x128 camera; target scene from seed + 1."""
    return uniform_scene(TINY_N, seed), uniform_scene(TINY_N, seed + 1), [tiny_camera()]


def mid_workload(seed: int = 0, n: int = MID_N, n_views: int = 20):
    """200k Gaussians in 64 clusters (10 m box), 1280x720, 20-view orbit at
    r = 12 m; targets from a perturbed copy."""
    sc = cluster_scene(n, 64, 10.0, seed)
    tgt = perturbed(sc, seed + 1)
    cams = orbit_cameras(n_views, 12.0, 1280, 720)
    return sc, tgt, cams


def large_scene(seed: int = 0, n: int = LARGE_N) -> Scene:
    """3M Gaussians in 256 clusters (30 m box)."""
    return cluster_scene(n, 256, 30.0, seed)


def large_views(n_views: int = 4, radius: float = 36.0, phase_deg: float = 0.0,
                resolutions=None) -> list[Camera]:
    """Orbit views at r = 36 m of the 30 m-box scene; uneven resolutions
    cycle through 1920x1080, 1600x1064, 1280x720, 960x540."""
    res = resolutions or BATCH_RESOLUTIONS
    cams = []
    for i in range(n_views):
        w, h = res[i % len(res)]
        cams += orbit_cameras(1, radius, w, h, phase_deg=phase_deg + 360.0 * i / n_views)
    return cams


def loss_images(shapes, seed: int, smooth: bool = False):
    """Rendered-image stand-ins and 8-bit RGBA references for the loss
    kernels: one (H, W, 3) float32 image in [0, 1] and one (H, W, 4) uint8
    target per (W, H).  smooth=True gives low-frequency images with flat
    regions (small window variances), otherwise uniform noise."""
    rng = np.random.default_rng(seed)
    imgs, tgts = [], []
    for (w, h) in shapes:
        if smooth:
            yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
            base = np.empty((h, w, 3))
            for c in range(3):
                fx, fy, ph = rng.uniform(0.01, 0.08), rng.uniform(0.01, 0.08), rng.uniform(0, 2 * np.pi)
                base[..., c] = 0.5 + 0.4 * np.sin(fx * xx + ph) * np.cos(fy * yy)
            img = np.clip(base + rng.normal(0, 0.01, base.shape), 0, 1)
            img[: h // 3, : w // 3] = 0.25            # a flat block
            tgt = np.clip(base + rng.normal(0, 0.03, base.shape), 0, 1)
        else:
            img = rng.uniform(0, 1, (h, w, 3))
            tgt = rng.uniform(0, 1, (h, w, 3))
        t8 = np.empty((h, w, 4), np.uint8)
        t8[..., :3] = np.rint(tgt * 255).astype(np.uint8)
        t8[..., 3] = rng.integers(0, 256, (h, w), dtype=np.uint8)
        imgs.append(img.astype(np.float32))
        tgts.append(t8)
    return imgs, tgts


MULTI_SIZES = (500_000, 500_000, 750_000, 750_000, 1_000_000, 1_250_000, 1_250_000, 6_000_000)


def multi_scene_workload(sizes=MULTI_SIZES, radius: float = 36.0):
    """Eight clustered scenes (seeds 0-7, 30 m box, about one cluster per
    12,000 Gaussians) with two views each: even scenes 1920x1080 + 960x540,
    odd scenes 1280x720 + 1600x900, on the r = 36 m orbit."""
    scenes, cams = [], []
    for k, n in enumerate(sizes):
        scenes.append(cluster_scene(n, max(16, n // 12000), 30.0, seed=k))
        res = [(1920, 1080), (960, 540)] if k % 2 == 0 else [(1280, 720), (1600, 900)]
        for i, (w, h) in enumerate(res):
            cams += orbit_cameras(1, radius, w, h, scene=k, phase_deg=45.0 * k + 60.0 * i)
    return scenes, cams
