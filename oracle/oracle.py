"""FP64 CPU oracle of one 3D Gaussian Splatting training step (VkSplat,
arxiv 2605.00219) -- Python side.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference arm are the only users.  It imports nothing from the
CUDA package; inputs come as plain numpy arrays (the seeded generators live in
a module of their own).

The heavy loops are plain C in gs_oracle.c (built here with gcc,
-ffp-contract=off); this file strings them together in the order of the
paper's training iteration (Sec. 2, Sec. 4):

  project (FP64) -> FP32 binning: count, emit keys, stable sort, tile ranges
  (Sec. 4.1, Sec. 4.4) -> compositing (FP64) -> L1 loss gradient (Sec. 4.5,
  L1 term) -> compositing backward (Sec. 4.2) -> projection backward and Adam
  in log-scale / logit-opacity space (Sec. 4.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

PSTRIDE = 24
NTHETA = 59

_lib = None


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into a shared library (gcc, FP contraction off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-fexcess-precision=standard", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcCam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32)]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        cam = ctypes.POINTER(OrcCam)
        L.orc_log32.argtypes = [ctypes.c_float]
        L.orc_log32.restype = ctypes.c_float
        L.orc_cull_r2.argtypes = [ctypes.c_float]
        L.orc_cull_r2.restype = ctypes.c_float
        L.orc_bin32_count.argtypes = [i64, vp, vp, vp, vp, cam, vp, vp, vp]
        L.orc_bin32_count.restype = None
        L.orc_bin32_emit.argtypes = [i64, vp, vp, vp, vp, cam, vp, vp, vp]
        L.orc_bin32_emit.restype = i64
        L.orc_stable_sort.argtypes = [i64, vp, vp]
        L.orc_stable_sort.restype = None
        L.orc_tile_ranges.argtypes = [i64, vp, cam, vp]
        L.orc_tile_ranges.restype = None
        L.orc_sh_basis.argtypes = [vp, vp, vp]
        L.orc_sh_basis.restype = None
        L.orc_project64.argtypes = [i64, vp, vp, vp, vp, vp, cam, vp]
        L.orc_project64.restype = None
        L.orc_render64.argtypes = [cam, i64, vp, vp, vp, vp, vp, vp, vp, dbl, vp, vp]
        L.orc_render64.restype = i64
        L.orc_render64_brute.argtypes = [cam, vp, i64, vp, vp, vp, vp]
        L.orc_render64_brute.restype = i64
        L.orc_raster_bwd64.argtypes = [cam, i64, vp, vp, vp, vp, vp, vp]
        L.orc_raster_bwd64.restype = None
        L.orc_project_bwd64.argtypes = [i64, vp, vp, vp, vp, vp, cam, vp, vp, vp]
        L.orc_project_bwd64.restype = None
        L.orc_adam64.argtypes = [i64, vp, vp, vp, vp, vp, dbl, dbl, dbl, i32]
        L.orc_adam64.restype = None
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = i32
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: leave as is); returns the
    count in effect.  For timing only: results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def make_cam(cam, tile_w: int = 16, tile_h: int = 16) -> OrcCam:
    """Camera in the oracle's struct: FP32 values, as the device stores them."""
    c = OrcCam()
    R = np.asarray(cam.R, np.float32).reshape(-1)
    t = np.asarray(cam.t, np.float32).reshape(-1)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.tile_w, c.tile_h = int(tile_w), int(tile_h)
    return c


def tiles_of(cam, tile_w=16, tile_h=16):
    return (cam.width + tile_w - 1) // tile_w, (cam.height + tile_h - 1) // tile_h


def tile_bits(n_tiles: int) -> int:
    b = 0
    while (1 << b) < n_tiles:
        b += 1
    return b


def key_shift(n_tiles: int) -> int:
    tb = tile_bits(n_tiles)
    return 32 - tb if tb >= 9 else 23


# --------------------------------------------------------------------------
# FP32 binning (bit-specified; Sec. 4.1 and Sec. 4.4)
# --------------------------------------------------------------------------

@dataclass
class Binning:
    count: np.ndarray        # (n,) uint32 tiles per Gaussian
    bin: np.ndarray          # (n, 8) float32 valid, mx, my, a, b, c, det, tz
    mant: np.ndarray         # (n,) uint32 23-bit depth code
    offset: np.ndarray       # (n + 1,) int64 exclusive scan of count
    keys_emit: np.ndarray    # (K,) uint32 keys in emission order
    gidx_emit: np.ndarray    # (K,) uint32 Gaussian of each emitted pair
    keys: np.ndarray         # (K,) uint32 sorted keys (stable)
    gidx: np.ndarray         # (K,) uint32 Gaussians in sorted order
    perm: np.ndarray         # (K,) int64 emission slot of each sorted entry
    ranges: np.ndarray       # (tiles, 2) int64 [start, end) per tile

    @property
    def K(self) -> int:
        return int(self.keys.shape[0])


def log32(x: float) -> float:
    """The binning's FP32 natural logarithm (fixed atanh series)."""
    return float(lib().orc_log32(float(np.float32(x))))


def cull_r2(o: float) -> float:
    """The binning's cull radius^2 for opacity o (negative: never blended)."""
    return float(lib().orc_cull_r2(float(np.float32(o))))


def bin32(scene, cam, tile_w=16, tile_h=16) -> Binning:
    L = lib()
    c = make_cam(cam, tile_w, tile_h)
    n = scene.n
    means = np.ascontiguousarray(scene.means, np.float32)
    quats = np.ascontiguousarray(scene.quats, np.float32)
    scales = np.ascontiguousarray(scene.scales, np.float32)
    opac = np.ascontiguousarray(scene.opacities, np.float32)
    count = np.zeros(n, np.uint32)
    b = np.zeros((n, 8), np.float32)
    mant = np.zeros(n, np.uint32)
    L.orc_bin32_count(n, _ptr(means), _ptr(quats), _ptr(scales), _ptr(opac), ctypes.byref(c), _ptr(count), _ptr(b),
                      _ptr(mant))
    offset = np.zeros(n + 1, np.int64)
    np.cumsum(count, out=offset[1:])
    K = int(offset[-1])
    keys = np.zeros(max(K, 1), np.uint32)
    gidx = np.zeros(max(K, 1), np.uint32)
    got = L.orc_bin32_emit(n, _ptr(means), _ptr(quats), _ptr(scales), _ptr(opac), ctypes.byref(c), _ptr(offset),
                           _ptr(keys), _ptr(gidx))
    assert got == K
    keys, gidx = keys[:K], gidx[:K]
    keys_emit, gidx_emit = keys.copy(), gidx.copy()
    slot = np.arange(K, dtype=np.uint32)
    skeys = keys.copy()
    L.orc_stable_sort(K, _ptr(skeys), _ptr(slot))
    tx, ty = tiles_of(cam, tile_w, tile_h)
    ranges = np.zeros((tx * ty, 2), np.int64)
    L.orc_tile_ranges(K, _ptr(skeys), ctypes.byref(c), _ptr(ranges))
    return Binning(count, b, mant, offset, keys_emit, gidx_emit, skeys, gidx_emit[slot.astype(np.int64)],
                   slot.astype(np.int64), ranges)


def sort64(b: Binning, cam, tile_w=16, tile_h=16) -> Binning:
    """The same tile lists ordered by 64-bit keys instead of the 32-bit keys
    of Sec. 4.4: tile id in the high 32 bits, the full binary32 depth t_z in
    the low 32 (its bit pattern orders like the value, t_z > 0), stable, so
    equal depths keep ascending Gaussian order.  The 32-bit key keeps only
    the top (32 - tile bits) bits of the depth code; the two orders differ
    only among entries of a tile whose truncated codes are equal."""
    tx, ty = tiles_of(cam, tile_w, tile_h)
    shift = key_shift(tx * ty)
    tile = (b.keys_emit >> np.uint32(shift)).astype(np.uint64)
    tz = np.ascontiguousarray(b.bin[b.gidx_emit.astype(np.int64), 7], np.float32)
    key64 = (tile << np.uint64(32)) | tz.view(np.uint32).astype(np.uint64)
    perm = np.argsort(key64, kind="stable")
    return Binning(b.count, b.bin, b.mant, b.offset, b.keys_emit, b.gidx_emit, b.keys_emit[perm],
                   b.gidx_emit[perm], perm.astype(np.int64), b.ranges)


# --------------------------------------------------------------------------
# FP64 forward / backward / Adam
# --------------------------------------------------------------------------

@dataclass
class Params64:
    """Activated parameters in FP64: means, quats, scales, opacities, sh."""
    means: np.ndarray
    quats: np.ndarray
    scales: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray

    @staticmethod
    def from_scene(scene) -> "Params64":
        f = lambda a: np.ascontiguousarray(a, np.float64)
        return Params64(f(scene.means), f(scene.quats), f(scene.scales), f(scene.opacities),
                        f(scene.sh).reshape(scene.n, 48))

    @property
    def n(self):
        return self.means.shape[0]

    def theta(self) -> np.ndarray:
        """Optimised variables (n, 59): mean, quat, log-scale, logit-opacity, SH."""
        o = self.opacities
        return np.concatenate([self.means, self.quats, np.log(self.scales),
                               np.log(o / (1 - o))[:, None], self.sh.reshape(self.n, 48)], axis=1)

    @staticmethod
    def from_theta(th: np.ndarray) -> "Params64":
        th = np.asarray(th, np.float64)
        return Params64(th[:, 0:3].copy(), th[:, 3:7].copy(), np.exp(th[:, 7:10]),
                        1.0 / (1.0 + np.exp(-th[:, 10])), th[:, 11:59].copy())


def project64(p: Params64, cam, tile_w=16, tile_h=16) -> np.ndarray:
    L = lib()
    c = make_cam(cam, tile_w, tile_h)
    proj = np.zeros((p.n, PSTRIDE), np.float64)
    L.orc_project64(p.n, _ptr(p.means), _ptr(p.quats), _ptr(p.scales), _ptr(p.opacities), _ptr(p.sh),
                    ctypes.byref(c), _ptr(proj))
    return proj


@dataclass
class Render:
    image: np.ndarray        # (H, W, 3)
    tfinal: np.ndarray       # (H, W)
    nlast: np.ndarray        # (H, W) int32
    blended: int
    unstable_px: np.ndarray  # (H, W) bool
    unstable_g: np.ndarray   # (n,) bool


def render64(cam, proj, b: Binning, bg=(0.0, 0.0, 0.0), margin=1e-4, tile_w=16, tile_h=16) -> Render:
    L = lib()
    c = make_cam(cam, tile_w, tile_h)
    H, W = cam.height, cam.width
    n = proj.shape[0]
    img = np.zeros((H, W, 3), np.float64)
    tf = np.zeros((H, W), np.float64)
    nl = np.zeros((H, W), np.int32)
    upx = np.zeros((H, W), np.uint8)
    ug = np.zeros(n, np.uint8)
    bgv = np.asarray(bg, np.float64)
    sg = np.ascontiguousarray(b.gidx, np.uint32)
    rg = np.ascontiguousarray(b.ranges, np.int64)
    blended = L.orc_render64(ctypes.byref(c), n, _ptr(proj), _ptr(sg), _ptr(rg), _ptr(bgv), _ptr(img),
                             _ptr(tf), _ptr(nl), float(margin), _ptr(upx), _ptr(ug))
    return Render(img, tf, nl, int(blended), upx.astype(bool), ug.astype(bool))


def render64_brute(cam, proj, order, bg=(0.0, 0.0, 0.0)):
    L = lib()
    c = make_cam(cam)
    H, W = cam.height, cam.width
    img = np.zeros((H, W, 3), np.float64)
    tf = np.zeros((H, W), np.float64)
    order = np.ascontiguousarray(order, np.uint32)
    bgv = np.asarray(bg, np.float64)
    blended = L.orc_render64_brute(ctypes.byref(c), _ptr(proj), order.shape[0], _ptr(order), _ptr(bgv),
                                   _ptr(img), _ptr(tf))
    return img, tf, int(blended)


def raster_bwd64(cam, proj, b: Binning, dLdC, bg=(0.0, 0.0, 0.0), tile_w=16, tile_h=16) -> np.ndarray:
    L = lib()
    c = make_cam(cam, tile_w, tile_h)
    n = proj.shape[0]
    g2 = np.zeros((n, 9), np.float64)
    dl = np.ascontiguousarray(dLdC, np.float64)
    bgv = np.asarray(bg, np.float64)
    sg = np.ascontiguousarray(b.gidx, np.uint32)
    rg = np.ascontiguousarray(b.ranges, np.int64)
    L.orc_raster_bwd64(ctypes.byref(c), n, _ptr(proj), _ptr(sg), _ptr(rg), _ptr(bgv), _ptr(dl), _ptr(g2))
    return g2


def project_bwd64(p: Params64, cam, proj, grad2d, out=None) -> np.ndarray:
    L = lib()
    c = make_cam(cam)
    g = np.zeros((p.n, NTHETA), np.float64) if out is None else out
    g2 = np.ascontiguousarray(grad2d, np.float64)
    L.orc_project_bwd64(p.n, _ptr(p.means), _ptr(p.quats), _ptr(p.scales), _ptr(p.opacities), _ptr(p.sh),
                        ctypes.byref(c), _ptr(proj), _ptr(g2), _ptr(g))
    return g


def adam64(theta, m, v, grad, lr, step, b1=0.9, b2=0.999, eps=1e-15):
    """In-place Adam on (n, 59) arrays; lr: 6 per-group rates."""
    L = lib()
    lr = np.asarray(lr, np.float64)
    assert lr.shape == (6,)
    for a in (theta, m, v, grad):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    L.orc_adam64(theta.shape[0], _ptr(theta), _ptr(m), _ptr(v), _ptr(grad), _ptr(lr), b1, b2, eps, int(step))


def sh_basis(d):
    L = lib()
    d = np.ascontiguousarray(d, np.float64)
    Y = np.zeros(16, np.float64)
    dY = np.zeros(48, np.float64)
    L.orc_sh_basis(_ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY.reshape(16, 3)


def l1_loss_grad(images, targets):
    """L1 loss over all pixels of all views, mean over 3 * sum(P):
    dL/dC = sign(C - C*) / (3 sum P), sign(0) = 0 (Sec. 4.5, L1 term)."""
    total = sum(int(np.prod(im.shape)) for im in images)
    loss = sum(float(np.abs(im - tg).sum()) for im, tg in zip(images, targets)) / total
    grads = [np.sign(im - tg) / total for im, tg in zip(images, targets)]
    return loss, grads


# --------------------------------------------------------------------------
# Whole step
# --------------------------------------------------------------------------

@dataclass
class StepResult:
    binnings: list
    projs: list
    renders: list
    loss: float
    dLdC: list
    grad2d: list
    grad: np.ndarray         # (n, 59) theta gradient
    theta: np.ndarray        # (n, 59) after Adam
    m: np.ndarray
    v: np.ndarray
    params: Params64         # activated parameters after Adam


def step(scene, cams, targets, lr, step_idx=1, m=None, v=None, bg=(0.0, 0.0, 0.0),
         tile_w=16, tile_h=16, margin=1e-4, grad_only=False) -> StepResult:
    """One training step over the views `cams` of one scene: forward, L1 over
    all views, backward, one Adam update.  `targets` are (H, W, 3) arrays."""
    p = Params64.from_scene(scene)
    bins, projs, rends = [], [], []
    for cam in cams:
        b = bin32(scene, cam, tile_w, tile_h)
        pr = project64(p, cam, tile_w, tile_h)
        r = render64(cam, pr, b, bg, margin, tile_w, tile_h)
        bins.append(b); projs.append(pr); rends.append(r)
    loss, dl = l1_loss_grad([r.image for r in rends], targets)
    grad = np.zeros((p.n, NTHETA), np.float64)
    g2s = []
    for cam, b, pr, d in zip(cams, bins, projs, dl):
        g2 = raster_bwd64(cam, pr, b, d, bg, tile_w, tile_h)
        g2s.append(g2)
        project_bwd64(p, cam, pr, g2, out=grad)
    theta = p.theta()
    mm = np.zeros_like(theta) if m is None else np.array(m, np.float64, copy=True)
    vv = np.zeros_like(theta) if v is None else np.array(v, np.float64, copy=True)
    if not grad_only:
        adam64(theta, mm, vv, grad, lr, step_idx)
    return StepResult(bins, projs, rends, loss, dl, g2s, grad, theta, mm, vv, Params64.from_theta(theta))


# --------------------------------------------------------------------------
# L1 + SSIM loss (Sec. 4.5: weighted sum of L1 and SSIM on channel-last
# renders, reference image stored as 8-bit RGBA)
# --------------------------------------------------------------------------

SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """1-D Gaussian window, normalised to sum 1 (the 2-D window is its outer
    product)."""
    x = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _wfilter(img, g):
    """Window-weighted sum with zero padding outside the image, same size."""
    from scipy.ndimage import correlate1d
    t = correlate1d(img, g, axis=0, mode="constant", cval=0.0)
    return correlate1d(t, g, axis=1, mode="constant", cval=0.0)


def rgba8_to_float(target_rgba8):
    """8-bit RGBA reference -> float RGB in [0, 1]."""
    return np.asarray(target_rgba8, np.float64)[..., :3] / 255.0


def rgba8_alpha(target_rgba8):
    """8-bit RGBA reference -> its alpha in [0, 1] (the mask)."""
    return np.asarray(target_rgba8, np.float64)[..., 3] / 255.0


def l1_ssim_loss_grad(images, targets, lam: float = 0.2, masks=None):
    """L = (1 - lam) L1 + lam (1 - SSIM) over all pixels and channels of all
    views (means over 3 x pixels); SSIM per channel with an 11x11 Gaussian
    window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2.  Returns
    (loss, [dL/dC per view]).

    The SSIM map at q depends on the rendered image x through the window
    moments mu_x, E[x^2], E[xy] at q; with A = dSSIM/dmu_x, B = dSSIM/dE[x^2]
    and Cc = dSSIM/dE[xy] at every q, dSSIM_sum/dx_p = (w * A)(p) +
    2 x_p (w * B)(p) + y_p (w * Cc)(p) (the window is symmetric).

    masks (alpha masking, Sec. 4.5; one (H, W) array in [0, 1] per view, the
    reference's alpha): the loss is taken on the masked images m x and m y,
    so masked-out pixels add nothing, and the chain rule multiplies the
    gradient by m."""
    g = ssim_window()
    total = sum(int(np.prod(im.shape)) for im in images)
    l1 = 0.0
    ssim_sum = 0.0
    grads = []
    if masks is None:
        masks = [None] * len(images)
    for x3, y3, m in zip(images, targets, masks):
        x3 = np.asarray(x3, np.float64)
        y3 = np.asarray(y3, np.float64)
        if m is not None:
            m3 = np.asarray(m, np.float64)[..., None]
            x3, y3 = x3 * m3, y3 * m3
        d = np.zeros_like(x3)
        for c in range(3):
            x, y = x3[..., c], y3[..., c]
            mx, my = _wfilter(x, g), _wfilter(y, g)
            vx = _wfilter(x * x, g) - mx * mx
            vy = _wfilter(y * y, g) - my * my
            cxy = _wfilter(x * y, g) - mx * my
            a1 = 2 * mx * my + SSIM_C1
            a2 = 2 * cxy + SSIM_C2
            b1 = mx * mx + my * my + SSIM_C1
            b2 = vx + vy + SSIM_C2
            s = a1 * a2 / (b1 * b2)
            ssim_sum += float(s.sum())
            A = 2 * my * (a2 - a1) / (b1 * b2) - 2 * mx * s / b1 + 2 * mx * s / b2
            B = -s / b2
            Cc = 2 * a1 / (b1 * b2)
            dS = _wfilter(A, g) + 2 * x * _wfilter(B, g) + y * _wfilter(Cc, g)
            d[..., c] = (1 - lam) * np.sign(x - y) / total - lam * dS / total
        l1 += float(np.abs(x3 - y3).sum())
        if m is not None:
            d = d * m3
        grads.append(d)
    loss = (1 - lam) * l1 / total + lam * (1 - ssim_sum / total)
    return loss, grads


# --------------------------------------------------------------------------
# Default densification (Sec. 4.6: the 3DGS default strategy, which the
# paper follows) and its gradient statistic
# --------------------------------------------------------------------------

def densify_stats64(res: StepResult, cams) -> np.ndarray:
    """Statistics one step adds, (n, 2): for every view in which a Gaussian
    is listed (tile count > 0), x += |dL/d(mean2D)| with the x component
    scaled by W/2, y by H/2, both by P_all / P_view (the gradient of that
    view's own mean loss), and y += 1."""
    n = res.grad.shape[0]
    p_all = float(sum(c.width * c.height for c in cams))
    st = np.zeros((n, 2), np.float64)
    for cam, b, g2 in zip(cams, res.binnings, res.grad2d):
        vis = b.count > 0
        fac = p_all / float(cam.width * cam.height)
        gx = g2[:, 0] * (0.5 * cam.width) * fac
        gy = g2[:, 1] * (0.5 * cam.height) * fac
        st[vis, 0] += np.hypot(gx, gy)[vis]
        st[vis, 1] += 1.0
    return st


@dataclass
class DenseScene:
    """One scene in rows: means (n,3), quats (n,4), scales (n,3) and
    opacities (n,) activated, sh (n,48) flat (index 3k + channel), Adam
    moments m, v (n,60) in the chunk order (mean xyz + pad, quaternion,
    log-scale xyz + logit-opacity, 48 SH), stats (n,2)."""
    means: np.ndarray
    quats: np.ndarray
    scales: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray
    m: np.ndarray
    v: np.ndarray
    stats: np.ndarray

    @property
    def n(self):
        return self.means.shape[0]

    def take(self, idx):
        return DenseScene(*(a[idx] for a in (self.means, self.quats, self.scales, self.opacities, self.sh,
                                              self.m, self.v, self.stats)))


def _rotation64(q):
    """Rotation matrices (n,3,3) of quaternions (w, x, y, z), normalised."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def densify64(sc: DenseScene, eps, scene_scale, grow_grad2d=2e-4, grow_scale3d=0.01, prune_opa=0.005,
              prune_scale3d=0.1, split_factor=1.6, grow=True, prune_big=False):
    """One refinement of the default strategy, in its three stages:
      1. clone: Gaussians whose mean statistic x / max(y, 1) exceeds
         grow_grad2d and whose largest scale is <= grow_scale3d * scene_scale
         get a copy appended (zero moments);
      2. split: the other high-statistic Gaussians of the original set are
         removed and two products appended (first products of all, then
         second products of all): mean + R(q) (scale * eps_k), scale /
         split_factor, the rest copied, zero moments;
      3. prune: Gaussians with opacity < prune_opa -- and with prune_big,
         largest scale > prune_scale3d * scene_scale -- are removed.
    The decisions compare binary32 stored values with binary32 thresholds
    (as the parameters are stored), the new means are FP64.  Statistics of
    the result are zero.  Returns (scene, (kept, clones, splits, total))."""
    f32 = np.float32
    n = sc.n
    eps = np.asarray(eps, np.float64).reshape(n, 2, 3)
    avg = sc.stats[:, 0].astype(f32) / np.maximum(sc.stats[:, 1].astype(f32), f32(1.0))
    high = np.zeros(n, bool) if not grow else avg > f32(grow_grad2d)
    smax = sc.scales.astype(f32).max(axis=1)
    small = smax <= f32(grow_scale3d) * f32(scene_scale)
    is_clone, is_split = high & small, high & ~small
    # stage 1: clone
    s1 = DenseScene(*(np.concatenate([a, a[is_clone]]) for a in (sc.means, sc.quats, sc.scales, sc.opacities,
                                                                 sc.sh, sc.m, sc.v, sc.stats)))
    s1.m[n:] = 0.0
    s1.v[n:] = 0.0
    split1 = np.concatenate([is_split, np.zeros(int(is_clone.sum()), bool)])
    # stage 2: split
    sel = np.nonzero(split1)[0]
    rest = s1.take(np.nonzero(~split1)[0])
    R = _rotation64(s1.quats[sel])
    sv = s1.scales[sel].astype(np.float64)
    prods = []
    for k in range(2):
        off = np.einsum("nij,nj->ni", R, sv * eps[sel, k])
        p = s1.take(sel)
        p.means = (p.means.astype(np.float64) + off)
        p.scales = (p.scales.astype(f32) / f32(split_factor)).astype(f32)
        p.m = np.zeros_like(p.m)
        p.v = np.zeros_like(p.v)
        prods.append(p)
    s2 = DenseScene(*(np.concatenate([getattr(rest, f), getattr(prods[0], f), getattr(prods[1], f)])
                      for f in ("means", "quats", "scales", "opacities", "sh", "m", "v", "stats")))
    # stage 3: prune
    prune = s2.opacities.astype(f32) < f32(prune_opa)
    if prune_big:
        prune |= s2.scales.astype(f32).max(axis=1) > f32(prune_scale3d) * f32(scene_scale)
    out = s2.take(np.nonzero(~prune)[0])
    out.stats = np.zeros_like(out.stats)
    n_orig = rest.n - int(is_clone.sum())      # rest = [original non-split rows, clone rows]
    kept = int((~prune[:n_orig]).sum())
    clones = int((~prune[n_orig:rest.n]).sum())
    splits = int((~prune[rest.n:rest.n + len(sel)]).sum())
    return out, (kept, clones, splits, out.n)


def reset_opacity64(sc: DenseScene, value=0.01) -> DenseScene:
    """o = min(o, value) (binary32) and zero logit-opacity moments."""
    out = sc.take(np.arange(sc.n))
    out.opacities = np.minimum(sc.opacities.astype(np.float32), np.float32(value))
    out.m[:, 11] = 0.0
    out.v[:, 11] = 0.0
    return out
