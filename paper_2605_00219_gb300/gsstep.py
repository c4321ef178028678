"""Thin Python binding of the C ABI in include/gs_step.h.

Argument marshalling only: every stage of the step runs in the CUDA kernels
of libgsstep.so.  Tensors are passed by device pointer; the stream is the
current torch CUDA stream unless one is given.  There is no CPU fallback: if
the library is missing or fails to load, the import of any stage fails.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# GS_DEBUG_LIB=1 in the environment loads the bounds-checked build instead
# (paper_2605_00219_gb300.build.build(debug=True))
LIB_PATH = os.path.join(HERE, "_lib", "libgsstep_debug.so" if os.environ.get("GS_DEBUG_LIB") == "1"
                        else "libgsstep.so")

MAX_VIEWS = 64
MAX_SCENES = 16
STORE_SH_BF16 = 0x1
STORE_MOMENTS_BF16 = 0x2
STATUS_CAPACITY = 0x1
STATUS_NONFINITE = 0x2
STATUS_TIMEOUT = 0x4
STATUS_BOUNDS = 0x8

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_NONFINITE",
                4: "GS_ERR_TIMEOUT", 5: "GS_ERR_CUDA", 6: "GS_ERR_UNIMPLEMENTED"}

# exported symbols (the C ABI)
SYMBOLS = ["gs_plan_create", "gs_plan_destroy", "gs_workspace_bytes", "gs_plan_query", "gs_workspace_init",
           "gs_project_fwd", "gs_bin_sort", "gs_raster_fwd", "gs_loss_l1", "gs_raster_bwd",
           "gs_project_bwd_adam", "gs_adam_advance", "gs_read_stats", "gs_workspace_buffer", "gs_status_str",
           "gs_loss_l1_noalloc", "gs_loss_l1_ssim", "gs_loss_l1_ssim_masked", "gs_densify_scratch_bytes", "gs_densify_count",
           "gs_densify_counts", "gs_densify_apply", "gs_reset_opacity", "gs_workspace_set_step"]
L1_NOALLOC_MAX_VALUES = 67108864


class gs_view(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("scene", ctypes.c_int32)]


class gs_tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("bwd_batch", ctypes.c_int32),
                ("bwd_impl", ctypes.c_int32), ("threads_per_tile", ctypes.c_int32)]


class gs_scene_buf(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("geom", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("m", ctypes.c_void_p), ("v", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


class gs_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 6), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("reserved", ctypes.c_int32)]


class gs_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("step", ctypes.c_int32), ("k_required", ctypes.c_int64),
                ("k_capacity", ctypes.c_int64), ("blended_pairs", ctypes.c_uint64), ("loss", ctypes.c_float),
                ("reserved", ctypes.c_float)]


class gs_densify_cfg(ctypes.Structure):
    _fields_ = [("grow_grad2d", ctypes.c_float), ("grow_scale3d", ctypes.c_float), ("prune_opa", ctypes.c_float),
                ("prune_scale3d", ctypes.c_float), ("scene_scale", ctypes.c_float), ("split_factor", ctypes.c_float),
                ("grow", ctypes.c_int32), ("prune_big", ctypes.c_int32)]


class GSError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libgsstep.so (built by paper_2605_00219_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GSError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run paper_2605_00219_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.gs_plan_create.argtypes = [ctypes.POINTER(i64), i32, ctypes.POINTER(gs_view), i32, i64,
                                     ctypes.POINTER(gs_tuning), i32, ctypes.POINTER(ctypes.c_int)]
        L.gs_plan_create.restype = vp
        L.gs_plan_destroy.argtypes = [vp]
        L.gs_plan_destroy.restype = None
        L.gs_workspace_bytes.argtypes = [vp]
        L.gs_workspace_bytes.restype = ctypes.c_size_t
        L.gs_plan_query.argtypes = [vp, i32]
        L.gs_plan_query.restype = i64
        L.gs_workspace_init.argtypes = [vp, vp, vp]
        L.gs_project_fwd.argtypes = [vp, vp, ctypes.POINTER(gs_scene_buf), vp, vp]
        L.gs_bin_sort.argtypes = [vp, vp, vp]
        L.gs_raster_fwd.argtypes = [vp, vp, vp, vp, vp]
        L.gs_loss_l1.argtypes = [vp, vp, vp, vp, vp, vp]
        L.gs_loss_l1_ssim.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp, vp]
        L.gs_loss_l1_ssim_masked.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp, vp]
        L.gs_raster_bwd.argtypes = [vp, vp, vp, vp, vp]
        L.gs_project_bwd_adam.argtypes = [vp, vp, ctypes.POINTER(gs_scene_buf), vp, ctypes.POINTER(gs_adam), vp, vp]
        L.gs_adam_advance.argtypes = [vp, vp, vp]
        L.gs_workspace_set_step.argtypes = [vp, vp, i32, vp]
        L.gs_read_stats.argtypes = [vp, vp, ctypes.POINTER(gs_stats), vp]
        L.gs_workspace_buffer.argtypes = [vp, vp, i32]
        L.gs_workspace_buffer.restype = vp
        L.gs_loss_l1_noalloc.argtypes = [vp, vp, vp, vp, i64, vp]
        L.gs_loss_l1_noalloc.restype = ctypes.c_int
        L.gs_densify_scratch_bytes.argtypes = [i64]
        L.gs_densify_scratch_bytes.restype = ctypes.c_size_t
        L.gs_densify_count.argtypes = [ctypes.POINTER(gs_scene_buf), i32, ctypes.POINTER(gs_densify_cfg), vp, vp]
        L.gs_densify_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), vp]
        L.gs_densify_apply.argtypes = [ctypes.POINTER(gs_scene_buf), i32, ctypes.POINTER(gs_densify_cfg), vp, vp,
                                       ctypes.POINTER(gs_scene_buf), vp]
        L.gs_reset_opacity.argtypes = [ctypes.POINTER(gs_scene_buf), i32, ctypes.c_float, vp]
        L.gs_status_str.argtypes = [ctypes.c_int]
        L.gs_status_str.restype = ctypes.c_char_p
        for name in ["gs_workspace_init", "gs_project_fwd", "gs_bin_sort", "gs_raster_fwd", "gs_loss_l1",
                     "gs_loss_l1_ssim", "gs_loss_l1_ssim_masked", "gs_raster_bwd", "gs_project_bwd_adam",
                     "gs_adam_advance", "gs_read_stats",
                     "gs_densify_count", "gs_densify_counts", "gs_densify_apply", "gs_reset_opacity",
                     "gs_workspace_set_step"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != GS_OK:
        raise GSError(f"{what}: {STATUS_NAMES.get(rc, rc)} ({lib().gs_status_str(rc).decode()})")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Static shape of a step (host object wrapping gs_plan)."""

    def __init__(self, scene_sizes, views, capacity: int = 0, tile=(16, 16), bwd_batch: int = 0,
                 storage_flags: int = 0, bwd_impl: int = 0, threads_per_tile: int = 0):
        L = lib()
        n_arr = (ctypes.c_int64 * len(scene_sizes))(*[int(x) for x in scene_sizes])
        v_arr = (gs_view * len(views))()
        for i, (w, h, s) in enumerate(views):
            v_arr[i] = gs_view(int(w), int(h), int(s))
        tun = gs_tuning(int(tile[0]), int(tile[1]), int(bwd_batch), int(bwd_impl), int(threads_per_tile))
        err = ctypes.c_int(0)
        h = L.gs_plan_create(n_arr, len(scene_sizes), v_arr, len(views), int(capacity), ctypes.byref(tun),
                             int(storage_flags), ctypes.byref(err))
        if not h:
            raise GSError(f"gs_plan_create: {STATUS_NAMES.get(err.value, err.value)}")
        self.handle = ctypes.c_void_p(h)
        self.scene_sizes = [int(x) for x in scene_sizes]
        self.views = [tuple(int(a) for a in v) for v in views]
        self.tile = tuple(tile)
        self.storage_flags = storage_flags
        self.bwd_impl = int(bwd_impl)
        self.bwd_batch = int(bwd_batch)
        self.threads_per_tile = int(threads_per_tile) or int(tile[0]) * int(tile[1])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.gs_plan_destroy(h)
            self.handle = None

    def query(self, what: int) -> int:
        return int(lib().gs_plan_query(self.handle, what))

    @property
    def pairs(self): return self.query(0)

    @property
    def tiles(self): return self.query(1)

    @property
    def pixels(self): return self.query(2)

    @property
    def capacity(self): return self.query(3)

    def workspace_bytes(self) -> int:
        return int(lib().gs_workspace_bytes(self.handle))


def scene_bufs(scenes):
    """gs_scene_buf array from a list of SceneBuffers."""
    arr = (gs_scene_buf * len(scenes))()
    for i, s in enumerate(scenes):
        st = getattr(s, "stats", None)
        arr[i] = gs_scene_buf(s.n, s.geom.data_ptr(), s.sh.data_ptr(),
                              s.m.data_ptr() if s.m is not None else None,
                              s.v.data_ptr() if s.v is not None else None,
                              st.data_ptr() if st is not None else None)
    return arr


def gs_workspace_init(plan: Plan, ws, stream=None):
    _check(lib().gs_workspace_init(plan.handle, _ptr(ws), _stream(stream)), "gs_workspace_init")


def gs_project_fwd(plan: Plan, ws, scenes, cams, stream=None):
    _check(lib().gs_project_fwd(plan.handle, _ptr(ws), scene_bufs(scenes), _ptr(cams), _stream(stream)),
           "gs_project_fwd")


def gs_bin_sort(plan: Plan, ws, stream=None):
    _check(lib().gs_bin_sort(plan.handle, _ptr(ws), _stream(stream)), "gs_bin_sort")


def gs_raster_fwd(plan: Plan, ws, bg, image, stream=None):
    _check(lib().gs_raster_fwd(plan.handle, _ptr(ws), _ptr(bg), _ptr(image), _stream(stream)), "gs_raster_fwd")


def gs_loss_l1(plan: Plan, ws, image, target, dl, stream=None):
    _check(lib().gs_loss_l1(plan.handle, _ptr(ws), _ptr(image), _ptr(target), _ptr(dl), _stream(stream)),
           "gs_loss_l1")


def gs_loss_l1_ssim(plan: Plan, ws, image, target_rgba8, lam, dl, stream=None):
    """target_rgba8: uint8 device tensor [pixels][4]; lam in [0, 1]."""
    _check(lib().gs_loss_l1_ssim(plan.handle, _ptr(ws), _ptr(image), _ptr(target_rgba8), float(lam), _ptr(dl),
                                 _stream(stream)), "gs_loss_l1_ssim")


def gs_loss_l1_ssim_masked(plan: Plan, ws, image, target_rgba8, lam, dl, stream=None):
    """gs_loss_l1_ssim with the reference's alpha (A / 255) as mask."""
    _check(lib().gs_loss_l1_ssim_masked(plan.handle, _ptr(ws), _ptr(image), _ptr(target_rgba8), float(lam),
                                        _ptr(dl), _stream(stream)), "gs_loss_l1_ssim_masked")


def gs_raster_bwd(plan: Plan, ws, image, dl, stream=None):
    _check(lib().gs_raster_bwd(plan.handle, _ptr(ws), _ptr(image), _ptr(dl), _stream(stream)), "gs_raster_bwd")


def make_adam(lr, beta1=0.9, beta2=0.999, eps=1e-15, step=1, seed=0) -> gs_adam:
    a = gs_adam()
    for i in range(6):
        a.lr[i] = float(lr[i])
    a.beta1, a.beta2, a.eps, a.step, a.seed = float(beta1), float(beta2), float(eps), int(step), int(seed)
    return a


def gs_project_bwd_adam(plan: Plan, ws, scenes, cams, adam: gs_adam | None, grads_out=None, stream=None):
    _check(lib().gs_project_bwd_adam(plan.handle, _ptr(ws), scene_bufs(scenes), _ptr(cams),
                                     ctypes.byref(adam) if adam is not None else None, _ptr(grads_out),
                                     _stream(stream)), "gs_project_bwd_adam")


def gs_adam_advance(plan: Plan, ws, stream=None):
    _check(lib().gs_adam_advance(plan.handle, _ptr(ws), _stream(stream)), "gs_adam_advance")


def gs_workspace_set_step(plan: Plan, ws, step: int, stream=None):
    _check(lib().gs_workspace_set_step(plan.handle, _ptr(ws), int(step), _stream(stream)), "gs_workspace_set_step")


def gs_read_stats(plan: Plan, ws, stream=None) -> gs_stats:
    st = gs_stats()
    _check(lib().gs_read_stats(plan.handle, _ptr(ws), ctypes.byref(st), _stream(stream)), "gs_read_stats")
    return st


def gs_workspace_buffer(plan: Plan, ws, which: int, numel: int, dtype=torch.int32):
    """A torch view (no copy) of a workspace buffer."""
    p = lib().gs_workspace_buffer(plan.handle, _ptr(ws), int(which))
    if not p:
        raise GSError(f"unknown workspace buffer {which}")
    base = ws.data_ptr()
    off = int(p) - base
    esz = torch.tensor([], dtype=dtype).element_size()
    assert off % esz == 0
    return ws.view(torch.uint8)[off:off + numel * esz].view(dtype)


def gs_gradient_records(plan: Plan, ws, k: int):
    """The first k gradient records (emission slots 0 .. k-1) as a (k, 9)
    float32 tensor (a copy).  Buffer 8 holds them as float4[cap][3]:
    (dL/d mean x, y, conic a, b), (conic c, opacity, r, g), (b, unused x 3)."""
    x = gs_workspace_buffer(plan, ws, 8, 12 * k, torch.float32)
    return x.view(k, 12)[:, :9].clone()


def gs_loss_l1_noalloc(image, target, dl, loss, stream=None):
    """L1 loss and gradient with no plan, no workspace and no device
    allocation (for callers that may not allocate); `loss` is a 1-element
    device float tensor.  See include/gs_step.h for the shared-scratch rules."""
    _check(lib().gs_loss_l1_noalloc(_ptr(image), _ptr(target), _ptr(dl), _ptr(loss), int(image.numel()),
                                    _stream(stream)), "gs_loss_l1_noalloc")


# ---------------------------------------------------------------------------
# Default densification
# ---------------------------------------------------------------------------

def make_densify_cfg(scene_scale, grow_grad2d=2e-4, grow_scale3d=0.01, prune_opa=0.005, prune_scale3d=0.1,
                     split_factor=1.6, grow=True, prune_big=False) -> gs_densify_cfg:
    return gs_densify_cfg(float(grow_grad2d), float(grow_scale3d), float(prune_opa), float(prune_scale3d),
                          float(scene_scale), float(split_factor), int(bool(grow)), int(bool(prune_big)))


def gs_densify_scratch_bytes(n: int) -> int:
    return int(lib().gs_densify_scratch_bytes(int(n)))


def gs_densify_count(scene, storage_flags: int, cfg: gs_densify_cfg, scratch, stream=None):
    _check(lib().gs_densify_count(scene_bufs([scene]), int(storage_flags), ctypes.byref(cfg), _ptr(scratch),
                                  _stream(stream)), "gs_densify_count")


def gs_densify_counts(scratch, stream=None):
    """(kept, clones, splits, total) -- synchronises the stream."""
    out = (ctypes.c_int64 * 4)()
    _check(lib().gs_densify_counts(_ptr(scratch), out, _stream(stream)), "gs_densify_counts")
    return tuple(int(x) for x in out)


def gs_densify_apply(scene_in, storage_flags: int, cfg: gs_densify_cfg, eps, scratch, scene_out, stream=None):
    _check(lib().gs_densify_apply(scene_bufs([scene_in]), int(storage_flags), ctypes.byref(cfg), _ptr(eps),
                                  _ptr(scratch), scene_bufs([scene_out]), _stream(stream)), "gs_densify_apply")


def gs_reset_opacity(scene, storage_flags: int, value: float, stream=None):
    _check(lib().gs_reset_opacity(scene_bufs([scene]), int(storage_flags), float(value), _stream(stream)),
           "gs_reset_opacity")
