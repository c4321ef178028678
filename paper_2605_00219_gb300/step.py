"""Device buffers and the training step built from the C-ABI calls.

`SceneBuffers` packs a scene into the device layout of include/gs_step.h
(chunk-major float4 SoA: geometry, SH, Adam moments).  `Trainer` owns one
plan and workspace and runs

    gs_project_fwd -> gs_bin_sort -> gs_raster_fwd -> gs_loss_l1 (or
    gs_loss_l1_ssim against an 8-bit RGBA target, or gs_loss_l1_ssim_masked
    with its alpha as mask) -> gs_raster_bwd
    -> gs_project_bwd_adam

on one stream, eagerly or as one captured CUDA graph whose replay reads the
cameras, targets and the Adam step counter from device memory.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import gsstep
from . import synth

# Per-group learning rates: mean, quaternion, log-scale, logit-opacity, SH
# degree 0, SH degrees 1-3.
DEFAULT_LR = (1.6e-4, 1e-3, 5e-3, 5e-2, 2.5e-3, 2.5e-3 / 20)


@dataclass
class SceneBuffers:
    n: int
    geom: torch.Tensor          # (3, n, 4) float32
    sh: torch.Tensor            # (12, n, 4) float32 or (6, n, 8) bfloat16
    m: torch.Tensor | None      # (15, n, 4) float32 or bfloat16
    v: torch.Tensor | None
    stats: torch.Tensor | None = None   # (n, 2) float32 densification statistics

    @property
    def storage_flags(self) -> int:
        return ((gsstep.STORE_SH_BF16 if self.sh.dtype == torch.bfloat16 else 0) |
                (gsstep.STORE_MOMENTS_BF16 if self.m is not None and self.m.dtype == torch.bfloat16 else 0))

    @staticmethod
    def empty_like_layout(ref: "SceneBuffers", n: int) -> "SceneBuffers":
        """Uninitialised buffers for n Gaussians in ref's layout."""
        dev = ref.geom.device
        return SceneBuffers(n, torch.empty((3, n, 4), dtype=torch.float32, device=dev),
                            torch.empty((ref.sh.shape[0], n, ref.sh.shape[2]), dtype=ref.sh.dtype, device=dev),
                            torch.empty((15, n, 4), dtype=ref.m.dtype, device=dev),
                            torch.empty((15, n, 4), dtype=ref.v.dtype, device=dev),
                            None if ref.stats is None else torch.empty((n, 2), dtype=torch.float32, device=dev))

    @staticmethod
    def from_scene(scene: synth.Scene, device="cuda", sh_bf16=False, mom_bf16=False, moments=True):
        n = scene.n
        geom = np.zeros((3, n, 4), np.float32)
        geom[0, :, :3] = scene.means
        geom[1] = scene.quats
        geom[2, :, :3] = scene.scales
        geom[2, :, 3] = scene.opacities
        flat = np.ascontiguousarray(scene.sh, np.float32).reshape(n, 48)
        g = torch.from_numpy(geom).to(device)
        if sh_bf16:
            sh = torch.from_numpy(flat.reshape(n, 6, 8).transpose(1, 0, 2).copy()).to(device).to(torch.bfloat16)
        else:
            sh = torch.from_numpy(flat.reshape(n, 12, 4).transpose(1, 0, 2).copy()).to(device)
        m = v = None
        if moments:
            mdt = torch.bfloat16 if mom_bf16 else torch.float32
            m = torch.zeros((15, n, 4), dtype=mdt, device=device)
            v = torch.zeros((15, n, 4), dtype=mdt, device=device)
        return SceneBuffers(n, g, sh.contiguous(), m, v)

    def to_scene(self) -> synth.Scene:
        geom = self.geom.detach().float().cpu().numpy()
        n = self.n
        if self.sh.dtype == torch.bfloat16:
            flat = self.sh.detach().float().cpu().numpy().transpose(1, 0, 2).reshape(n, 48)
        else:
            flat = self.sh.detach().cpu().numpy().transpose(1, 0, 2).reshape(n, 48)
        return synth.Scene(geom[0, :, :3].copy(), geom[1].copy(), geom[2, :, :3].copy(), geom[2, :, 3].copy(),
                           flat.reshape(n, 16, 3).copy())


def camera_params(cams) -> np.ndarray:
    return np.stack([c.pose_params() for c in cams]).astype(np.float32)


class Trainer:
    """One plan + workspace; runs the step over `cameras` (each with .scene)."""

    def __init__(self, scenes, cameras, capacity: int = 0, tile=(16, 16), bwd_batch: int = 0,
                 sh_bf16: bool = False, mom_bf16: bool = False, bg=None, lr=DEFAULT_LR, device="cuda",
                 bwd_impl: int = 0, loss: str = "l1", ssim_lambda: float = 0.2, seed: int = 0,
                 threads_per_tile: int = 0):
        if loss not in ("l1", "l1_ssim", "l1_ssim_masked"):
            raise ValueError(f"loss must be 'l1', 'l1_ssim' or 'l1_ssim_masked', not {loss!r}")
        self.loss = loss
        self.ssim_lambda = float(ssim_lambda)
        self.seed = int(seed)         # stochastic rounding of BF16 storage
        self.device = torch.device(device)
        self.scenes = [s if isinstance(s, SceneBuffers) else
                       SceneBuffers.from_scene(s, device, sh_bf16, mom_bf16) for s in scenes]
        flags = (gsstep.STORE_SH_BF16 if sh_bf16 else 0) | (gsstep.STORE_MOMENTS_BF16 if mom_bf16 else 0)
        self.plan = gsstep.Plan([s.n for s in self.scenes], [(c.width, c.height, c.scene) for c in cameras],
                                capacity, tile, bwd_batch, flags, bwd_impl, threads_per_tile)
        self.ws = torch.empty(self.plan.workspace_bytes(), dtype=torch.uint8, device=self.device)
        self.cams = torch.from_numpy(camera_params(cameras)).to(self.device)
        P = self.plan.pixels
        self.image = torch.zeros((P, 3), dtype=torch.float32, device=self.device)
        if loss == "l1":
            self.target = torch.zeros((P, 3), dtype=torch.float32, device=self.device)
        else:
            self.target = torch.zeros((P, 4), dtype=torch.uint8, device=self.device)
        self.dl = torch.zeros((P, 3), dtype=torch.float32, device=self.device)
        self.bg = None if bg is None else torch.tensor(bg, dtype=torch.float32, device=self.device)
        self.view_shapes = [(c.width, c.height) for c in cameras]
        self.lr = tuple(lr)
        self.graph = None
        self._pair = None
        gsstep.gs_workspace_init(self.plan, self.ws)

    # -- inputs -------------------------------------------------------------
    def set_cameras(self, cameras):
        self.cams.copy_(torch.from_numpy(camera_params(cameras)), non_blocking=False)

    def set_target(self, images):
        """images: list of (H, W, 3) arrays/tensors, one per view.  With the
        L1 + SSIM loss the target is 8-bit RGBA: uint8 (H, W, 4) images are
        taken as they are, float images in [0, 1] are rounded to bytes."""
        if self.loss == "l1":
            flat = torch.cat([torch.as_tensor(np.asarray(im, np.float32)).reshape(-1, 3) for im in images])
            self.target.copy_(flat)
            return
        parts = []
        for im in images:
            a = np.asarray(im)
            if a.dtype != np.uint8:
                a = np.clip(np.rint(np.asarray(a, np.float64) * 255.0), 0, 255).astype(np.uint8)
            if a.shape[-1] == 3:
                a = np.concatenate([a, np.full(a.shape[:-1] + (1,), 255, np.uint8)], axis=-1)
            parts.append(torch.from_numpy(np.ascontiguousarray(a).reshape(-1, 4)))
        self.target.copy_(torch.cat(parts))

    def image_views(self, img=None):
        img = self.image if img is None else img
        out, o = [], 0
        for (w, h) in self.view_shapes:
            out.append(img[o:o + w * h].view(h, w, 3))
            o += w * h
        return out

    # -- stages -------------------------------------------------------------
    def forward(self, stream=None):
        gsstep.gs_project_fwd(self.plan, self.ws, self.scenes, self.cams, stream)
        gsstep.gs_bin_sort(self.plan, self.ws, stream)
        gsstep.gs_raster_fwd(self.plan, self.ws, self.bg, self.image, stream)
        return self.image

    def backward_adam(self, step: int = 0, stream=None):
        if self.loss == "l1":
            gsstep.gs_loss_l1(self.plan, self.ws, self.image, self.target, self.dl, stream)
        elif self.loss == "l1_ssim":
            gsstep.gs_loss_l1_ssim(self.plan, self.ws, self.image, self.target, self.ssim_lambda, self.dl, stream)
        else:   # the reference's alpha as mask
            gsstep.gs_loss_l1_ssim_masked(self.plan, self.ws, self.image, self.target, self.ssim_lambda, self.dl,
                                          stream)
        gsstep.gs_raster_bwd(self.plan, self.ws, self.image, self.dl, stream)
        adam = gsstep.make_adam(self.lr, step=step, seed=self.seed)
        gsstep.gs_project_bwd_adam(self.plan, self.ws, self.scenes, self.cams, adam, None, stream)
        if step <= 0:
            gsstep.gs_adam_advance(self.plan, self.ws, stream)

    def step(self, step: int = 0, stream=None):
        """One training step; step <= 0 takes Adam's t from the device counter."""
        self.forward(stream)
        self.backward_adam(step, stream)

    # -- graphs -------------------------------------------------------------
    def capture(self):
        """Capture one whole step (device step counter) in a CUDA graph."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.step(0, s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def capture_pair(self):
        """Two graphs of the step reading targets and cameras from two
        buffer sets, so that the host copy of one step's inputs can overlap
        the previous step (see run_from_host)."""
        t2, c2 = torch.empty_like(self.target), torch.empty_like(self.cams)
        ga = self.capture()
        self.target, t2 = t2, self.target
        self.cams, c2 = c2, self.cams
        gb = self.capture()
        bufs_b = (self.target, self.cams)
        self.target, self.cams = t2, c2
        self._pair = ((ga, (self.target, self.cams)), (gb, bufs_b))
        self.graph = ga

    def run_from_host(self, host_target, host_cams, steps: int):
        """`steps` graph-replayed steps whose inputs come from host memory:
        step k's targets and cameras (host_target(k), host_cams(k): pinned CPU
        tensors) are copied on a side stream while step k - 1 runs, and each
        step's statistics are read back after it.  Returns the losses."""
        if getattr(self, "_pair", None) is None:
            self.capture_pair()
        main = torch.cuda.current_stream(self.device)
        side = torch.cuda.Stream(device=self.device)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]

        def issue(k):
            _, (tb, cb) = self._pair[k % 2]
            with torch.cuda.stream(side):
                if k >= 2:
                    side.wait_event(free[k % 2])
                tb.copy_(host_target(k), non_blocking=True)
                cb.copy_(host_cams(k), non_blocking=True)
                copied[k % 2].record(side)

        losses = []
        issue(0)
        for k in range(steps):
            if k + 1 < steps:
                issue(k + 1)
            main.wait_event(copied[k % 2])
            self._pair[k % 2][0].replay()
            free[k % 2].record(main)
            losses.append(float(self.stats().loss))
        return losses

    def stats(self) -> gsstep.gs_stats:
        return gsstep.gs_read_stats(self.plan, self.ws)

    def buffer(self, which: int, numel: int, dtype=torch.int32):
        return gsstep.gs_workspace_buffer(self.plan, self.ws, which, numel, dtype)

    # -- default densification ----------------------------------------------
    def enable_densify_stats(self):
        """Let gs_project_bwd_adam accumulate the densification statistics."""
        for sb in self.scenes:
            if sb.stats is None:
                sb.stats = torch.zeros((sb.n, 2), dtype=torch.float32, device=self.device)
        self.graph = None
        self._pair = None

    def densify(self, scene_scale, generator=None, **cfg):
        """One refinement of the default strategy on every scene (clone /
        split / prune, see gs_densify_apply), then a new plan and workspace for
        the new sizes (the Adam step counter carries over; a captured graph is
        dropped).  Returns [(kept, clones, splits, total)] per scene."""
        t = int(self.stats().step)
        out = []
        for k, sb in enumerate(self.scenes):
            c = gsstep.make_densify_cfg(scene_scale, **cfg)
            scratch = torch.empty(gsstep.gs_densify_scratch_bytes(sb.n), dtype=torch.uint8, device=self.device)
            gsstep.gs_densify_count(sb, sb.storage_flags, c, scratch)
            counts = gsstep.gs_densify_counts(scratch)
            eps = torch.randn((sb.n, 6), dtype=torch.float32, device=self.device, generator=generator)
            nb = SceneBuffers.empty_like_layout(sb, counts[3])
            gsstep.gs_densify_apply(sb, sb.storage_flags, c, eps, scratch, nb)
            self.scenes[k] = nb
            out.append(counts)
        self._replan(t)
        return out

    def reset_opacity(self, value: float = 0.01):
        for sb in self.scenes:
            gsstep.gs_reset_opacity(sb, sb.storage_flags, value)

    # -- checkpoints -----------------------------------------------------------
    def state_dict(self) -> dict:
        """Parameters, both Adam moments, densification statistics (when
        kept) and the Adam step counter, as host tensors.  Every kernel of the
        step is deterministic and the BF16 rounding is keyed by (seed, step,
        Gaussian), so training resumed from a checkpoint repeats the
        uninterrupted run bit for bit."""
        scenes = []
        for sb in self.scenes:
            d = {"n": sb.n, "geom": sb.geom.cpu(), "sh": sb.sh.cpu(), "m": sb.m.cpu(), "v": sb.v.cpu()}
            if sb.stats is not None:
                d["stats"] = sb.stats.cpu()
            scenes.append(d)
        return {"scenes": scenes, "step": int(self.stats().step), "seed": self.seed, "lr": list(self.lr)}

    def load_state_dict(self, state: dict):
        """Restore a checkpoint of a trainer with the same views and scene
        sizes (re-plans when the sizes differ, e.g. after densification)."""
        self.seed = int(state["seed"])
        self.lr = tuple(state["lr"])
        new = []
        for d in state["scenes"]:
            sb = SceneBuffers(int(d["n"]), d["geom"].to(self.device), d["sh"].to(self.device),
                              d["m"].to(self.device), d["v"].to(self.device),
                              d["stats"].to(self.device) if "stats" in d else None)
            new.append(sb)
        same = [s.n for s in new] == [s.n for s in self.scenes]
        self.scenes = new
        if same:
            gsstep.gs_workspace_set_step(self.plan, self.ws, int(state["step"]))
            self.graph = None
            self._pair = None
        else:
            self._replan(int(state["step"]))

    def _replan(self, step: int):
        p = self.plan
        self.plan = gsstep.Plan([s.n for s in self.scenes], p.views, 0, p.tile, p.bwd_batch, p.storage_flags,
                                p.bwd_impl)
        self.ws = torch.empty(self.plan.workspace_bytes(), dtype=torch.uint8, device=self.device)
        gsstep.gs_workspace_init(self.plan, self.ws)
        gsstep.gs_workspace_set_step(self.plan, self.ws, step)
        self.graph = None
        self._pair = None
