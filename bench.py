"""Benchmark of the 3DGS training step on one GB300.

Headline workload ("batched BF16"): 3M Gaussians (256 clusters in a 30 m
box), four 1920x1080 orbit views per step, SH coefficients and both Adam
moments stored in BF16 (FP32 arithmetic), tile shape and raster-backward
implementation picked by the Thompson-sampling autotuner, the whole step
(projection, binning/sort, raster forward, L1 gradient, raster backward,
projection backward + Adam) in one CUDA graph.

It is compared with the plain FP32 single-view form (same scene, one
1920x1080 view per step, FP32 storage, 16x16 tiles) at an equal number of
1080p views seen: `value` is 1080p view-steps per second (views per step x
steps per second); the plain form's steps/s is reported beside it.  A short
training run of both storage precisions on the same schedule gives the
rendered-PSNR difference on a held-out 1080p view.  `--workload uneven`
runs the batch of four uneven views (1920x1080, 1600x1064, 1280x720,
960x540) instead, `--workload plain` the plain form alone, `--workload
multiscene` eight scenes of 0.5-6M Gaussians (12M in all) with two views
each of mixed resolution (16 views per step, BF16 storage, 16x16 tiles;
no plain comparison, PSNR or CPU baseline).

Inputs (parameters, moments, targets, cameras) are resident in HBM when the
timed region starts; the working set (about 1.5 GB of parameters and
moments plus 2 GB of workspace) is far larger than L2, so no flush is used.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched|uneven|plain|multiscene]

One JSON line on rank 0.  `--impl reference` times the CPU oracle (FP64, the
plain restatement of the paper's step) on a bounded sample of the same
workload on this host's cores.  With N > 1 (torchrun) every rank trains an
independent replica on its own GPU (the step has no exchange between GPUs);
value = all ranks' work / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steps/s (batched BF16 vs plain FP32, ΔPSNR<0.05dB) at 3M Gaussians 1080p"
N_GAUSS = 3_000_000
RES_1080 = (1920, 1080)
BATCH_RES = [(1920, 1080), (1600, 1064), (1280, 720), (960, 540)]
PX_1080 = 1920 * 1080
LR = (1.6e-4 * 30.0, 1e-3, 5e-3, 5e-2, 2.5e-3, 2.5e-3 / 20)   # mean lr scaled by the 30 m scene extent

# DRAM bytes (read + write) of one launch (for the sort: of its launches in
# one step), from ncu DRAM counters of the headline step (3M Gaussians, BF16,
# 4 x 1920x1080, 16x16 tiles, pixel-parallel raster backward).  Valid only
# while the kernel sources hash to the recorded prefixes.
MEASURED_TRAFFIC = {
    "raster_bwd": (3760561664, {"raster_bwd.cu": "1bd9c982611a3a21"}),
    "project_bwd_adam": (3303079168, {"project_bwd_adam.cu": "25d756dbe4558831"}),
    "raster_fwd": (1647618560, {"raster_fwd.cu": "9bbe3a93408bf2b9"}),
    "project_fwd": (1741351168, {"project_fwd.cu": "b375359fd7001cef"}),
    "bin_sort": (1483329536, {"bin_sort.cu": "d92d0a747dcb654f"}),
    "loss_l1": (259586048, {"raster_fwd.cu": "9bbe3a93408bf2b9"}),
}
TRAFFIC_COMMON = {"gs_device.cuh": "89b3b04643ff706e", "gs_internal.cuh": "9a90b6b319a8d190"}


def _measured_traffic(kernel: str, headline: bool):
    """ncu DRAM bytes of `kernel` if its sources are unchanged, else None."""
    import hashlib
    if not headline or kernel not in MEASURED_TRAFFIC:
        return None
    nbytes, files = MEASURED_TRAFFIC[kernel]
    for name, prefix in {**files, **TRAFFIC_COMMON}.items():
        path = os.path.join(ROOT, "paper_2605_00219_gb300", "csrc", name)
        try:
            if hashlib.sha1(open(path, "rb").read()).hexdigest()[:16] != prefix:
                return None
        except OSError:
            return None
    return nbytes


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "uneven", "plain", "multiscene"])
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--tune-rounds", type=int, default=24)
    ap.add_argument("--psnr-steps", type=int, default=200)
    ap.add_argument("--tile", default=None, help="fix the tile shape (e.g. 16x16) instead of autotuning")
    ap.add_argument("--threads-per-tile", type=int, default=0,
                    help="fix the raster threads per tile (0: one per pixel) when the shape is fixed")
    ap.add_argument("--bwd-impl", type=int, default=None, choices=[0, 1, 2],
                    help="fix the raster-backward implementation instead of autotuning")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--fp32", action="store_true",
                    help="FP32 storage for the batched form too (the batched-and-autotuned configuration with "
                         "--workload uneven)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--loss", default="l1", choices=["l1", "l1_ssim"],
                    help="photometric loss of the step: L1 against FP32 targets, or (1 - lambda) L1 + lambda "
                         "(1 - SSIM) with lambda = 0.2 against 8-bit RGBA targets (fixed tile and implementation; "
                         "no plain, PSNR or CPU legs)")
    return ap.parse_args()


def _dist():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest `value` over all ranks of the initialised process group (the
    bench's time is the slowest replica's); the value itself with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, views_per_step: int, ms_per_step: float) -> float:
    """Views trained per second by all replicas (each rank one replica)."""
    return world * views_per_step * 1e3 / ms_per_step


def _views(workload):
    from paper_2605_00219_gb300 import synth
    if workload == "plain":
        return synth.large_views(1, resolutions=[RES_1080])
    if workload == "uneven":
        return synth.large_views(4, resolutions=BATCH_RES)
    return synth.large_views(4, resolutions=[RES_1080])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms from the
    moment the first sample has arrived (entered before the warm-up, left
    after the timed region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu, self.period, self.proc, self.lines = gpu_index, period_ms, None, []
        self.reader = None

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        first = threading.Event()

        def read():
            for line in self.proc.stdout:
                self.lines.append(line)
                first.set()
        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        first.wait(5.0)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            if self.reader is not None:
                self.reader.join(timeout=5)
        return False

    def summary(self):
        rows = []
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "period_ms": self.period,
                "window": "warm-up and timed replays"}


# ----------------------------------------------------------------------------
# CPU oracle (bounded sample)
# ----------------------------------------------------------------------------

def _oracle_target(orc, tscene, cam):
    """Target image of one view rendered by the oracle from the target scene
    (no input of the oracle comes from the CUDA path)."""
    return orc.render64(cam, orc.project64(orc.Params64.from_scene(tscene), cam), orc.bin32(tscene, cam)).image


def time_oracle_step(orc, scene, cams, targets, lr):
    """Wall-clock seconds of one full, un-sampled oracle step over `cams`
    (FP32 binning, FP64 projection, compositing, L1 gradient, compositing and
    projection backward, one Adam update over every Gaussian)."""
    t0 = time.perf_counter()
    r = orc.step(scene, cams, targets, lr)
    return time.perf_counter() - t0, sum(x.blended for x in r.renders)


def cpu_baseline_leg(scene, tscene, cams):
    """The oracle timed on this host: one full step over the first view of
    the measured workload (all Gaussians, every tile), on all cores; and the
    tiny and mid-size configurations (2,000 Gaussians at 128x128; 200k at
    1280x720, one orbit view per step) on one thread and on all cores."""
    from oracle import oracle as orc
    from paper_2605_00219_gb300 import synth
    orc.build()
    cores = orc.set_threads(os.cpu_count() or 1)
    cam = cams[0]
    tgt = _oracle_target(orc, tscene, cam)
    t, blended = time_oracle_step(orc, scene, [cam], [tgt], LR)
    out = {"value": 1.0 / t, "unit": "view-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"one full oracle step over 1 of the {len(cams)} views ({cam.width}x{cam.height}, all "
                     f"{scene.n} Gaussians, every tile, L1 against an oracle-rendered target, Adam over every "
                     f"Gaussian): {t:.1f} s measured, not scaled",
           "blended_pairs_per_s": blended / t, "configs": {}}
    small = {"tiny: 2,000 Gaussians, 128x128": synth.tiny_workload(0),
             "mid: 200k Gaussians, 1280x720": synth.mid_workload(0)}
    for name, (sc, tsc, cs) in small.items():
        c = cs[0]
        tg = _oracle_target(orc, tsc, c)
        lr = (1e-3,) * 6 if sc.n < 10000 else LR
        row = {}
        for label, threads in (("1_thread", 1), ("all_cores", cores)):
            orc.set_threads(threads)
            reps = 5 if sc.n < 10000 else 1
            best = min(time_oracle_step(orc, sc, [c], [tg], lr)[0] for _ in range(reps))
            row[label] = {"s_per_step": best, "steps_per_s": 1.0 / best, "threads": threads}
        out["configs"][name] = row
    orc.set_threads(cores)
    return out


def reference_arm(args):
    """The oracle on this host's cores, as the reference arm: each step is one
    full, un-sampled oracle step over one view of the workload (rotating
    through its views), against oracle-rendered targets from the same target
    scene.  A step takes tens of seconds, so at most 3 timed steps and 1
    warm-up step run; the line reports the counts that ran."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2605_00219_gb300 import synth
    orc.build()
    cores = orc.set_threads(os.cpu_count() or 1)
    scene = synth.large_scene(0, args.n)
    tscene = synth.perturbed(scene, 1)
    cams = _views(args.workload)
    steps = max(1, min(args.steps, 3))
    warm = min(args.warmup, 1)
    used = [cams[i % len(cams)] for i in range(warm + steps)]
    targets = {id(c): _oracle_target(orc, tscene, c) for c in used}
    times, blended = [], 0
    for i, c in enumerate(used):
        t, b = time_oracle_step(orc, scene, [c], [targets[id(c)]], LR)
        if i >= warm:
            times.append(t)
            blended += b
    mean = sum(times) / len(times)
    value = 1.0 / mean
    sample = (f"{steps} timed and {warm} warm-up steps (of the requested {args.steps} and {args.warmup}); each "
              f"one full oracle step over one of the {len(cams)} views, all {scene.n} Gaussians, every tile, "
              f"not scaled")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "view-steps/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {args.n / 1e6:.3g}M Gaussians, views "
                                   f"{[f'{c.width}x{c.height}' for c in cams]}, one view per oracle step; FP64 "
                                   "CPU oracle; value in view-steps/s", "global_batch": 1, "seq_len": 0,
                       "parallelism": "none"},
            "cpu_baseline": {"value": value, "unit": "view-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "blended_pairs_per_s": blended / sum(times)},
            "e2e": {"value": value, "unit": "view-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def _render_targets(stepmod, tscene, cams):
    tr = stepmod.Trainer([tscene], cams, lr=LR)
    tr.forward()
    out = tr.image.clone()
    del tr
    return out


def _time_replays(torch, tr, steps, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        tr.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _rgba8(torch, flat):
    """FP32 (P, 3) images in [0, 1] -> 8-bit RGBA (P, 4), alpha 255."""
    rgb = (flat * 255.0).round().clamp(0, 255).to(torch.uint8)
    return torch.cat([rgb, torch.full_like(rgb[:, :1], 255)], dim=1)


def _stage_times(torch, gsstep, tr, reps, stream):
    loss_stage = "loss_l1" if tr.loss == "l1" else "loss_l1_ssim"
    stages = ["project_fwd", "bin_sort", "raster_fwd", loss_stage, "raster_bwd", "project_bwd_adam"]
    acc = {s: 0.0 for s in stages}
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
        ev[0].record(stream)
        gsstep.gs_project_fwd(tr.plan, tr.ws, tr.scenes, tr.cams)
        ev[1].record(stream)
        gsstep.gs_bin_sort(tr.plan, tr.ws)
        ev[2].record(stream)
        gsstep.gs_raster_fwd(tr.plan, tr.ws, tr.bg, tr.image)
        ev[3].record(stream)
        if tr.loss == "l1":
            gsstep.gs_loss_l1(tr.plan, tr.ws, tr.image, tr.target, tr.dl)
        else:
            gsstep.gs_loss_l1_ssim(tr.plan, tr.ws, tr.image, tr.target, tr.ssim_lambda, tr.dl)
        ev[4].record(stream)
        gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
        ev[5].record(stream)
        gsstep.gs_project_bwd_adam(tr.plan, tr.ws, tr.scenes, tr.cams, gsstep.make_adam(tr.lr, step=0))
        ev[6].record(stream)
        gsstep.gs_adam_advance(tr.plan, tr.ws)
        torch.cuda.synchronize()
        for i, s in enumerate(stages):
            acc[s] += ev[i].elapsed_time(ev[i + 1]) / reps
    return acc


def _psnr(torch, img, ref):
    mse = float(((img.double() - ref.double()) ** 2).mean().item())
    return 10.0 * math.log10(1.0 / max(mse, 1e-30))


def _psnr_run(torch, stepmod, synth, scene, cams, targets, tile, impl, tpt, bf16, steps, heldout_cam,
              heldout_tgt):
    """Train `steps` steps from `scene` and return the held-out view's PSNR."""
    tr = stepmod.Trainer([scene], cams, lr=LR, tile=tile, bwd_impl=impl, sh_bf16=bf16, mom_bf16=bf16,
                         threads_per_tile=tpt)
    tr.target.copy_(targets)
    for _ in range(steps):
        tr.step(0)
    ev = stepmod.Trainer([tr.scenes[0]], [heldout_cam], lr=LR, tile=tile, bwd_impl=impl, threads_per_tile=tpt,
                         sh_bf16=bf16, mom_bf16=bf16)
    ev.forward()
    torch.cuda.synchronize()
    return _psnr(torch, ev.image, heldout_tgt), float(tr.stats().loss)


def main():
    args = _args()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import autotune, gsstep, synth
    from paper_2605_00219_gb300 import step as stepmod

    stream = torch.cuda.current_stream()
    if args.loss != "l1":
        args.no_plain, args.psnr_steps, args.no_cpu = True, 0, True
        if args.tile is None and args.bwd_impl is None:
            args.tile = "16x16"
    multi = args.workload == "multiscene"
    if multi:
        # eight scenes of 0.5-6M Gaussians with two views each, one step
        import dataclasses
        scenes, cams = synth.multi_scene_workload()
        scene = scenes[-1]
        targets = torch.cat([_render_targets(stepmod, synth.perturbed(sc, k + 1),
                                             [dataclasses.replace(c, scene=0) for c in cams if c.scene == k])
                             for k, sc in enumerate(scenes)])
        args.no_plain, args.psnr_steps, args.no_cpu = True, 0, True
        if args.tile is None:
            args.tile = "16x16"
    else:
        scene = synth.large_scene(0, args.n)
        tscene = synth.perturbed(scene, 1)
        cams = _views(args.workload)
        targets = _render_targets(stepmod, tscene, cams)
        scenes = [scene]
    batched = args.workload != "plain"
    px = sum(c.width * c.height for c in cams)
    equiv = px / PX_1080
    nviews = len(cams)

    # ---- plain FP32 single view (reference form of the comparison)
    plain_ms = None
    if not args.no_plain:
        plain_cam = synth.large_views(1, resolutions=[RES_1080])[0]
        plain_tgt = _render_targets(stepmod, tscene, [plain_cam])
        plain = stepmod.Trainer([scene], [plain_cam], lr=LR)
        plain.target.copy_(plain_tgt)
        plain.step(0)
        plain.capture()
        for _ in range(args.warmup):
            plain.replay()
        torch.cuda.synchronize()
        plain_ms = _time_replays(torch, plain, args.steps, stream)
        del plain

    # ---- the measured form
    sh16 = batched and not args.fp32
    all_bufs = [stepmod.SceneBuffers.from_scene(sc, sh_bf16=sh16, mom_bf16=sh16) for sc in scenes]
    bufs = all_bufs[0]
    fixed = args.tile is not None or args.bwd_impl is not None
    if batched and not fixed:
        best, tuner, trainers = autotune.tune_trainer([bufs], cams, rounds=args.tune_rounds, lr=LR, sh_bf16=sh16,
                                                      mom_bf16=sh16, target=targets)
        tr = trainers[best]
        for c, t in list(trainers.items()):
            if c != best:
                del trainers[c]
        tile, impl, tpt = best
        tune_info = {"chosen": {"tile": list(tile), "bwd_impl": impl, "threads_per_tile": tpt},
                     "pulls": {autotune.describe(c): n for c, n in zip(tuner.candidates, tuner.pulls)},
                     "mean_ms": {autotune.describe(c): round(p.mean, 3)
                                 for c, p in zip(tuner.candidates, tuner.post) if p.n}}
    else:
        tile = tuple(int(x) for x in args.tile.split("x")) if args.tile else (16, 16)
        impl = args.bwd_impl if args.bwd_impl is not None else 0
        tpt = args.threads_per_tile or tile[0] * tile[1]
        tr = stepmod.Trainer(all_bufs, cams, lr=LR, tile=tile, bwd_impl=impl, sh_bf16=sh16, mom_bf16=sh16,
                             loss=args.loss, threads_per_tile=tpt)
        tr.target.copy_(targets if args.loss == "l1" else _rgba8(torch, targets))
        tr.step(0)
        tune_info = None
    tr.capture()
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            tr.replay()
        torch.cuda.synchronize()
        st = tr.stats()
        if st.status:
            raise RuntimeError(f"device status {st.status:#x} (k_required={st.k_required}, "
                               f"capacity={st.k_capacity})")
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = _time_replays(torch, tr, args.steps, stream)
    if ws > 1:
        ms = max_over_ranks(ms, "cuda")
        torch.distributed.barrier()
    st = tr.stats()
    K = int(st.k_required)
    blended = int(st.blended_pairs)

    acc = _stage_times(torch, gsstep, tr, max(3, min(args.steps, 10)), stream)
    evaluated = int(tr.buffer(5, tr.plan.pixels).to(torch.int64).sum().item())

    # ---- end to end: host targets and cameras in, statistics out, every step
    pinned_tgt = tr.target.cpu().pin_memory()
    pinned_cam = tr.cams.cpu().pin_memory()
    h2d = pinned_tgt.numel() * pinned_tgt.element_size() + pinned_cam.numel() * pinned_cam.element_size()
    # two graphs over two input buffer sets: step k's host copy runs on a side
    # stream while step k - 1 computes; every step still copies its own inputs
    # from pinned host memory and reads its statistics back
    tr.capture_pair()
    tr.run_from_host(lambda k: pinned_tgt, lambda k: pinned_cam, max(args.warmup, 2))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    tr.run_from_host(lambda k: pinned_tgt, lambda k: pinned_cam, args.steps)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / args.steps
    d2h = 48

    # ---- rendered-PSNR difference, FP32 vs BF16 storage, same schedule
    psnr = None
    if args.psnr_steps > 0 and rank == 0:
        held = synth.large_views(1, resolutions=[RES_1080], phase_deg=45.0)[0]
        held_tgt = _render_targets(stepmod, tscene, [held])
        p32, l32 = _psnr_run(torch, stepmod, synth, scene, cams, targets, tile, impl, tpt, False, args.psnr_steps, held,
                             held_tgt)
        p16, l16 = _psnr_run(torch, stepmod, synth, scene, cams, targets, tile, impl, tpt, True, args.psnr_steps, held,
                             held_tgt)
        psnr = {"steps": args.psnr_steps, "fp32_db": p32, "bf16_db": p16, "delta_db": abs(p16 - p32),
                "loss_fp32": l32, "loss_bf16": l16, "heldout": "1920x1080 orbit view at +45 deg"}

    # ---- roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    n = sum(sc.n for sc in scenes)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sm_count * 128 * 2 * 2.070e9 / 1e12
    work = stage_work([sc.n for sc in scenes], [c.scene for c in cams], K, evaluated, blended, px,
                      int(tr.plan.tiles), sh16, args.loss)
    rooflines = stage_rooflines(work, acc, hbm_peak, alu_peak)
    headline = (args.workload == "batched" and args.n == N_GAUSS and tuple(tile) == (16, 16) and impl == 0
                and tpt == 128
                and args.loss == "l1")
    for k, r in rooflines.items():
        r["traffic"] = _measured_traffic(k, headline)
    dom = max(rooflines, key=lambda k: acc[k])
    roof = dict(rooflines[dom])
    roof["kernel"] = dom

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline_leg(scene, tscene, cams)

    if rank == 0:
        value = whole_job_rate(ws, nviews, ms)
        desc = ("multi-scene BF16: 8 scenes of " + "/".join(f"{sc.n / 1e6:.3g}" for sc in scenes) +
                f"M Gaussians ({n / 1e6:.3g}M in all), views per step " if multi else
                (("batched BF16: " if sh16 else "batched FP32: ") if batched else "plain FP32: ") +
                f"{n / 1e6:.3g}M Gaussians (256 clusters, 30 m box), views per step ") + \
               "+".join(f"{c.width}x{c.height}" for c in cams) + \
               (", BF16 SH and Adam moments (FP32 math)" if sh16 else ", FP32 storage") + \
               f", tile {tile[0]}x{tile[1]}, raster_bwd impl {impl}, {tpt} threads per tile, " + \
               ("L1 loss" if args.loss == "l1" else "0.8 L1 + 0.2 (1 - SSIM) loss against 8-bit RGBA targets") + \
               ", whole step in one CUDA graph; value = " + \
               f"view-steps/s ({nviews} views per step x steps/s; {equiv:.3f} 1080p-equivalents of pixels per step)"
        line = {
            "metric": METRIC, "value": value, "unit": "view-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "global_batch": ws * len(cams), "seq_len": 0,
                       "parallelism": f"replicas{ws}" if ws > 1 else "none",
                       "l2": "inputs larger than L2 (no flush)",
                       "storage": "BF16 SH and Adam moments, FP32 geometry" if sh16 else "FP32",
                       "views_per_step": nviews},
            "e2e": {"value": ws * nviews * 1e3 / e2e_ms, "unit": "view-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(args.steps * launches_per_step(tr.plan)),
            "roofline": roof,
            "rooflines": rooflines,
            "plain_fp32": None if plain_ms is None else {
                "steps_per_s": 1e3 / plain_ms, "ms_per_step": plain_ms,
                "workload": "one 1920x1080 view per step, FP32 storage, 16x16 tiles, impl 0"},
            "batched_steps_per_s": 1e3 / ms,
            "views_per_s": nviews * 1e3 / ms,
            "equiv_1080p_views_per_s": equiv * 1e3 / ms,
            "speedup_vs_plain_fp32": None if plain_ms is None else (nviews * 1e3 / ms) / (1e3 / plain_ms),
            "psnr": psnr,
            "autotune": tune_info,
            "stage_ms": acc,
            "intersections": K,
            "evaluated_pairs": evaluated,
            "blended_pairs": blended,
            "tiles": int(tr.plan.tiles),
            "pixels": int(px),
            "blended_pairs_per_s": blended * 1e3 / ms,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "memory_gib": {
                "workspace": tr.ws.numel() / 2 ** 30,
                "scene_buffers": sum(t.numel() * t.element_size() for sb in tr.scenes
                                     for t in (sb.geom, sb.sh, sb.m, sb.v) if t is not None) / 2 ** 30,
                "images_targets_gradients": 3 * tr.image.numel() * 4 / 2 ** 30,
            },
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# FP32 operations per pair of the raster kernels.  Every pair inside a
# pixel's n_last is evaluated (pixel offset, exponent, the 3-sigma and 1/255
# tests: 14 operations and one ex2); a blended pair costs more on top: the
# forward's compensated transmittance product, stop test and colour FMAs (13),
# the backward's compensated division, dL/dalpha and the nine gradient terms
# with their accumulation (31, the rest of the backward's 45 per pair).  An
# operation occupies one FP32-pipe lane slot; it is counted as 2 FLOP, like
# the FMA in the peak (SMs x 128 lanes x 2 x clock).
OPS_TEST, OPS_BLEND_FWD, OPS_BLEND_BWD = 14, 13, 31
SSIM_OPS = 209                    # FP32 operations per pixel and channel of the L1 + SSIM loss


def stage_work(scene_sizes, view_scenes, K, evaluated, blended, px, tiles, sh16, loss="l1"):
    """Algorithmic work of each stage of one step, as (bound, amount): bytes
    for the HBM-bound stages, FP32 FLOP (2 per operation) for the ALU-bound
    ones.  Per-unit figures are the method's, not this layout's: padding,
    the separate binning record and record gathers wider than the data are
    not counted.

    scene_sizes: Gaussians per scene; view_scenes: the scene of each view (a
    view pairs with the Gaussians of its own scene); K: intersections;
    evaluated: pairs within every pixel's n_last; blended: pairs composited;
    px: pixels of all views; tiles: tiles of all views."""
    n = sum(scene_sizes)
    pairs = sum(scene_sizes[s] for s in view_scenes)
    # projection: parameters read once per step for all views (44 B of
    # geometry + 48 SH coefficients: 236 B FP32, 140 B with BF16 SH); 48 B
    # written per (view, Gaussian) pair (mean, conic, opacity, colour, depth,
    # tile count)
    fwd_bytes = n * (140 if sh16 else 236) + pairs * 48
    # fused Adam: the 59 parameters and both moments read and written
    # (2 x (236 + 472) = 1416 B FP32; 2 x (140 + 236) = 752 B with BF16 SH
    # and moments), a 36-byte gradient (9 floats) read per intersection, and
    # each pair's count and offset
    adam_bytes = n * (752 if sh16 else 1416) + K * 36 + pairs * 8
    # sort: the count scan (4 B in, 4 B out per pair), emission (count and
    # offset read per pair), and the floor for sorting: one 8-byte key and
    # value written and read once per intersection; 8 B of range per tile.
    # The buckets, the per-tile merge passes and the pair gathers of this
    # implementation are not counted.
    sort_bytes = pairs * 16 + K * 16 + tiles * 8
    work = {
        "project_bwd_adam": ("hbm", adam_bytes),
        "project_fwd": ("hbm", fwd_bytes),
        "raster_bwd": ("alu", 2.0 * (evaluated * OPS_TEST + blended * OPS_BLEND_BWD)),
        "raster_fwd": ("alu", 2.0 * (evaluated * OPS_TEST + blended * OPS_BLEND_FWD)),
        "bin_sort": ("hbm", sort_bytes),
    }
    if loss == "l1":
        # image and gradient (FP32 RGB) and the FP32 RGB target
        work["loss_l1"] = ("hbm", px * (12 + 12 + 12))
    else:
        # ALU-bound: per pixel and channel, 11 taps of the horizontal pass
        # (5 moment FMAs + 3 products) and of the vertical pass (5 FMAs), and
        # 11 taps of both passes of the 3 partials (3 FMAs each): 209 FP32
        # operations, the window halo not counted
        work["loss_l1_ssim"] = ("alu", px * 3 * SSIM_OPS * 2)
    return work


def stage_rooflines(work, stage_ms, hbm_peak_gbs, alu_peak_tflops):
    """Roofline record of each stage: its algorithmic work (stage_work) over
    its measured time in ms, against the HBM or FP32 peak."""
    out = {}
    for k, (bound, amount) in work.items():
        sec = stage_ms[k] * 1e-3
        if bound == "hbm":
            r = {"bound": "hbm", "achieved": amount / sec / 1e9, "peak": hbm_peak_gbs, "unit": "GB/s"}
        else:
            r = {"bound": "alu", "achieved": amount / sec / 1e12, "peak": alu_peak_tflops, "unit": "TFLOP/s"}
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = None
        out[k] = r
    return out


def launches_per_step(plan) -> int:
    """Kernels of this library launched by one step (see the launchers)."""
    project = 2                                        # header reset + projection
    binsort = 3 + 3 + 1 + 1 + 2                        # count scan (with K and the capacity check), tile scan
                                                       # (with the ranges), order, emit, sort (long and short
                                                       # lists)
    return project + binsort + 1 + 1 + 1 + 1 + 1       # raster fwd, loss, raster bwd, proj bwd+adam, advance


if __name__ == "__main__":
    main()
