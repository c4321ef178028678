"""Benchmark of the 3DGS training step on GB300.

Default workload: 3M Gaussians (256 clusters in a 30 m box), one 1920x1080
view per step, FP32 storage, 16x16 tiles: project_fwd -> bin_sort ->
raster_fwd -> L1 gradient -> raster_bwd -> project_bwd_adam, captured in one
CUDA graph.  Inputs (parameters, Adam moments, target image, camera) are
resident in HBM when the timed region starts; the working set (about 2.2 GB
of parameters and moments) is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  `--impl reference` times the CPU oracle (FP64, the
plain restatement of the paper's step) on a bounded sample of the same
workload on this host's cores.  With N > 1 (torchrun) every rank trains an
independent replica of the workload on its own GPU (the step has no
exchange between GPUs); value = all ranks' steps / max time.
"""
from __future__ import annotations

import argparse
import json
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
RES = (1920, 1080)
LR = (1.6e-4 * 30.0, 1e-3, 5e-3, 5e-2, 2.5e-3, 2.5e-3 / 20)   # mean lr scaled by the 30 m scene extent


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GAUSS)
    ap.add_argument("--bwd-impl", type=int, default=0, choices=[0, 1],
                    help="raster backward: 0 pixel-parallel warp reductions, 1 per-Gaussian batches")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-sample-tiles", type=int, default=16,
                    help="oracle renders 1 in this many tiles (bounded CPU sample)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(n):
    from paper_2605_00219_gb300 import synth
    scene = synth.large_scene(0, n)
    cam = synth.large_views(1, resolutions=[RES])[0]
    target_scene = synth.perturbed(scene, 1)
    return scene, target_scene, cam


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
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
                "reasons": reasons, "samples": len(rows)}


def run_cpu_oracle(scene, target_img, cam, sample_tiles: int):
    """One oracle step on a bounded sample: projection, FP32 binning, L1 and
    Adam over everything; compositing and its backward on 1 in
    `sample_tiles` tiles.  Returns (seconds for a full step, by scaling the
    tile-bound part, details)."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    p = orc.Params64.from_scene(scene)
    b = orc.bin32(scene, cam)
    P = orc.project64(p, cam)
    t1 = time.perf_counter()
    ntiles = b.ranges.shape[0]
    keep = np.zeros(ntiles, bool)
    keep[::sample_tiles] = True
    bs = orc.Binning(b.count, b.bin, b.mant, b.offset, b.keys_emit, b.gidx_emit, b.keys, b.gidx, b.perm,
                     np.where(keep[:, None], b.ranges, 0))
    r = orc.render64(cam, P, bs)
    loss, (dl,) = orc.l1_loss_grad([r.image], [target_img])
    g2 = orc.raster_bwd64(cam, P, bs, dl)
    t2 = time.perf_counter()
    grad = orc.project_bwd64(p, cam, P, g2)
    th = p.theta()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    orc.adam64(th, m, v, grad, LR, 1)
    t3 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * sample_tiles + (t3 - t2)
    return full, {"measured_s": t3 - t0, "tiles_sampled": int(keep.sum()), "tiles": int(ntiles),
                  "blended_pairs_sampled": r.blended}


def reference_arm(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as orc
    orc.build()
    scene, tscene, cam = _workload(args.n)
    # target from the oracle itself (bounded: the same tile sample)
    target = np.zeros((cam.height, cam.width, 3))
    times = []
    for i in range(args.warmup + args.steps):
        t, info = run_cpu_oracle(scene, target, cam, args.cpu_sample_tiles)
        if i >= args.warmup:
            times.append(t)
    mean = sum(times) / len(times)
    value = 1.0 / mean
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.n // 1_000_000}M Gaussians, one {RES[0]}x{RES[1]} view per step, "
                                   "FP64 CPU oracle", "global_batch": 1, "seq_len": 0, "parallelism": "none"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"compositing and its backward on 1 in {args.cpu_sample_tiles} tiles, "
                                       "scaled to the full image; projection, binning and Adam over all"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2605_00219_gb300 import build
    build.build()
    from paper_2605_00219_gb300 import gsstep, step as stepmod

    scene, tscene, cam = _workload(args.n)
    # target: the perturbed scene rendered by the same forward (setup, untimed)
    tgt_tr = stepmod.Trainer([tscene], [cam], lr=LR)
    tgt_tr.forward()
    target = tgt_tr.image.clone()
    del tgt_tr
    tr = stepmod.Trainer([scene], [cam], lr=LR, bwd_impl=args.bwd_impl)
    tr.target.copy_(target)
    torch.cuda.synchronize()

    # eager warm-up (sets kernel attributes), then graph capture
    tr.step(0)
    tr.capture()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        tr.replay()
    torch.cuda.synchronize()
    st = tr.stats()
    if st.status:
        raise RuntimeError(f"device status {st.status:#x} (k_required={st.k_required}, capacity={st.k_capacity})")

    # ---- timed region: K graph replays
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            tr.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    st = tr.stats()
    blended = int(st.blended_pairs)
    K = int(st.k_required)

    # ---- per-stage timing: the same launches, eager, CUDA events on the stream
    stages = ["project_fwd", "bin_sort", "raster_fwd", "loss_l1", "raster_bwd", "project_bwd_adam"]
    acc = {s: 0.0 for s in stages}
    reps = max(3, min(args.steps, 10))
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
        ev[0].record(stream)
        gsstep.gs_project_fwd(tr.plan, tr.ws, tr.scenes, tr.cams)
        ev[1].record(stream)
        gsstep.gs_bin_sort(tr.plan, tr.ws)
        ev[2].record(stream)
        gsstep.gs_raster_fwd(tr.plan, tr.ws, tr.bg, tr.image)
        ev[3].record(stream)
        gsstep.gs_loss_l1(tr.plan, tr.ws, tr.image, tr.target, tr.dl)
        ev[4].record(stream)
        gsstep.gs_raster_bwd(tr.plan, tr.ws, tr.image, tr.dl)
        ev[5].record(stream)
        gsstep.gs_project_bwd_adam(tr.plan, tr.ws, tr.scenes, tr.cams, gsstep.make_adam(LR, step=0))
        ev[6].record(stream)
        gsstep.gs_adam_advance(tr.plan, tr.ws)
        torch.cuda.synchronize()
        for i, s in enumerate(stages):
            acc[s] += ev[i].elapsed_time(ev[i + 1]) / reps
    nl = tr.buffer(5, tr.plan.pixels).to(torch.int64)
    evaluated = int(nl.sum().item())

    # ---- end to end through the public API with host buffers
    pinned_tgt = target.cpu().pin_memory()
    pinned_cam = tr.cams.cpu().pin_memory()
    loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
    h2d = pinned_tgt.numel() * 4 + pinned_cam.numel() * 4
    loss_dev = tr.ws[:0]  # placeholder, the loss is read from the workspace header
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    f0.record(stream)
    for _ in range(args.steps):
        tr.target.copy_(pinned_tgt, non_blocking=True)
        tr.cams.copy_(pinned_cam, non_blocking=True)
        tr.replay()
        s2 = tr.stats()        # synchronous D2H of the step statistics (loss, status)
        loss_host[0] = s2.loss
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / args.steps
    d2h = 48  # gs_stats header
    del loss_dev

    value = ws * 1e3 / ms
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    n = scene.n
    adam_bytes = n * (240 + 480) * 2 + K * 48 + n * 8
    adam_ms = acc["project_bwd_adam"]
    fwd_bytes = n * 240 + n * (48 + 16 + 4)
    dominant = max(stages, key=lambda s: acc[s])
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    clk_sum = clk.summary()
    alu_peak_tflops = sm_count * 128 * 2 * 2.070e9 / 1e12
    FLOP_BWD, FLOP_FWD = 90.0, 28.0   # FP32 FLOP (FMA = 2) per evaluated pair
    rooflines = {
        "project_bwd_adam": {"bound": "hbm", "achieved": adam_bytes / (adam_ms * 1e-3) / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "traffic": None},
        "project_fwd": {"bound": "hbm", "achieved": fwd_bytes / (acc["project_fwd"] * 1e-3) / 1e9,
                        "peak": hbm_peak, "unit": "GB/s", "traffic": None},
        "raster_bwd": {"bound": "alu", "achieved": evaluated * FLOP_BWD / (acc["raster_bwd"] * 1e-3) / 1e12,
                       "peak": alu_peak_tflops, "unit": "TFLOP/s", "traffic": None},
        "raster_fwd": {"bound": "alu", "achieved": evaluated * FLOP_FWD / (acc["raster_fwd"] * 1e-3) / 1e12,
                       "peak": alu_peak_tflops, "unit": "TFLOP/s", "traffic": None},
    }
    for r in rooflines.values():
        r["frac"] = r["achieved"] / r["peak"]
    dom = dominant if dominant in rooflines else "raster_bwd"
    roof = dict(rooflines[dom])
    roof["kernel"] = dom

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        from oracle import oracle as orc
        orc.build()
        tgt_np = target.view(RES[1], RES[0], 3).cpu().numpy().astype(np.float64)
        t_full, info = run_cpu_oracle(scene, tgt_np, cam, args.cpu_sample_tiles)
        cpu = {"value": 1.0 / t_full, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one oracle step: projection, binning and Adam over all {n} Gaussians, compositing "
                         f"and its backward on {info['tiles_sampled']} of {info['tiles']} tiles, scaled "
                         f"to the full image ({info['measured_s']:.1f} s measured)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"plain FP32 single view: {n / 1e6:.0f}M Gaussians (256 clusters, 30 m box), "
                                   f"one {RES[0]}x{RES[1]} view per step, 16x16 tiles, whole step in one CUDA graph",
                       "global_batch": ws, "seq_len": 0, "parallelism": f"replicas{ws}" if ws > 1 else "none",
                       "l2": "inputs larger than L2 (2.2 GB parameters + moments)"},
            "e2e": {"value": ws * 1e3 / e2e_ms, "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": None,
            "roofline": roof,
            "rooflines": rooflines,
            "stage_ms": acc,
            "intersections": K,
            "blended_pairs_per_s": blended * value / ws,
            "evaluated_pairs": evaluated,
            "views_per_s": value,
            "clocks": clk_sum,
            "cpu_baseline": cpu,
        }
        line["gpu_launches"] = int(args.steps * launches_per_step(tr.plan))
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def launches_per_step(plan) -> int:
    """Kernels of this library launched by one step (see the launchers)."""
    views = len(plan.views)
    key_bits = 0
    for (w, h, _) in plan.views:
        tx, ty = (w + plan.tile[0] - 1) // plan.tile[0], (h + plan.tile[1] - 1) // plan.tile[1]
        tb = max(0, int(np.ceil(np.log2(tx * ty))))
        key_bits = max(key_bits, 32 if tb >= 9 else 23 + tb)
    passes = (key_bits + 7) // 8 + (1 if views > 1 else 0)
    project = 2                         # header reset + projection
    binsort = 3 + 1 + 1 + passes * (1 + 3 + 1) + 1 + 1
    return project + binsort + 1 + 1 + 1 + 1 + 1   # raster fwd, loss, raster bwd, proj bwd+adam, step advance


if __name__ == "__main__":
    main()
