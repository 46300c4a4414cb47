#!/usr/bin/env python
"""Calibration iterations per second of the differentiable splatting path.

One iteration ("step") = the whole hot path for every frame of the batch:
camera poses (Eq. 1), projection (Eq. 2-3), tile binning + depth sort,
compositing (Phi, Eq. 5), L1 loss (Eq. 4) and its gradient, the reverse
compositing backward, the projection backward and the gradient w.r.t. the
extrinsic and the time offset.  The optimiser step is not included.

Workload (default): 1,000,000 LiDAR-anchored Gaussians accumulated from 50
synthetic 64-beam sweeps along a 10 m/s drive; 8 camera frames of 1408x376;
the current extrinsic perturbed by 5 deg / 0.5 m and the time offset by
50 ms from the one the target images were rendered with.  The batched path
is one CUDA-graph replay per iteration; the per-frame path launches the
same kernels frame by frame.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
"""
import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "calib iters/s (fwd+bwd, 8×1408×376, 1M Gaussians) batched vs per-frame"
WORKLOAD = "1M LiDAR-anchored Gaussians (50 synthetic 64-beam sweeps, 10 m/s drive), 8 frames 1408x376"


def workload_label(n, frames):
    """The batched workload's description for a run at n Gaussians and
    `frames` frames (the headline label at the defaults)."""
    if n == 1_000_000 and frames == 8:
        return WORKLOAD
    ns = "%gM" % (n / 1e6) if n >= 1_000_000 else "%gK" % (n / 1e3)
    return ("%s LiDAR-anchored Gaussians (50 synthetic 64-beam sweeps, 10 m/s drive), %d frame%s 1408x376"
            % (ns, frames, "" if frames == 1 else "s"))
# Arithmetic per composited (pixel, Gaussian) pair, i.e. per pair with
# alpha >= alpha_min before the pixel stops (Eq. 5).  The roofline uses the
# planned per-pair figures: about 20 flop (and one 2^x) forward and three
# times that backward.  A recount of the kernels' own arithmetic, comparisons
# not counted, is reported beside them:
# forward: dx, dy (2), exponent (7), + log2 o (1), 2^e and the alpha clamp (2),
# 1 - alpha (1), T (1 - alpha) (1), alpha T (1), colour (3 fma = 6): 21;
# backward: the same exponent and alpha (12), 1 - alpha, 1/(1 - alpha), T
# recovery (3), alpha T (1), c . g (5), dL/dalpha (3), light behind (2),
# dL/de (1), de dx, de dy (2), dA, dB, dC (6), sums for the mean and F (3),
# colour gradient (6): 44.
FLOP_PER_PAIR_FWD, FLOP_PER_PAIR_BWD = 20.0, 60.0
RECOUNT_PER_PAIR_FWD, RECOUNT_PER_PAIR_BWD = 21.0, 44.0
# oracle sample per frame for the CPU baseline, the same in both arms
CPU_PIXELS = 40
L2_NOTE = "inputs larger than L2: each iteration's workspace (GBs) exceeds the 129 MB L2"
KERNEL_NAMES = {1: "project", 2: "bin_sort", 3: "render_fwd", 4: "render_bwd", 5: "project_bwd", 6: "loss"}
KERNEL_SOURCES = {1: "project.cu", 2: "binsort.cu", 3: "render.cu", 4: "render.cu", 5: "project.cu",
                  6: "loss.cu"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--gaussians", type=int, default=1_000_000)
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--per-frame-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper-loop", action="store_true",
                    help="skip the second measurement: L_photo (with D-SSIM) on the bottom half of every frame")
    ap.add_argument("--cpu-pixels", type=int, default=CPU_PIXELS, help="oracle pixels per frame sample")
    ap.add_argument("--autotune", action="store_true", help="pick tile/batch with the autotuner first")
    ap.add_argument("--workload", choices=["batched", "uneven"], default="batched",
                    help="batched: 1M Gaussians, 8 frames 1408x376 (the headline); uneven: three scenes "
                         "of 300k/1M/3M Gaussians with 4 frames each at 704x188/1408x376/1920x1080")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest value of x over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------- CPU oracle leg

def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "model": model}


def oracle_c1_loop(iters=30):
    """The oracle's calibration loop on the 64-Gaussian 64x48 scene, unsampled:
    `iters` iterations of the forward of every pixel, the L1 loss against the
    target render and the backward of every pixel (one thread)."""
    import oracle
    from paper_2403_11577_gb300 import scenes
    p = scenes.tiny_problem()
    f, sc = p.frames[0], p.scenes[0]
    tgt = oracle.render(sc, f, p.ext_target[0], 0.0)[0]
    t0 = time.perf_counter()
    for _ in range(iters):
        rgb = oracle.render(sc, f, p.ext[0], 0.0)[0]
        _, g = oracle.l1(rgb, tgt)
        oracle.backward(sc, f, p.ext[0], 0.0, g)
    secs = time.perf_counter() - t0
    return {"iters": iters, "seconds": secs, "value": iters / secs, "unit": "iters/s",
            "workload": "64 Gaussians, one 64x48 frame, L1 against the target render, every pixel"}


def oracle_iteration_seconds(problem, pixels_per_frame, frame_ids, seed=0):
    """Seconds the FP64 oracle needs for one calibration iteration over the
    whole workload, extrapolated from a bounded sample: for each frame in
    frame_ids, the projection + depth sort, the forward of `pixels_per_frame`
    sampled pixels and the backward of those pixels are timed; per-pixel
    costs are scaled to all pixels of all frames."""
    import oracle
    rng = np.random.default_rng(seed)
    per_frame_fixed, per_pixel, sample_s = [], [], 0.0
    for fi in frame_ids:
        f = problem.frames[fi]
        sc = problem.scenes[f.scene_id]
        e, d = problem.ext[f.camera_id], float(problem.delta[f.camera_id])
        cam = f.camera
        one = np.array([[cam.width // 2, cam.height // 2]])
        pix = np.stack([rng.integers(0, cam.width, pixels_per_frame),
                        rng.integers(0, cam.height, pixels_per_frame)], 1)
        t0 = time.perf_counter()
        oracle.render(sc, f, e, d, pixels=one)
        t1 = time.perf_counter()
        oracle.render(sc, f, e, d, pixels=pix)
        t2 = time.perf_counter()
        oracle.backward(sc, f, e, d, np.ones((1, 3)), pixels=one)
        t3 = time.perf_counter()
        oracle.backward(sc, f, e, d, np.ones((len(pix), 3)), pixels=pix)
        t4 = time.perf_counter()
        fixed = (t1 - t0) + (t3 - t2)
        per_frame_fixed.append(fixed)
        per_pixel.append(max(((t2 - t1) - (t1 - t0)) + ((t4 - t3) - (t3 - t2)), 0.0) / pixels_per_frame)
        sample_s += t4 - t0
    n_pix = sum(f.camera.width * f.camera.height for f in problem.frames)
    total = np.mean(per_frame_fixed) * len(problem.frames) + np.mean(per_pixel) * n_pix
    return total, sample_s


# ---------------------------------------------------------- our path

UNEVEN = "3 scenes: 300k/1M/3M LiDAR-anchored Gaussians, 4 frames each at 704x188/1408x376/1920x1080"


def build_problem(args):
    """The workload; targets are rendered at ext_target/delta_target, the
    iteration runs at ext/delta (5 deg, 0.5 m, 50 ms away)."""
    from paper_2403_11577_gb300 import scenes
    if args.workload == "uneven":
        p = scenes.uneven_problem()
        rng = np.random.default_rng(7)
        p.ext_target, p.delta_target = p.ext.copy(), np.zeros(p.num_cameras)
        p.ext = p.ext + np.concatenate([rng.normal(0, 0.05, (p.num_cameras, 3)),
                                        rng.normal(0, 0.3, (p.num_cameras, 3))], 1)
        p.delta = np.full(p.num_cameras, 0.05)
        return p
    return scenes.calibration_problem(seed=0, n=args.gaussians, frames=args.frames)


def bench_config(args, problem, opts=None):
    """The workload's description, identical in both arms."""
    n = sum(sc.n for sc in problem.scenes)
    fr = len(problem.frames)
    batched = args.workload == "batched"
    return {"workload": workload_label(n, fr) if batched else UNEVEN, "gaussians": n, "frames": fr,
            "image": "1408x376" if batched else "704x188/1408x376/1920x1080",
            "tile": opts.tile if opts else args.tile, "batch": opts.batch if opts else args.batch,
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "single",
            "l2": L2_NOTE}


def source_sha(kernel_id):
    path = os.path.join(ROOT, "paper_2403_11577_gb300", "csrc", KERNEL_SOURCES[kernel_id])
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def load_traffic(kernel_id):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or
    None if missing or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = d.get(KERNEL_NAMES[kernel_id])
    if not ent or ent.get("source_sha") != source_sha(kernel_id):
        return None
    return ent.get("bytes_per_launch_full")


def paper_loop(args, problem, scene, opts, ext, delta, ext_t, delta_t, dev, world):
    """Calibration iterations/s with L_photo (lambda1 = 0.2) on the bottom
    half of the frames, timed like the main metric (graph replays)."""
    import copy
    import dataclasses

    import torch

    from paper_2403_11577_gb300 import capi, render
    pc = copy.copy(problem)
    pc.frames = [dataclasses.replace(f, row0=f.camera.height // 2) for f in problem.frames]
    frames = render.Plan.frames_from_problem(pc, scene)
    cap = render.default_pair_capacity(frames, opts.tile)
    while True:
        plan = render.Plan(frames, scene.n, pc.num_cameras, len(pc.scenes), opts, cap, dev)
        plan.forward(scene, ext_t, delta_t)
        st = plan.stats()
        plan.forward(scene, ext, delta)
        if not (st.status | plan.stats().status) & capi.GS_DEV_PAIR_OVERFLOW:
            break
        cap = int(min(cap * 2, (1 << 32) - 1))
    plan.forward(scene, ext_t, delta_t)
    target = plan.rgb.clone()
    step = render.CalibStep(plan, scene, target, ext, delta, graph=True, loss="photo")
    for _ in range(args.warmup):
        step()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        step()
    b.record()
    torch.cuda.synchronize()
    t = max_over_ranks(a.elapsed_time(b) / 1e3, world)
    la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    capi.gs_profile_events(capi.GS_PROF_LOSS, la, lb)
    ts = []
    for _ in range(3):
        step._body()
        torch.cuda.synchronize()
        ts.append(la.elapsed_time(lb))
    capi.gs_profile_events(capi.GS_PROF_NONE)
    loss = step.loss.cpu().numpy()
    pairs = int(plan.stats().num_pairs)
    # voxel downsampling of the scene's points at the finest voxel of the
    # paper's schedule (2 cm), timed alone
    va, vb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vox = []
    for _ in range(3):
        va.record()
        kept = render.voxel_downsample(scene.X, 0.02)
        vb.record()
        torch.cuda.synchronize()
        vox.append(va.elapsed_time(vb))
    # the attribute model F(X | Theta) (hash-grid MLP) over the 2 cm voxel points
    from paper_2403_11577_gb300 import ngp
    Xk = scene.X[kept].contiguous()
    mlp = ngp.HashGridMLP(ngp.HashGridConfig.for_points(scene.X), device=dev)
    attrs = {"rgb": torch.empty_like(Xk), "logit_opacity": torch.empty(Xk.shape[0], device=dev),
             "log_scale": torch.empty_like(Xk), "quat": torch.empty((Xk.shape[0], 4), device=dev)}
    grads = {k: torch.randn_like(v) for k, v in attrs.items()}
    tf, tb = [], []
    for _ in range(4):
        va.record()
        mlp.forward(Xk, attrs)
        vb.record()
        torch.cuda.synchronize()
        tf.append(va.elapsed_time(vb))
        va.record()
        mlp.backward(Xk, grads)
        vb.record()
        torch.cuda.synchronize()
        tb.append(va.elapsed_time(vb))
    # the paper's whole iteration with the attribute model in the loop: F(X | Theta)
    # writes the scene's attributes, the graph renders and back-propagates
    # L_photo, and the MLP backward carries the attribute gradients into Theta
    # (the optimiser excluded, as above)
    mlp_full = ngp.HashGridMLP(ngp.HashGridConfig.for_points(scene.X), device=dev)
    live = {k: getattr(scene, k) for k in ("rgb", "logit_opacity", "log_scale", "quat")}

    def mlp_iter():
        mlp_full.forward(scene.X, live)
        step()
        mlp_full.backward(scene.X, step.grads)

    for _ in range(args.warmup):
        mlp_iter()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        mlp_iter()
    b.record()
    torch.cuda.synchronize()
    t_mlp = max_over_ranks(a.elapsed_time(b) / 1e3, world)
    return {"value": world * args.steps / t, "unit": "iters/s", "ms_per_step": t * 1e3 / args.steps,
            "with_mlp": {"value": world * args.steps / t_mlp, "unit": "iters/s",
                         "ms_per_step": t_mlp * 1e3 / args.steps,
                         "what": "F(X | Theta) forward over the 1M Gaussians, the graph above, F backward"},
            "voxel_downsample_ms": statistics.median(vox), "voxel_kept_2cm": int(kept.numel()),
            "ngp_forward_ms": statistics.median(tf[1:]), "ngp_backward_ms": statistics.median(tb[1:]),
            "loss": "L_photo = 0.8 L1 + 0.2 D-SSIM (11x11 Gaussian window), rows 188-375 of each 1408x376 frame",
            "loss_ms": statistics.median(ts), "pairs_per_iter": pairs,
            "l_photo": float(loss[0]), "l1": float(loss[1]), "dssim": float(loss[2])}


def adam_steps(args, step, scene, ext, delta):
    """The timed iteration followed by one Adam step, as the calibration loop
    runs it: torch's Adam on the Gaussians' attributes (their gradients are
    the graph's own output buffers) and on the extrinsic rotation,
    translation and delta, whose new values go back into the graph's static
    pose inputs.  Timed like the main metric; the parameters are restored
    afterwards."""
    import torch

    from paper_2403_11577_gb300.calib import GAUSS_LR
    keys = list(GAUSS_LR)
    saved = {k: getattr(scene, k).clone() for k in keys}
    ext0, delta0 = ext.clone(), delta.clone()
    for k in keys:
        getattr(scene, k).grad = step.grads[k]
    opt_s = torch.optim.Adam([{"params": [getattr(scene, k)], "lr": GAUSS_LR[k]} for k in keys], eps=1e-15)
    rot, trans, dp = ext[:, :3].clone(), ext[:, 3:].clone(), delta.clone()
    for t in (rot, trans, dp):
        t.grad = torch.zeros_like(t)
    opt_c = torch.optim.Adam([{"params": [rot], "lr": 1e-4}, {"params": [trans], "lr": 5e-3},
                              {"params": [dp], "lr": 1e-3}], eps=1e-15)

    def one():
        step()
        g = step.grads
        rot.grad.copy_(g["ext"][:, :3])
        trans.grad.copy_(g["ext"][:, 3:])
        dp.grad.copy_(g["delta"])
        opt_s.step()
        opt_c.step()
        ext[:, :3].copy_(rot)
        ext[:, 3:].copy_(trans)
        delta.copy_(dp)

    for _ in range(3):
        one()
    n = min(args.steps, 50)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        one()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    for k in keys:
        getattr(scene, k).grad = None
        getattr(scene, k).copy_(saved[k])
    ext.copy_(ext0)
    delta.copy_(delta0)
    torch.cuda.synchronize()
    return {"value": 1e3 / ms, "unit": "iters/s", "ms_per_step": ms, "steps": n,
            "what": "the iteration plus one torch Adam step on the 1M Gaussians' attributes and on the "
                    "extrinsic and delta (excluded from the main value)"}


def visible_records(plan):
    """Records with a non-empty tile rectangle (visible in their frame)."""
    import torch

    from paper_2403_11577_gb300 import capi
    R = plan.batch.num_records
    rect = plan.ws_view(capi.WS_RECT, torch.int32, 2 * R).view(-1, 2)
    x0, y0 = rect[:, 0] & 0xFFFF, (rect[:, 0] >> 16) & 0xFFFF
    x1, y1 = rect[:, 1] & 0xFFFF, (rect[:, 1] >> 16) & 0xFFFF
    return int(((x0 <= x1) & (y0 <= y1)).sum().item())


def stage_rooflines(kernel_ms, st, plan, scene, opts, clock_mhz, sms, peaks):
    """Each stage against its roofline, on the planned algorithmic work per
    unit: projection 44 B per Gaussian read once + 32 B per visible record
    written; bin + sort 2 x 12 B per pair + 8 B per visible record (the
    lower bound), with the radix-pass model beside it; render forward 20 flop
    and render backward 60 flop per composited pair, with the kernels' own
    recount beside; projection backward 44 B per Gaussian read + 36 B per
    visible record + 44 B per Gaussian written.  The pipe and shared-memory
    utilisations come from the committed ncu summary (profiles/), when it
    was taken on the same kernel source."""
    N, P = scene.n, int(st.num_pairs)
    V = visible_records(plan)
    R = plan.batch.num_records
    tpass = max(1, (int(plan.batch.num_tiles - 1).bit_length() + 7) // 8)
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp32 = sms * 128 * 2 * clock_mhz * 1e6 / 1e12
    ncu = load_ncu_metrics()
    out = {}
    work = {
        "project": ("hbm", 44 * N + 32 * V, "44 B per Gaussian + 32 B per visible record", None),
        "bin_sort": ("hbm", 24 * P + 8 * V, "2 x 12 B per pair + 8 B per visible record",
                     {"radix_pass_model_bytes": 4 * 24 * R + tpass * 24 * P,
                      "what": "4 record passes + %d tile passes, 24 B per item each (read + write of key and "
                              "value, histogram read)" % tpass}),
        "render_fwd": ("alu", FLOP_PER_PAIR_FWD * st.eval_fwd, "20 flop per composited pair (+ one 2^x)",
                       {"recount_flop_per_pair": RECOUNT_PER_PAIR_FWD}),
        "render_bwd": ("alu", FLOP_PER_PAIR_BWD * st.eval_bwd, "60 flop per composited pair",
                       {"recount_flop_per_pair": RECOUNT_PER_PAIR_BWD}),
        "project_bwd": ("hbm", 44 * N + 36 * V + 44 * N, "44 B per Gaussian read + 36 B per visible record "
                        "+ 44 B per Gaussian written", None),
    }
    for name, ms in kernel_ms.items():
        if name not in work or not ms:
            continue
        bound, units, what, extra = work[name]
        if bound == "hbm":
            ach = units / (ms / 1e3) / 1e9
            ent = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                   "algorithmic_bytes": int(units), "unit_work": what, "ms": ms,
                   "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)"}
        else:
            ach = units / (ms / 1e3) / 1e12
            ent = {"bound": "alu", "achieved": ach, "peak": fp32, "unit": "TFLOP/s", "frac": ach / fp32,
                   "units_per_launch": int(units / (FLOP_PER_PAIR_FWD if name == "render_fwd" else FLOP_PER_PAIR_BWD)),
                   "unit_work": what, "ms": ms,
                   "peak_basis": "FP32: %d SMs x 128 lanes x 2 flop x %.0f MHz (median SM clock in the timed "
                                 "region)" % (sms, clock_mhz)}
            rec = extra["recount_flop_per_pair"] * ent["units_per_launch"] / (ms / 1e3) / 1e12
            ent["recount"] = {"flop_per_pair": extra["recount_flop_per_pair"], "achieved": rec, "frac": rec / fp32}
            extra = None
        if extra:
            ent.update(extra)
        if name in ncu:
            ent["ncu"] = ncu[name]
        out[name] = ent
    return out


def load_ncu_metrics():
    """Per-kernel utilisations from profiles/ncu_stage_metrics.json, kept only
    where the summary's kernel source hash matches this tree."""
    path = os.path.join(ROOT, "profiles", "ncu_stage_metrics.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return {}
    out = {}
    ids = {v: k for k, v in KERNEL_NAMES.items()}
    for name, ent in d.get("kernels", {}).items():
        if name in ids and ent.get("source_sha") == source_sha(ids[name]):
            out[name] = {k: v for k, v in ent.items() if k != "source_sha"}
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2403_11577_gb300 import build, capi, render
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t_setup = time.time()
    problem = build_problem(args)
    scene = render.DeviceScene.from_problem(problem, dev)
    opts = render.RenderOptions(tile=args.tile, batch=args.batch)
    tuning = {"tile": args.tile, "batch": args.batch,
              "source": "fixed on the command line" if (args.tile, args.batch) != (16, 64) else
              "fixed: the autotuner's choice for this workload on GB300 (profiles/autotune_c3_1M_8x1408x376.md)"}
    if args.autotune:
        from paper_2403_11577_gb300 import autotune
        best = autotune.tune(problem, scene)
        opts = render.RenderOptions(tile=best["tile"], batch=best["batch"])
        tuning = {"tile": best["tile"], "batch": best["batch"], "source": "autotuner, this run",
                  "table_ms": best["table"]}
    ext = torch.tensor(problem.ext, dtype=torch.float64, device=dev)
    delta = torch.tensor(problem.delta, dtype=torch.float64, device=dev)
    ext_t = torch.tensor(problem.ext_target, dtype=torch.float64, device=dev)
    delta_t = torch.tensor(problem.delta_target, dtype=torch.float64, device=dev)
    frames = render.Plan.frames_from_problem(problem, scene)
    cap = render.default_pair_capacity(frames, opts.tile)
    while True:
        plan = render.Plan(frames, scene.n, problem.num_cameras, len(problem.scenes), opts, cap, dev)
        plan.forward(scene, ext_t, delta_t)
        st = plan.stats()
        plan.forward(scene, ext, delta)
        st2 = plan.stats()
        if not (st.status | st2.status) & capi.GS_DEV_PAIR_OVERFLOW:
            break
        cap = int(min(cap * 2, (1 << 32) - 1))
    plan.forward(scene, ext_t, delta_t)
    target = plan.rgb.clone()
    step = render.CalibStep(plan, scene, target, ext, delta, graph=True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = plan.stats()
    setup_s = time.time() - t_setup

    # timed region: K graph replays
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    barrier(world)
    t_ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    t_max = max_over_ranks(t_ms / 1e3, world)
    value = world * args.steps / t_max

    # per-frame path (same work, launched frame by frame, no graph)
    pf = render.PerFrameStep(problem, scene, target, ext, delta, opts, pair_capacity=cap)
    for _ in range(2):
        pf()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.per_frame_steps):
        pf()
    e1.record()
    torch.cuda.synchronize()
    per_frame = args.per_frame_steps / (e0.elapsed_time(e1) / 1e3)
    del pf

    # per-kernel durations on the launching stream (eager, one step each)
    kernel_ms = {}
    for kid in KERNEL_NAMES:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        capi.gs_profile_events(kid, a, b)
        ts = []
        for _ in range(3):
            step._body()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        kernel_ms[KERNEL_NAMES[kid]] = statistics.median(ts)
    capi.gs_profile_events(capi.GS_PROF_NONE)
    dom = max(KERNEL_NAMES, key=lambda k: kernel_ms[KERNEL_NAMES[k]])
    # the dominant kernel inside graph replays: events captured as graph nodes
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    capi.gs_profile_events(dom, a, b)
    pstep = render.CalibStep(plan, scene, target, ext, delta, graph=True)
    capi.gs_profile_events(capi.GS_PROF_NONE)
    durs = []
    for _ in range(min(args.steps, 50)):
        pstep()
        torch.cuda.synchronize()
        durs.append(a.elapsed_time(b))
    dom_ms = statistics.mean(durs)
    del pstep
    st = plan.stats()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    clock_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    roof = dict(stage_rooflines({KERNEL_NAMES[dom]: dom_ms}, st, plan, scene, opts, clock_mhz, sms,
                                peaks)[KERNEL_NAMES[dom]])
    # the committed capture is scaled to the 8-frame batched workload's launch
    headline = args.workload == "batched" and args.gaussians == 1_000_000 and args.frames == 8 and \
        opts.tile == 16 and opts.batch == 64
    roof["traffic"] = load_traffic(dom) if headline else None
    roof["kernel"] = KERNEL_NAMES[dom]
    roof["launch_ms"] = dom_ms

    stages = stage_rooflines(kernel_ms, st, plan, scene, opts, clock_mhz, sms, peaks)
    with_adam = adam_steps(args, step, scene, ext, delta)

    # end to end through the public API with host buffers: per step the
    # target images go host->device from pinned memory and the loss and the
    # calibration gradients come back.  The copy of step k + 1's targets runs
    # on a copy stream into a device staging buffer while step k computes
    # (double-buffered); each step then moves its staged targets into the
    # graph's input with a device-to-device copy.  Every step's host->device
    # copy and its device->host reads lie inside the timed region.
    tgt_host = target.cpu().pin_memory()
    loss_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    dext_h = torch.zeros_like(step.grads["ext"], device="cpu").pin_memory()
    ddel_h = torch.zeros_like(step.grads["delta"], device="cpu").pin_memory()
    h2d = tgt_host.numel() * 4
    d2h = 8 + dext_h.numel() * 8 + ddel_h.numel() * 8
    copy_stream = torch.cuda.Stream()
    stage = [torch.empty_like(step.target) for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    main = torch.cuda.current_stream()

    def stage_copy(k):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(freed[b])  # step k - 2 has moved its targets out of this buffer
            stage[b].copy_(tgt_host, non_blocking=True)
            copied[b].record(copy_stream)

    torch.cuda.synchronize()
    e0.record()
    w1 = time.perf_counter()
    stage_copy(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            stage_copy(k + 1)
        main.wait_event(copied[k % 2])
        step.target.copy_(stage[k % 2])
        freed[k % 2].record(main)
        step()
        loss_h.copy_(step.loss[:1], non_blocking=True)
        dext_h.copy_(step.grads["ext"], non_blocking=True)
        ddel_h.copy_(step.grads["delta"], non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - w1
    e2e_t = max_over_ranks(max(e0.elapsed_time(e1) / 1e3, e2e_wall), world)
    e2e = world * args.steps / e2e_t

    # the paper's own loop on the same scene and poses: L_photo = 0.8 L1 + 0.2
    # D-SSIM (Eq. 4) on the bottom half of every frame (Sec. III-D), whose top
    # half is then neither binned nor rendered
    paper = None
    if not args.no_paper_loop and args.workload == "batched":
        paper = paper_loop(args, problem, scene, opts, ext, delta, ext_t, delta_t, dev, world)

    # kernels per iteration: pose 1, project 1, bin_sort (4 record passes x 3,
    # count/scan/emit 3, range init 1, tile passes x 3 (the last also finds
    # the ranges), order 1), render fwd 1, L1 2, render bwd 1, projection
    # bwd 1, pose grad 3 (two twist reduction stages and the per-camera
    # gradient)
    tile_bits = max(0, math.ceil(math.log2(max(plan.batch.num_tiles, 1))))
    tile_passes = (tile_bits + 7) // 8
    launches_per_step = 1 + 1 + (12 + 3 + 1 + 3 * tile_passes + 1) + 1 + 2 + 1 + 1 + 3
    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(args, problem, opts),
        "pairs_per_iter": int(st.num_pairs), "workspace_gb": plan.ws_bytes / 1e9,
        "tuning": tuning,
        "per_frame": {"value": per_frame, "unit": "iters/s", "speedup_batched": value / world / per_frame},
        "kernel_ms": kernel_ms,
        "composited_pairs": {"fwd": int(st.eval_fwd), "bwd": int(st.eval_bwd)},
        "roofline": roof,
        "stages": stages,
        "e2e": {"value": e2e, "unit": "iters/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "wall_timed_s": wall, "setup_s": setup_s,
        "loss": float(step.loss[0].item()),
    }
    out["with_adam"] = with_adam
    if paper is not None:
        out["paper_loop"] = paper
    if args.workload != "batched":
        out["metric"] = "calib iters/s (fwd+bwd, uneven batch: 3 scenes, 12 frames)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, sample = oracle_sampled_iterations(problem, args.cpu_pixels, range(len(problem.frames)))
        out["cpu_baseline"] = {"value": 1.0 / secs, "unit": "iters/s", "cores": 1, "kind": "oracle",
                               "host": host_cpu(),
                               "sample": "FP64 oracle, one thread, once per frame (the reference arm's step): "
                                         "projection + global depth sort, forward and backward of %d sampled "
                                         "pixels, extrapolated to a full iteration (%d frames, all pixels); "
                                         "the mean over the %d frames (%.1f s of CPU)" %
                                         (args.cpu_pixels, len(problem.frames), len(problem.frames), sample),
                               "c1_loop": oracle_c1_loop(30)}
    return out


def oracle_sampled_iterations(problem, pixels, frame_ids):
    """Mean extrapolated full-iteration seconds over one sample per frame id
    (frame i, `pixels` sampled pixels, seed i), and the CPU seconds spent."""
    times, spent = [], 0.0
    for i in frame_ids:
        secs, sample = oracle_iteration_seconds(problem, pixels, [i % len(problem.frames)], seed=i)
        times.append(secs)
        spent += sample
    return float(np.mean(times)), spent


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores, on this workload; each step
    is a bounded sample extrapolated to one full iteration."""
    if rank != 0:
        return None
    problem = build_problem(args)
    fr = len(problem.frames)
    for i in range(args.warmup):  # warm-up samples (not timed)
        oracle_iteration_seconds(problem, args.cpu_pixels, [i % fr], seed=1000 + i)
    # step i: frame i mod F with `cpu_pixels` sampled pixels, extrapolated to a
    # full iteration; the same sample the GPU arm's cpu_baseline takes
    secs, sample_total = oracle_sampled_iterations(problem, args.cpu_pixels, range(args.steps))
    v = 1.0 / secs
    return {"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "steps_extrapolated": "each step times a bounded sample (one frame's projection and sort, %d sampled "
                                  "pixels forward and backward) and extrapolates it to a full iteration; "
                                  "ms_per_step is that extrapolated time, not a timed region" % args.cpu_pixels,
            "config": bench_config(args, problem),
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": "per step: one frame's projection + global sort, forward and backward of %d "
                                       "sampled pixels, extrapolated to %d frames x 529,408 pixels (%.1f s CPU "
                                       "total)" % (args.cpu_pixels, fr, sample_total)},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    else:
        out = run_ours(args, world, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
