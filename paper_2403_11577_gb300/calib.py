"""Synthetic spatiotemporal calibration with the splatting path (3DGS-Calib,
Sec. III and Sec. IV-B).

Jointly optimises the Gaussian attributes (colour, opacity, scale, rotation;
the means stay at the LiDAR points, Sec. III-B), the camera-to-LiDAR
extrinsic and the time offset with Adam, against target images rendered at
the true calibration:

  L_total = L_photo + lambda_2 * L_scale      (Eq. 4, 7-8)
  L_photo = L1 (loss="l1") or (1 - lambda_1) L1 + lambda_1 D-SSIM with
            lambda_1 = 0.2 (loss="photo", Eq. 4), optionally on the bottom
            half of each image only (crop, Sec. III-D)
  L_scale = sum_g || s_g - mean(s_g) ||_1     (activated scales, lambda_2 = 1e-3)

Learning rates follow Sec. IV-B (rotation 1e-4, translation 5e-3, time
offset 1e-3, each decayed linearly to 0.1x by the end), with a warm-up
during which only the scene is trained.  Gaussian attributes start as in
Sec. IV-B: random colours, opacity 0.1, identity rotation; the scales start
from the scene's own.  Every iteration's splatting, loss gradient and
calibration gradient is one CUDA-graph replay of the library's kernels;
L_scale and Adam are plain torch on the parameter tensors.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np
import torch

from . import build, ngp, render, scenes

GAUSS_LR = {"rgb": 2.5e-3, "logit_opacity": 5e-2, "log_scale": 5e-3, "quat": 1e-3}


def rotation_error_deg(omega_a, omega_b):
    """Geodesic angle between two rotations given as rotation vectors."""
    from scipy.spatial.transform import Rotation
    ra, rb = Rotation.from_rotvec(omega_a), Rotation.from_rotvec(omega_b)
    return float(np.degrees((ra * rb.inv()).magnitude()))


def errors(ext, delta, ext_true, delta_true):
    """Calibration errors of one camera."""
    return {"rot_deg": rotation_error_deg(ext[:3], ext_true[:3]),
            "trans_cm": float(100 * np.linalg.norm(ext[3:] - ext_true[3:])),
            "delta_ms": float(1000 * abs(delta - delta_true))}


def rig_errors(ext, delta, ext_true, delta_true):
    """Worst error over the cameras, plus the per-camera errors when there
    is more than one camera."""
    per = [errors(ext[c], float(delta[c]), ext_true[c], float(delta_true[c])) for c in range(len(ext))]
    out = {k: max(e[k] for e in per) for k in per[0]}
    if len(per) > 1:
        out["cameras"] = per
    return out


def run_calibration(problem, iters=3000, warmup=500, lr_rot=1e-4, lr_trans=5e-3, lr_delta=1e-3,
                    lambda_scale=1e-3, opts=None, seed=0, log_every=250, reinit=True, train_scene=True,
                    scene_lr_scale=1.0, device="cuda", loss="l1", schedule=None, clamp_scale=True, model="direct",
                    mlp_lr=1e-2, grid_weight_decay=1e-4):
    """Calibrate every camera of `problem` (its ext/delta are the start,
    ext_target/delta_target the truth; errors are the worst over cameras).
    train_scene=False keeps the Gaussian attributes fixed (calibration only).

    schedule: coarse-to-fine voxelization (Sec. III-D), a list of
    (voxel size in metres, iterations).  Each phase renders one point per
    voxel of the accumulated cloud (gs_voxel_downsample), with every
    Gaussian's scale bounded by the voxel size when clamp_scale.  The
    attributes live on the full cloud, so each phase continues from their
    current values; iters is then the sum of the phases.  Targets are always
    rendered from the full cloud at the true calibration.

    model="mlp" learns the attributes through F(X | Theta) (Sec. III-C,
    ngp.HashGridMLP): every iteration evaluates it for the rendered
    Gaussians and carries their attribute gradients back into Theta (Adam,
    lr mlp_lr, weight decay grid_weight_decay on the hash grid as in the
    paper); model="direct" learns per-Gaussian attributes.

    Returns a dict with the error history, the final errors, the wall time
    and, with a schedule, the Gaussians and time of each phase."""
    build.build()
    dev = torch.device(device)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    full = render.DeviceScene.from_problem(problem, dev)
    opts = opts or render.RenderOptions(tile=problem.tile)
    # targets: the true calibration and the scene's true attributes
    e_true = torch.tensor(problem.ext_target, dtype=torch.float64, device=dev)
    d_true = torch.tensor(problem.delta_target, dtype=torch.float64, device=dev)
    plan = render.Plan.for_problem(problem, full, opts)
    plan.forward(full, e_true, d_true)
    target = plan.rgb.clone()
    del plan
    # parameters (on the full cloud)
    if reinit:
        n = full.n
        full.rgb.copy_(torch.rand((n, 3), generator=gen).to(dev))
        full.logit_opacity.fill_(math.log(0.1 / 0.9))
        full.quat.zero_()
        full.quat[:, 0] = 1.0
    ext = torch.tensor(problem.ext, dtype=torch.float64, device=dev)
    delta = torch.tensor(problem.delta, dtype=torch.float64, device=dev)
    params = {k: getattr(full, k) for k in GAUSS_LR}
    for t in params.values():
        t.grad = torch.zeros_like(t)
    rot = ext[:, :3].clone()
    trans = ext[:, 3:].clone()
    rot.grad, trans.grad = torch.zeros_like(rot), torch.zeros_like(trans)
    delta_p = delta.clone()
    delta_p.grad = torch.zeros_like(delta_p)
    opt_scene = torch.optim.Adam([{"params": [params[k]], "lr": GAUSS_LR[k] * scene_lr_scale} for k in GAUSS_LR],
                                 eps=1e-15)
    mlp = None
    if model == "mlp":
        mlp = ngp.HashGridMLP(ngp.HashGridConfig.for_points(full.X), device=dev, seed=seed)
        nt = mlp.cfg.levels * mlp.cfg.T * 2
        grid, net = mlp.theta[:nt], mlp.theta[nt:]
        grid.grad, net.grad = mlp.grad[:nt], mlp.grad[nt:]
        opt_scene = torch.optim.Adam([{"params": [grid], "weight_decay": grid_weight_decay},
                                      {"params": [net], "weight_decay": 0.0}], lr=mlp_lr, betas=(0.9, 0.99),
                                     eps=1e-15)
    elif model != "direct":
        raise ValueError("model must be 'direct' or 'mlp'")
    opt_cal = torch.optim.Adam([{"params": [rot], "lr": lr_rot}, {"params": [trans], "lr": lr_trans},
                                {"params": [delta_p], "lr": lr_delta}], eps=1e-15)
    base_lrs = [g["lr"] for g in opt_cal.param_groups]
    phases = list(schedule) if schedule else [(None, iters)]
    iters = sum(n for _, n in phases)
    history, phase_log = [], []
    e_true_np, d_true_np = np.asarray(problem.ext_target), np.asarray(problem.delta_target)
    torch.cuda.synchronize()
    t0 = time.time()
    it = 0
    for voxel, n_it in phases:
        tp = time.time()
        if voxel is None:
            idx, scene, opts_p = None, full, opts
        else:
            idx = render.voxel_downsample(full.X, voxel)
            scene = full.subset(idx)
            opts_p = dataclasses.replace(opts, scale_max=voxel) if clamp_scale else opts
        plan = render.Plan.for_problem(problem, scene, opts_p)
        step = render.CalibStep(plan, scene, target, ext, delta, graph=True, loss=loss)
        for _ in range(n_it):
            # the graph reads ext/delta (and a phase's Gaussians) from static tensors
            ext[:, :3].copy_(rot)
            ext[:, 3:].copy_(trans)
            delta.copy_(delta_p)
            if mlp is not None:
                mlp.forward(scene.X, {k: getattr(scene, k) for k in GAUSS_LR})
            elif idx is not None and train_scene:
                for k in GAUSS_LR:
                    getattr(scene, k).copy_(params[k][idx])
            loss_v = step()
            if mlp is not None and train_scene:
                g = dict(step.grads)
                if lambda_scale > 0:  # L_scale (Eq. 7) on the predicted scales
                    with torch.enable_grad():
                        ls = scene.log_scale.detach().requires_grad_(True)
                        sc = torch.exp(ls)
                        reg = lambda_scale * (sc - sc.mean(dim=1, keepdim=True)).abs().sum()
                        (g_ls,) = torch.autograd.grad(reg, ls)
                    g["log_scale"] = g["log_scale"] + g_ls
                mlp.backward(scene.X, g)
                opt_scene.step()
            elif train_scene:
                for k in GAUSS_LR:
                    if idx is None:
                        params[k].grad.copy_(step.grads[k])
                    else:
                        params[k].grad.zero_()
                        params[k].grad[idx] = step.grads[k]
                # L_scale on the activated scales (Eq. 7) of the rendered Gaussians
                if lambda_scale > 0:
                    with torch.enable_grad():
                        ls = (params["log_scale"] if idx is None else params["log_scale"][idx]).detach()
                        ls.requires_grad_(True)
                        sc = torch.exp(ls)
                        reg = lambda_scale * (sc - sc.mean(dim=1, keepdim=True)).abs().sum()
                        (g_ls,) = torch.autograd.grad(reg, ls)
                    if idx is None:
                        params["log_scale"].grad.add_(g_ls)
                    else:
                        params["log_scale"].grad[idx] += g_ls
                opt_scene.step()
            if it >= warmup:
                frac = (it - warmup) / max(1, iters - warmup)
                for g, lr0 in zip(opt_cal.param_groups, base_lrs):
                    g["lr"] = lr0 * (1.0 - 0.9 * frac)
                rot.grad.copy_(step.grads["ext"][:, :3])
                trans.grad.copy_(step.grads["ext"][:, 3:])
                delta_p.grad.copy_(step.grads["delta"])
                opt_cal.step()
            # keep quaternions away from zero norm
            if train_scene and mlp is None and it % 100 == 99:
                with torch.no_grad():
                    q = params["quat"]
                    q.div_(q.norm(dim=1, keepdim=True).clamp_min(1e-8))
            if log_every and (it % log_every == 0 or it == iters - 1):
                e_np = torch.cat([rot, trans], 1).cpu().numpy()
                err = rig_errors(e_np, delta_p.cpu().numpy(), e_true_np, d_true_np)
                err.update(it=it, loss=float(loss_v.item()))
                history.append(err)
            it += 1
        torch.cuda.synchronize()
        if voxel is not None:
            e_np = torch.cat([rot, trans], 1).cpu().numpy()
            phase_log.append({"voxel_m": voxel, "iters": n_it, "gaussians": scene.n, "wall_s": time.time() - tp,
                              "errors": rig_errors(e_np, delta_p.cpu().numpy(), e_true_np, d_true_np)})
        del step, plan
    torch.cuda.synchronize()
    wall = time.time() - t0
    e_np = torch.cat([rot, trans], 1).cpu().numpy()
    final = rig_errors(e_np, delta_p.cpu().numpy(), e_true_np, d_true_np)
    start = rig_errors(np.asarray(problem.ext), np.asarray(problem.delta), e_true_np, d_true_np)
    out = {"start": start, "final": final, "wall_s": wall, "iters": iters, "warmup": warmup,
           "history": history, "ms_per_iter": 1e3 * wall / iters}
    if schedule:
        out["phases"] = phase_log
    return out


def parse_schedule(text):
    """"0.10:2000,0.05:500,0.02:500" -> [(0.10, 2000), (0.05, 500), (0.02, 500)]."""
    out = []
    for part in text.split(","):
        v, n = part.split(":")
        out.append((float(v), int(n)))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--gaussians", type=int, default=1_000_000)
    ap.add_argument("--trajectory", choices=["straight", "zigzag"], default="zigzag")
    ap.add_argument("--loss", choices=["l1", "photo"], default="l1",
                    help="l1, or L_photo = 0.8 L1 + 0.2 D-SSIM (Eq. 4)")
    ap.add_argument("--crop", action="store_true", help="losses on the bottom half of each image (Sec. III-D)")
    ap.add_argument("--cameras", type=int, default=1, help="forward cameras of the rig, calibrated jointly")
    ap.add_argument("--schedule", default=None,
                    help="coarse-to-fine voxelization, e.g. 0.10:2000,0.05:500,0.02:500 (Sec. III-D, Sec. IV-C)")
    ap.add_argument("--attributes", choices=["random", "surface"], default="random",
                    help="the target scene's Gaussian shapes and opacities: i.i.d. random, or smooth along surfaces")
    ap.add_argument("--model", choices=["direct", "mlp"], default="direct",
                    help="joint mode: per-Gaussian attributes, or the hash-grid MLP F(X | Theta) (Sec. III-C)")
    ap.add_argument("--no-scale-clamp", action="store_true",
                    help="with --schedule: do not bound the scales by the voxel size")
    ap.add_argument("--mode", choices=["joint", "pose"], default="joint",
                    help="joint: re-initialised scene trained with the calibration; "
                         "pose: the scene's attributes fixed at their true values")
    a = ap.parse_args()
    p = scenes.calibration_problem(seed=a.seed, n=a.gaussians, trajectory=a.trajectory, cameras=a.cameras,
                                   attributes=a.attributes)
    if a.crop:
        for f in p.frames:
            f.row0 = f.camera.height // 2
    sched = parse_schedule(a.schedule) if a.schedule else None
    kw = dict(seed=a.seed, loss=a.loss, schedule=sched, clamp_scale=not a.no_scale_clamp, model=a.model)
    if a.mode == "pose":
        res = run_calibration(p, iters=a.iters, warmup=0, reinit=False, train_scene=False, **kw)
    else:
        res = run_calibration(p, iters=a.iters, warmup=a.warmup, reinit=True, **kw)
    res.update(trajectory=a.trajectory, mode=a.mode, seed=a.seed, gaussians=a.gaussians, loss=a.loss, crop=a.crop,
               cameras=a.cameras, schedule=a.schedule, scale_clamp=not a.no_scale_clamp, model=a.model,
               attributes=a.attributes)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
