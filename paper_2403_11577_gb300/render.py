"""Batch planning, workspace, autograd wrapper and the calibration step.

Everything here is plumbing around the C-ABI of libgs3dcalib.so: device
memory (torch tensors), the current stream, CUDA-graph capture and a
torch.autograd.Function.  Every step of the splatting path itself runs in
the library's kernels.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi


@dataclass
class RenderOptions:
    """Renderer settings (the paper defers the renderer to 3DGS and EWA)."""
    near_z: float = 0.2
    lowpass: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    scale_max: float = float("inf")
    bg: tuple = (0.0, 0.0, 0.0)
    tile: int = 16
    batch: int = 64
    frustum_margin: float = 0.15
    exact_tiles: bool = True  # bin each Gaussian only to the tiles its ellipse meets

    def c(self) -> capi.GsOpts:
        o = capi.GsOpts()
        o.near_z, o.lowpass, o.alpha_min = self.near_z, self.lowpass, self.alpha_min
        o.alpha_max, o.t_min, o.scale_max = self.alpha_max, self.t_min, self.scale_max
        o.bg = (C.c_float * 3)(*self.bg)
        o.tile, o.batch, o.frustum_margin = self.tile, self.batch, self.frustum_margin
        o.exact_tiles = int(bool(self.exact_tiles))
        return o


@dataclass
class DeviceScene:
    """Gaussians of all scenes (concatenated) and the LiDAR trajectories."""
    X: torch.Tensor            # [N,3] f32
    quat: torch.Tensor         # [N,4] f32
    log_scale: torch.Tensor    # [N,3] f32
    logit_opacity: torch.Tensor  # [N] f32
    rgb: torch.Tensor          # [N,3] f32
    traj_t: torch.Tensor       # [K] f64
    traj_pose: torch.Tensor    # [K,7] f64 (p, q)
    traj_offset: torch.Tensor  # [S+1] i32
    gauss_offset: list = field(default_factory=list)  # per scene
    gauss_count: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    def subset(self, idx: torch.Tensor) -> "DeviceScene":
        """The Gaussians idx (ascending global indices), same trajectories;
        each scene keeps its kept Gaussians in order."""
        idx = idx.to(self.X.device)
        offs, counts = [], []
        for o, c in zip(self.gauss_offset, self.gauss_count):
            lo = int(torch.searchsorted(idx, torch.tensor(o, device=idx.device)))
            hi = int(torch.searchsorted(idx, torch.tensor(o + c, device=idx.device)))
            offs.append(lo)
            counts.append(hi - lo)
        return DeviceScene(X=self.X[idx].contiguous(), quat=self.quat[idx].contiguous(),
                           log_scale=self.log_scale[idx].contiguous(),
                           logit_opacity=self.logit_opacity[idx].contiguous(), rgb=self.rgb[idx].contiguous(),
                           traj_t=self.traj_t, traj_pose=self.traj_pose, traj_offset=self.traj_offset,
                           gauss_offset=offs, gauss_count=counts)

    @staticmethod
    def from_problem(problem, device="cuda") -> "DeviceScene":
        sc = problem.scenes

        def cat(name, dtype):
            return torch.from_numpy(np.ascontiguousarray(np.concatenate([getattr(s, name) for s in sc]),
                                                         dtype=dtype)).to(device)
        traj_pose = np.concatenate([np.concatenate([s.traj_p, s.traj_q], axis=1) for s in sc])
        offs = np.zeros(len(sc) + 1, np.int32)
        offs[1:] = np.cumsum([len(s.traj_t) for s in sc])
        goff = [0]
        for s in sc[:-1]:
            goff.append(goff[-1] + s.n)
        return DeviceScene(
            X=cat("X", np.float32), quat=cat("quat", np.float32), log_scale=cat("log_scale", np.float32),
            logit_opacity=cat("logit_opacity", np.float32), rgb=cat("rgb", np.float32),
            traj_t=cat("traj_t", np.float64),
            traj_pose=torch.from_numpy(np.ascontiguousarray(traj_pose, np.float64)).to(device),
            traj_offset=torch.from_numpy(offs).to(device), gauss_offset=goff, gauss_count=[s.n for s in sc])


def voxel_downsample(X: torch.Tensor, voxel: float) -> torch.Tensor:
    """Indices (int64, ascending) of the points kept by the accumulated-LiDAR
    voxel downsampling of Sec. III-D (gs_voxel_downsample): one point per
    occupied voxel, the one of smallest index."""
    n = int(X.shape[0])
    _raw, scratch = _aligned_workspace(capi.gs_voxel_scratch_size(n), X.device)
    idx = torch.empty(max(n, 1), dtype=torch.int32, device=X.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=X.device)
    capi.gs_voxel_downsample(X.contiguous(), voxel, idx, cnt, scratch)
    return idx[:int(cnt.item())].long()


def _aligned_workspace(nbytes: int, device) -> tuple:
    """A uint8 tensor whose data pointer is 256-byte aligned."""
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % 256
    return raw, raw[off:off + nbytes]


class Plan:
    """A planned batch of frames with its workspace and image outputs.

    frames: list of dicts with width, height, fx, fy, cx, cy, camera_id,
    traj_id, gauss_offset, gauss_count, timestamp and optionally row0 (the
    first image row rendered; the frame's image is rows [row0, height)).
    """

    def __init__(self, frames, num_gaussians, num_cameras, num_trajs, opts: RenderOptions,
                 pair_capacity: int, device="cuda"):
        self.opts = opts
        self.copts = opts.c()
        self.device = torch.device(device)
        F = len(frames)
        arr = (capi.GsFrame * F)()
        for i, fr in enumerate(frames):
            for k in ("width", "height", "fx", "fy", "cx", "cy", "camera_id", "traj_id", "gauss_offset",
                      "gauss_count", "timestamp"):
                setattr(arr[i], k, fr[k])
            arr[i].row0 = fr.get("row0", 0)
        self.frames_host = arr
        self.frames_dev = torch.empty(C.sizeof(capi.GsFrame) * F, dtype=torch.uint8, device=self.device)
        self.batch = capi.gs_batch_init(arr, num_gaussians, num_cameras, num_trajs, opts.tile, pair_capacity,
                                        self.frames_dev)
        self.ws_bytes = capi.gs_workspace_size(self.batch)
        self._ws_raw, self.ws = _aligned_workspace(self.ws_bytes, self.device)
        self.ws.zero_()
        self.offsets = capi.gs_workspace_offsets(self.batch)
        P = self.batch.num_pixels
        self.rgb = torch.empty((P, 3), dtype=torch.float32, device=self.device)
        self.T = torch.empty(P, dtype=torch.float32, device=self.device)
        self.last = torch.empty(P, dtype=torch.int32, device=self.device)
        self.generation = 0

    # -- construction helpers
    @staticmethod
    def frames_from_problem(problem, scene: DeviceScene, frame_ids=None):
        out = []
        ids = range(len(problem.frames)) if frame_ids is None else frame_ids
        for i in ids:
            f = problem.frames[i]
            c = f.camera
            out.append(dict(width=c.width, height=c.height, fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy,
                            camera_id=f.camera_id, traj_id=f.scene_id,
                            gauss_offset=scene.gauss_offset[f.scene_id],
                            gauss_count=scene.gauss_count[f.scene_id], timestamp=f.timestamp, row0=f.row0))
        return out

    @staticmethod
    def for_problem(problem, scene: DeviceScene, opts: RenderOptions | None = None, pair_capacity=None,
                    frame_ids=None, device="cuda") -> "Plan":
        opts = opts or RenderOptions(tile=problem.tile)
        frames = Plan.frames_from_problem(problem, scene, frame_ids)
        if pair_capacity is None:
            pair_capacity = default_pair_capacity(frames, opts.tile)
        return Plan(frames, scene.n, problem.num_cameras, len(problem.scenes), opts, pair_capacity, device)

    # -- per-frame views
    @property
    def num_frames(self) -> int:
        return self.batch.num_frames

    def frame(self, i):
        return self.frames_host[i]

    def image(self, t, i):
        """View of frame i's pixels of a [P,...] tensor as [H - row0, W, ...]
        (image rows row0 .. H-1)."""
        fr = self.frames_host[i]
        rows = fr.height - fr.row0
        n = fr.width * rows
        return t[fr.pixel_offset:fr.pixel_offset + n].view(rows, fr.width, *t.shape[1:])

    def ws_view(self, idx, dtype, count, start=0):
        """Typed view of a workspace region (offset index idx, capi.WS_*)."""
        esize = torch.tensor([], dtype=dtype).element_size()
        off = self.offsets[idx] + start * esize
        return self.ws[off:off + count * esize].view(dtype)

    def stats(self):
        return capi.gs_read_stats(self.batch, self.ws)

    # -- the path (C-ABI calls)
    def pose(self, scene: DeviceScene, ext, delta):
        capi.gs_pose_compose(self.batch, scene.traj_t, scene.traj_pose, scene.traj_offset, ext, delta, self.ws)

    def project(self, scene: DeviceScene, quat=None, log_scale=None, logit_opacity=None):
        capi.gs_project(self.batch, scene.X, scene.quat if quat is None else quat,
                        scene.log_scale if log_scale is None else log_scale,
                        scene.logit_opacity if logit_opacity is None else logit_opacity, self.copts, self.ws)

    def bin_sort(self):
        capi.gs_bin_sort(self.batch, self.copts, self.ws)

    def render_fwd(self, colors):
        capi.gs_render_fwd(self.batch, colors, self.copts, self.ws, self.rgb, self.T, self.last)
        self.generation += 1
        return self.rgb

    def forward(self, scene: DeviceScene, ext, delta, quat=None, log_scale=None, logit_opacity=None, rgb=None):
        self.pose(scene, ext, delta)
        self.project(scene, quat, log_scale, logit_opacity)
        self.bin_sort()
        return self.render_fwd(scene.rgb if rgb is None else rgb)

    def backward(self, scene: DeviceScene, dL_drgb, grads: dict, ext, quat=None, log_scale=None,
                 logit_opacity=None, rgb=None, accumulate=False):
        """grads: dict with quat, log_scale, logit_opacity, rgb (f32) and
        ext [C,6], delta [C] (f64) tensors to write (or add) into."""
        capi.gs_render_bwd(self.batch, scene.X, scene.quat if quat is None else quat,
                           scene.log_scale if log_scale is None else log_scale,
                           scene.logit_opacity if logit_opacity is None else logit_opacity,
                           scene.rgb if rgb is None else rgb, self.copts, self.ws, self.T, self.last, dL_drgb,
                           grads["quat"], grads["log_scale"], grads["logit_opacity"], grads["rgb"],
                           accumulate=accumulate)
        capi.gs_pose_grad(self.batch, ext, self.ws, grads["ext"], grads["delta"], grads.get("xi"),
                          accumulate=accumulate)


def default_pair_capacity(frames, tile, per_pixel=24.0, minimum=1 << 16):
    """Pair capacity heuristic: per_pixel pairs per pixel of the batch."""
    px = sum(f["width"] * (f["height"] - f.get("row0", 0)) for f in frames)
    return int(min(max(minimum, per_pixel * px), (1 << 32) - 1))


def empty_grads(scene: DeviceScene, num_cameras: int, xi=False):
    d = scene.X.device
    g = dict(quat=torch.zeros_like(scene.quat), log_scale=torch.zeros_like(scene.log_scale),
             logit_opacity=torch.zeros_like(scene.logit_opacity), rgb=torch.zeros_like(scene.rgb),
             ext=torch.zeros((num_cameras, 6), dtype=torch.float64, device=d),
             delta=torch.zeros(num_cameras, dtype=torch.float64, device=d))
    if xi:
        g["xi"] = torch.zeros((num_cameras, 6), dtype=torch.float64, device=d)
    return g


class SplatFn(torch.autograd.Function):
    """rgb = Phi(X^n, alpha, s, r^n, c) for every frame of a plan (Eq. 5),
    differentiable w.r.t. the Gaussian parameters and, through the pose of
    Eq. 1, the extrinsic and time offset.  The means X are fixed (Sec.
    III-B) and get no gradient.  One application per plan may be in flight:
    the plan's workspace holds the state the backward needs."""

    @staticmethod
    def forward(ctx, plan: Plan, scene: DeviceScene, quat, log_scale, logit_opacity, rgb, ext, delta):
        quat, log_scale, logit_opacity, rgb = (t.detach().contiguous() for t in (quat, log_scale, logit_opacity, rgb))
        ext, delta = ext.detach().contiguous(), delta.detach().contiguous()
        out = plan.forward(scene, ext, delta, quat, log_scale, logit_opacity, rgb).clone()
        ctx.plan, ctx.scene, ctx.gen = plan, scene, plan.generation
        ctx.save_for_backward(quat, log_scale, logit_opacity, rgb, ext)
        return out

    @staticmethod
    def backward(ctx, grad_rgb):
        plan, scene = ctx.plan, ctx.scene
        if plan.generation != ctx.gen:
            raise RuntimeError("SplatFn: the plan was used for another forward before this backward")
        quat, log_scale, logit_opacity, rgb, ext = ctx.saved_tensors
        g = empty_grads(scene, plan.batch.num_cameras)
        plan.backward(scene, grad_rgb.contiguous().float(), g, ext, quat, log_scale, logit_opacity, rgb)
        return None, None, g["quat"], g["log_scale"], g["logit_opacity"], g["rgb"], g["ext"], g["delta"]


def render(plan: Plan, scene: DeviceScene, quat, log_scale, logit_opacity, rgb, ext, delta):
    return SplatFn.apply(plan, scene, quat, log_scale, logit_opacity, rgb, ext, delta)


class CalibStep:
    """One calibration iteration (the unit of the benchmark): pose, project,
    bin + sort, render, the loss with its gradient, render/projection
    backward and pose gradient, for every frame of the plan.  loss="l1" is
    the L1 term of Eq. 4; loss="photo" is L_photo = (1 - lambda1) L1 +
    lambda1 D-SSIM (lambda1 = 0.2 in the paper).  With graph=True the whole
    iteration is one CUDA-graph replay; all inputs and outputs are static
    tensors (update them in place).  self.loss[0] is the loss; for "photo",
    self.loss[1:3] are its L1 and D-SSIM parts."""

    def __init__(self, plan: Plan, scene: DeviceScene, target, ext, delta, graph=True, loss="l1", lambda1=0.2):
        if loss not in ("l1", "photo"):
            raise ValueError("loss must be 'l1' or 'photo'")
        self.plan, self.scene = plan, scene
        self.target = target
        self.ext, self.delta = ext, delta
        self.kind, self.lambda1 = loss, lambda1
        self.loss = torch.zeros(3, dtype=torch.float64, device=plan.device)
        self.dL = torch.zeros_like(plan.rgb)
        self.grads = empty_grads(scene, plan.batch.num_cameras)
        self.graph = None
        if graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                self._body()  # warm-up outside capture
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._body()
            torch.cuda.synchronize()

    def _body(self):
        p = self.plan
        p.forward(self.scene, self.ext, self.delta)
        if self.kind == "photo":
            capi.gs_loss_photo(p.batch, p.rgb, self.target, self.lambda1, self.loss, self.dL, p.ws)
        else:
            capi.gs_loss_l1(p.batch, p.rgb, self.target, 1.0, self.loss, self.dL, p.ws)
        p.backward(self.scene, self.dL, self.grads, self.ext)

    def __call__(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()
        return self.loss[:1]


class PerFrameStep:
    """The same iteration launched frame by frame: one plan per frame, no
    graph, every kernel re-reads all Gaussians for each frame."""

    def __init__(self, problem, scene: DeviceScene, target, ext, delta, opts: RenderOptions, pair_capacity=None):
        self.scene, self.ext, self.delta = scene, ext, delta
        self.plans = [Plan.for_problem(problem, scene, opts, None if pair_capacity is None else pair_capacity,
                                       frame_ids=[i]) for i in range(len(problem.frames))]
        self.targets, off = [], 0
        for p in self.plans:
            n = p.batch.num_pixels
            self.targets.append(target[off:off + n])
            off += n
        self.total = off
        self.loss = [torch.zeros(1, dtype=torch.float64, device=scene.X.device) for _ in self.plans]
        self.dL = [torch.zeros_like(p.rgb) for p in self.plans]
        self.grads = empty_grads(scene, problem.num_cameras)

    def __call__(self):
        for i, p in enumerate(self.plans):
            p.forward(self.scene, self.ext, self.delta)
            n = p.batch.num_pixels
            capi.gs_loss_l1(p.batch, p.rgb, self.targets[i], n / self.total, self.loss[i], self.dL[i], p.ws)
            p.backward(self.scene, self.dL[i], self.grads, self.ext, accumulate=i > 0)
        return self.loss
