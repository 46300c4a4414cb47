"""FP64 CPU oracle for the 3DGS-Calib splatting path -- TEST INFRASTRUCTURE.

Only the tests, `__graft_entry__.smoke()` and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and never
calls it; it consumes the seeded inputs of `paper_2403_11577_gb300.scenes`
(a module with none of the method's arithmetic).

The computation lives in `gs_oracle.c` (plain C, double precision); this
module only marshals numpy arrays.  Citations (paper sections and equations)
are in the C source next to each step.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class OrOpts(C.Structure):
    _fields_ = [("near_z", C.c_double), ("lowpass", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("t_min", C.c_double), ("scale_max", C.c_double),
                ("bg", C.c_double * 3), ("frustum_margin", C.c_double)]


class OrCam(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double)]


# Per-pixel flags (see gs_oracle.c): the renderer decides in float32, the
# oracle in FP64 with a bound on the float32 evaluation's error.
#   FLAG_BRANCH: an ambiguous skip or stop decision; every outcome is given
#     as an alternative result (render(..., alternatives=True)), and the
#     pixel's gradient depends on the outcome.
#   FLAG_CLAMP_EDGE: an alpha within the bound of alpha_max (colour
#     continuous, gradient not).
#   FLAG_DEPTH_TIE / FLAG_NEAR_EDGE / FLAG_BRANCH_LIMIT: the depth order or
#     the near-plane culling is not decided in float32, or more outcomes than
#     MAX_BRANCHES: no outcome set is given (FLAGS_UNDECIDED).
FLAG_BRANCH, FLAG_CLAMP_EDGE, FLAG_DEPTH_TIE, FLAG_NEAR_EDGE, FLAG_BRANCH_LIMIT = 1, 2, 4, 16, 32
FLAGS_UNDECIDED = FLAG_DEPTH_TIE | FLAG_NEAR_EDGE | FLAG_BRANCH_LIMIT
MAX_BRANCHES = 16


@dataclass
class Opts:
    """Renderer readings of what the paper leaves open (defaults follow the
    3DGS renderer the paper builds on, Sec. III-B)."""
    near_z: float = 0.2
    lowpass: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    scale_max: float = float("inf")
    bg: tuple = (0.0, 0.0, 0.0)
    frustum_margin: float = 0.15

    def c(self) -> OrOpts:
        return OrOpts(self.near_z, self.lowpass, self.alpha_min, self.alpha_max, self.t_min,
                      self.scale_max, (C.c_double * 3)(*self.bg), self.frustum_margin)


SMOOTH = Opts(alpha_min=0.0, alpha_max=1.0, t_min=0.0)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.or_l1.restype = C.c_double
        _lib.or_dssim.restype = C.c_double
        _lib.or_bin_sort.restype = C.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cam(cam) -> OrCam:
    return OrCam(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy))


def lidar_pose(scene, tau):
    """T_L(tau): (R_wL, p_wL, dR/dtau, dp/dtau), Sec. III-A."""
    R, p, dR, dp = np.zeros(9), np.zeros(3), np.zeros(9), np.zeros(3)
    tt, tp, tq = _f64(scene.traj_t), _f64(scene.traj_p), _f64(scene.traj_q)
    lib().or_lidar_pose(_p(tt), _p(tp), _p(tq), C.c_int(len(tt)), C.c_double(tau),
                        _p(R), _p(p), _p(dR), _p(dp))
    return R.reshape(3, 3), p, dR.reshape(3, 3), dp


def frame_pose(scene, ext, delta, t):
    """World-to-camera (R_cw, t_cw) of a frame at camera time t (Eq. 1-2)."""
    R, tc = np.zeros(9), np.zeros(3)
    tt, tp, tq = _f64(scene.traj_t), _f64(scene.traj_p), _f64(scene.traj_q)
    e = _f64(ext)
    lib().or_frame_pose(_p(tt), _p(tp), _p(tq), C.c_int(len(tt)), _p(e), C.c_double(delta),
                        C.c_double(t), _p(R), _p(tc))
    return R.reshape(3, 3), tc


def _gauss(scene):
    """Gaussian parameters widened to float64 (exact for float32 inputs)."""
    return (_f64(scene.X), _f64(scene.quat), _f64(scene.log_scale), _f64(scene.logit_opacity),
            _f64(scene.rgb))


def project(scene, cam, R_cw, t_cw, opts: Opts = Opts(), tile: int = 16):
    """Per-Gaussian projection (FP64) for one camera pose."""
    X, q, ls, lo, _ = _gauss(scene)
    n = scene.n
    out = dict(valid=np.zeros(n, np.int32), depth=np.zeros(n), mean=np.zeros((n, 2)),
               conic=np.zeros((n, 3)), opacity=np.zeros(n), extent=np.zeros((n, 2)),
               cov=np.zeros((n, 3)), rect=np.zeros((n, 4), np.int32))
    b = np.zeros((n, 7))
    lib().or_project(C.c_int(n), _p(X), _p(q), _p(ls), _p(lo), C.byref(_cam(cam)),
                     _p(_f64(R_cw)), _p(_f64(t_cw)), C.byref(opts.c()), C.c_int(tile),
                     _p(out["valid"]), _p(out["depth"]), _p(out["mean"]), _p(out["conic"]),
                     _p(out["opacity"]), _p(out["extent"]), _p(out["cov"]), _p(out["rect"]), _p(b))
    # depth key (float32) and whether its rounding / the near-plane culling
    # is undecided; bounds of the float32 mean, conic and log2 opacity
    out["zkey"] = b[:, 0].astype(np.float32)
    out["zamb"] = b[:, 1] != 0
    out["near_undecided"] = b[:, 2] != 0
    out["mean_err"] = b[:, 3:5]
    out["conic_err"] = b[:, 5]
    out["logop_err"] = b[:, 6]
    return out


def _pix(pixels):
    if pixels is None:
        return None, 0
    pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    return pix, len(pix)


def render_pose(scene, cam, R_cw, t_cw, opts: Opts = Opts(), pixels=None, alternatives=False):
    """Render one frame for a given world-to-camera pose.

    Returns rgb [P,3], T_final [P], last [P] (Gaussian id or -1), flags [P]
    for the FP64 outcome of every decision; P = all pixels in row-major
    order, or the given (u, v) pixels.  With alternatives=True a fifth item
    (nalt [P], alt [P, MAX_BRANCHES-1, 5]) gives, per pixel, the other
    outcomes of its ambiguous decisions as (r, g, b, T_final, last)."""
    X, q, ls, lo, rgb = _gauss(scene)
    pix, npix = _pix(pixels)
    P = npix if pix is not None else cam.width * cam.height
    out_rgb, out_T = np.zeros((P, 3)), np.zeros(P)
    out_last, out_flags = np.zeros(P, np.int32), np.zeros(P, np.int32)
    nalt = np.zeros(P, np.int32) if alternatives else None
    alt = np.zeros((P, MAX_BRANCHES - 1, 5)) if alternatives else None
    lib().or_render(C.c_int(scene.n), _p(X), _p(q), _p(ls), _p(lo), _p(rgb), C.byref(_cam(cam)),
                    _p(_f64(R_cw)), _p(_f64(t_cw)), C.byref(opts.c()), C.c_int(npix),
                    _p(pix) if pix is not None else None,
                    _p(out_rgb), _p(out_T), _p(out_last), _p(out_flags),
                    _p(nalt) if alternatives else None, _p(alt) if alternatives else None)
    if alternatives:
        return out_rgb, out_T, out_last, out_flags, (nalt, alt)
    return out_rgb, out_T, out_last, out_flags


def _frame_pixels(frame, pixels):
    """The frame's image pixels (rows row0 .. H-1, row-major) when no pixel
    list is given and the frame is cropped."""
    row0 = getattr(frame, "row0", 0)
    if pixels is not None or row0 == 0:
        return pixels
    cam = frame.camera
    v, u = np.mgrid[row0:cam.height, 0:cam.width]
    return np.stack([u.ravel(), v.ravel()], 1)


def render(scene, frame, ext, delta, opts: Opts = Opts(), pixels=None, alternatives=False):
    """Render a frame at the pose of Eq. 1 for extrinsic ext (omega, t) and
    time offset delta (a cropped frame: its rows row0 .. H-1)."""
    R, t = frame_pose(scene, ext, delta, frame.timestamp)
    return render_pose(scene, frame.camera, R, t, opts, _frame_pixels(frame, pixels), alternatives)


def backward(scene, frame, ext, delta, dL_dC, opts: Opts = Opts(), pixels=None):
    """Gradients of sum_p dL_dC[p] . C(p) for one frame: Gaussian parameters
    (q, log_scale, logit_opacity, rgb), calibration (ext[6], delta), and the
    per-Gaussian 2D gradients (mean2d, conic, opacity)."""
    X, q, ls, lo, rgb = _gauss(scene)
    pix, npix = _pix(_frame_pixels(frame, pixels))
    n = scene.n
    g = dict(quat=np.zeros((n, 4)), log_scale=np.zeros((n, 3)), logit_opacity=np.zeros(n),
             rgb=np.zeros((n, 3)), ext=np.zeros(6), delta=np.zeros(1), mean2d=np.zeros((n, 2)),
             conic=np.zeros((n, 3)), opacity=np.zeros(n))
    tt, tp, tq = _f64(scene.traj_t), _f64(scene.traj_p), _f64(scene.traj_q)
    dl = _f64(dL_dC).reshape(-1, 3)
    lib().or_backward(C.c_int(n), _p(X), _p(q), _p(ls), _p(lo), _p(rgb), C.byref(_cam(frame.camera)),
                      _p(tt), _p(tp), _p(tq), C.c_int(len(tt)), _p(_f64(ext)), C.c_double(delta),
                      C.c_double(frame.timestamp), C.byref(opts.c()), C.c_int(npix),
                      _p(pix) if pix is not None else None, _p(dl),
                      _p(g["quat"]), _p(g["log_scale"]), _p(g["logit_opacity"]), _p(g["rgb"]),
                      _p(g["ext"]), _p(g["delta"]), _p(g["mean2d"]), _p(g["conic"]), _p(g["opacity"]))
    return g


def l1(C_img, C_gt):
    """Mean absolute error (the L1 term of Eq. 4) and its gradient."""
    a, b = _f64(C_img).ravel(), _f64(C_gt).ravel()
    grad = np.zeros_like(a)
    loss = lib().or_l1(C.c_int64(a.size), _p(a), _p(b), _p(grad))
    return loss, grad.reshape(np.shape(C_img))


def dssim(imgs, tgts, with_map=False):
    """D-SSIM part of Eq. 4 (1 - mean SSIM, 11x11 Gaussian window of sigma
    1.5, zero padding) over a batch of HxWx3 images, and its gradient with
    respect to the rendered images (a list like `imgs`)."""
    shapes = [np.shape(a) for a in imgs]
    rows = np.array([s[0] for s in shapes], np.int32)
    cols = np.array([s[1] for s in shapes], np.int32)
    sizes = [s[0] * s[1] * 3 for s in shapes]
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    a = np.concatenate([_f64(x).ravel() for x in imgs])
    b = np.concatenate([_f64(x).ravel() for x in tgts])
    grad = np.zeros_like(a)
    smap = np.zeros_like(a) if with_map else None
    loss = lib().or_dssim(C.c_int(len(imgs)), rows.ctypes.data_as(C.POINTER(C.c_int32)),
                          cols.ctypes.data_as(C.POINTER(C.c_int32)), off.ctypes.data_as(C.POINTER(C.c_int64)),
                          _p(a), _p(b), _p(grad), _p(smap) if with_map else None)
    grads = [grad[o:o + n].reshape(s) for o, n, s in zip(off, sizes, shapes)]
    if with_map:
        return loss, grads, [smap[o:o + n].reshape(s) for o, n, s in zip(off, sizes, shapes)]
    return loss, grads


def photo_loss(imgs, tgts, lambda1=0.2):
    """L_photo = (1 - lambda1) L1 + lambda1 D-SSIM (Eq. 4, lambda1 = 0.2 in
    the paper) over a batch of HxWx3 images, both means over every value of
    the batch, and its gradient per image."""
    a = np.concatenate([_f64(x).ravel() for x in imgs])
    b = np.concatenate([_f64(x).ravel() for x in tgts])
    l1_loss, g1 = l1(a, b)
    ds, gs = dssim(imgs, tgts)
    off = np.concatenate([[0], np.cumsum([np.size(x) for x in imgs])])
    grads = [(1 - lambda1) * g1[off[i]:off[i + 1]].reshape(np.shape(imgs[i])) + lambda1 * gs[i]
             for i in range(len(imgs))]
    return (1 - lambda1) * l1_loss + lambda1 * ds, grads


def bin_sort(frames_tiles, n_per_frame, rect, depth, cap=None):
    """Tile binning + stable depth order of per-(frame, Gaussian) records.

    frames_tiles: [(tiles_x, tiles_y)] per frame; n_per_frame: records per
    frame.  Returns keys uint64 [P], vals uint32 [P], ranges int64 [T,2]."""
    F = len(frames_tiles)
    rec_off = np.zeros(F + 1, np.int64)
    rec_off[1:] = np.cumsum(n_per_frame)
    tiles_x = np.array([t[0] for t in frames_tiles], np.int32)
    counts = np.array([t[0] * t[1] for t in frames_tiles], np.int64)
    tile_off = np.zeros(F, np.int32)
    tile_off[1:] = np.cumsum(counts)[:-1]
    T = int(counts.sum())
    rect = np.ascontiguousarray(rect, np.int32)
    depth = np.ascontiguousarray(depth, np.float32)
    r = rect.reshape(-1, 4)
    ne = (r[:, 0] <= r[:, 2]) & (r[:, 1] <= r[:, 3])
    P = int((((r[:, 2] - r[:, 0] + 1) * (r[:, 3] - r[:, 1] + 1)).astype(np.int64) * ne).sum())
    cap = P if cap is None else cap
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros((max(T, 1), 2), np.int64)
    got = lib().or_bin_sort(C.c_int(F), _p(rec_off), _p(tile_off), _p(tiles_x), _p(rect), _p(depth),
                            C.c_int64(cap), C.c_int32(T), _p(keys), _p(vals), _p(ranges))
    if got < 0:
        raise OverflowError("pair count %d exceeds capacity %d" % (P, cap))
    return keys[:P], vals[:P], ranges[:T]


# ------------------------------------------------------- voxel downsampling

VOXEL_LIMIT = 1 << 20  # voxel coordinates must lie in (-2^20, 2^20)


def voxel_downsample(X, voxel):
    """Accumulated-LiDAR downsampling (Sec. III-D): one point per occupied
    voxel of edge `voxel`, the point of smallest index.  A point's voxel is
    (floor(x / voxel), floor(y / voxel), floor(z / voxel)) with the quotient
    taken in float32, the points' own precision, so that the integer voxel
    coordinates are decided in the same precision as on the GPU.  Points with
    a non-finite coordinate or a voxel coordinate outside (-2^20, 2^20) are
    dropped.  Returns the kept indices in ascending order."""
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 3)
    with np.errstate(invalid="ignore", over="ignore"):
        q = np.floor(X / np.float32(voxel))
    ok = np.all(np.isfinite(q), axis=1) & np.all(np.abs(q) < VOXEL_LIMIT, axis=1)
    idx = np.nonzero(ok)[0]
    if len(idx) == 0:
        return idx.astype(np.int64)
    _, first = np.unique(q[ok].astype(np.int64), axis=0, return_index=True)
    return np.sort(idx[first]).astype(np.int64)


# ------------------------------------------------------------ problem level

def render_problem(problem, opts: Opts = Opts(), ext=None, delta=None, pixels=None):
    """Render every frame of a problem; returns a list of (rgb, T, last, flags)."""
    ext = problem.ext if ext is None else ext
    delta = problem.delta if delta is None else delta
    out = []
    for f in problem.frames:
        sc = problem.scenes[f.scene_id]
        pix = None if pixels is None else pixels[len(out)]
        out.append(render(sc, f, ext[f.camera_id], float(delta[f.camera_id]), opts, pix))
    return out


def backward_problem(problem, dL_dC_per_frame, opts: Opts = Opts(), ext=None, delta=None, pixels=None):
    """Sum of per-frame backward passes; Gaussian grads per scene, calibration
    grads per camera."""
    ext = problem.ext if ext is None else ext
    delta = problem.delta if delta is None else delta
    scenes = [dict(quat=0, log_scale=0, logit_opacity=0, rgb=0) for _ in problem.scenes]
    d_ext = np.zeros((problem.num_cameras, 6))
    d_delta = np.zeros(problem.num_cameras)
    for i, f in enumerate(problem.frames):
        sc = problem.scenes[f.scene_id]
        pix = None if pixels is None else pixels[i]
        g = backward(sc, f, ext[f.camera_id], float(delta[f.camera_id]), dL_dC_per_frame[i], opts, pix)
        for k in scenes[f.scene_id]:
            scenes[f.scene_id][k] = scenes[f.scene_id][k] + g[k]
        d_ext[f.camera_id] += g["ext"]
        d_delta[f.camera_id] += g["delta"][0]
    return scenes, d_ext, d_delta
