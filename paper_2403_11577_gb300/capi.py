"""ctypes binding of libgs3dcalib.so (include/gs3dcalib.h).

Argument marshalling only: every function takes torch tensors, checks their
dtype, device and contiguity, and passes raw pointers plus the current CUDA
stream to the C entry point of the same name.  There is no fallback: if the
library is not built, or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

# --------------------------------------------------------------- structures


class GsFrame(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("camera_id", C.c_int32), ("traj_id", C.c_int32),
                ("gauss_offset", C.c_int32), ("gauss_count", C.c_int32), ("timestamp", C.c_double),
                ("record_offset", C.c_int64), ("pixel_offset", C.c_int64), ("tile_offset", C.c_int32),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("row0", C.c_int32)]


class GsOpts(C.Structure):
    _fields_ = [("near_z", C.c_float), ("lowpass", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("t_min", C.c_float), ("scale_max", C.c_float),
                ("bg", C.c_float * 3), ("tile", C.c_int32), ("batch", C.c_int32), ("frustum_margin", C.c_float),
                ("exact_tiles", C.c_int32)]


class GsBatch(C.Structure):
    _fields_ = [("frames_dev", C.c_void_p), ("num_frames", C.c_int32), ("num_cameras", C.c_int32),
                ("num_trajs", C.c_int32), ("num_gaussians", C.c_int32), ("tile", C.c_int32),
                ("num_tiles", C.c_int32), ("num_records", C.c_int64), ("num_pixels", C.c_int64),
                ("pair_capacity", C.c_int64)]


class GsNgp(C.Structure):
    _fields_ = [("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3), ("levels", C.c_int32),
                ("log2_table", C.c_int32), ("res", C.c_int32 * 16)]


class GsStats(C.Structure):
    _fields_ = [("status", C.c_uint32), ("reserved", C.c_uint32), ("num_pairs", C.c_uint64),
                ("eval_fwd", C.c_uint64), ("eval_bwd", C.c_uint64)]


GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_UNSUPPORTED = 0, 1, 2, 3, 4
GS_DEV_PAIR_OVERFLOW, GS_DEV_NONFINITE = 1, 2
(GS_PROF_NONE, GS_PROF_PROJECT, GS_PROF_BIN_SORT, GS_PROF_RENDER_FWD, GS_PROF_RENDER_BWD, GS_PROF_PROJECT_BWD,
 GS_PROF_LOSS) = range(7)
WS_STATS, WS_POSE32, WS_POSE64, WS_RECT, WS_DEPTH, WS_SPLAT, WS_GRAD2D, WS_KEYS, WS_VALS, WS_RANGES = range(10)

_P = C.c_void_p
_SIGS = {
    "gs_version": ([], C.c_char_p),
    "gs_struct_sizes": ([_P, C.c_int32], C.c_int32),
    "gs_profile_events": ([C.c_int32, _P, _P], C.c_int32),
    "gs_batch_init": ([_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64, _P, _P], C.c_int32),
    "gs_workspace_size": ([_P], C.c_size_t),
    "gs_workspace_offsets": ([_P, _P, C.c_int32], C.c_int32),
    "gs_read_stats": ([_P, _P, _P, _P], C.c_int32),
    "gs_reset_status": ([_P, _P, _P], C.c_int32),
    "gs_pose_compose": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int32),
    "gs_project": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int32),
    "gs_bin_sort": ([_P, _P, _P, _P], C.c_int32),
    "gs_render_fwd": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int32),
    "gs_loss_l1": ([_P, _P, _P, C.c_int64, C.c_float, _P, _P, _P, _P], C.c_int32),
    "gs_loss_photo": ([_P, _P, _P, C.c_float, C.c_float, _P, _P, _P, _P], C.c_int32),
    "gs_render_bwd": ([_P] * 15 + [C.c_int32, _P], C.c_int32),
    "gs_pose_grad": ([_P] * 6 + [C.c_int32, _P], C.c_int32),
    "gs_bin_sort_noalloc": ([_P] * 9, C.c_int32),
    "gs_voxel_scratch_size": ([C.c_int64], C.c_size_t),
    "gs_ngp_param_count": ([_P], C.c_int64),
    "gs_ngp_fault": ([_P], C.c_int32),
    "gs_ngp_forward": ([_P, _P, _P, C.c_int64, _P, _P, _P, _P, _P], C.c_int32),
    "gs_ngp_backward": ([_P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P], C.c_int32),
    "gs_voxel_downsample": ([_P, C.c_int64, C.c_float, _P, _P, _P, _P], C.c_int32),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libgs3dcalib.so is not built (expected at %s); run "
                               "paper_2403_11577_gb300.build.build()" % path)
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        sizes = (C.c_size_t * 4)()
        L.gs_struct_sizes(sizes, 4)
        mine = [C.sizeof(GsFrame), C.sizeof(GsOpts), C.sizeof(GsBatch), C.sizeof(GsStats)]
        if list(sizes) != mine:
            raise RuntimeError("struct layout mismatch with libgs3dcalib.so: %s vs %s" % (list(sizes), mine))
        _lib = L
    return _lib


def declared_symbols(header: str | None = None):
    """Names of the functions declared in include/gs3dcalib.h."""
    import re
    header = header or os.path.join(_build.INCLUDE, "gs3dcalib.h")
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gs_[a-z0-9_]+)\s*\(", text, re.M)))


class GsError(RuntimeError):
    pass


def _check(code, what):
    if code != GS_OK:
        raise GsError("%s failed with status %d" % (what, code))


def _ptr(t, dtype=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


F32, F64, I32 = torch.float32, torch.float64, torch.int32

# ------------------------------------------------------------ entry points


def gs_version() -> str:
    return lib().gs_version().decode()


def gs_struct_sizes():
    """sizeof(gs_frame), sizeof(gs_opts), sizeof(gs_batch), sizeof(gs_stats)."""
    out = (C.c_size_t * 4)()
    n = lib().gs_struct_sizes(out, 4)
    return [int(out[i]) for i in range(n)]


def gs_profile_events(kernel, start=None, stop=None):
    """Bracket every launch of `kernel` (GS_PROF_*) with the given
    torch.cuda.Event objects (timing enabled); GS_PROF_NONE disables."""
    for ev in (start, stop):
        if ev is not None and not ev.cuda_event:  # torch creates the event on first record
            ev.record()
    if start is not None or stop is not None:
        torch.cuda.synchronize()
    s = C.c_void_p(start.cuda_event) if start is not None else None
    e = C.c_void_p(stop.cuda_event) if stop is not None else None
    _check(lib().gs_profile_events(int(kernel), s, e), "gs_profile_events")


def gs_batch_init(frames_host, num_gaussians, num_cameras, num_trajs, tile, pair_capacity, frames_dev):
    """frames_host: ctypes array of GsFrame (filled in place); frames_dev: a
    CUDA uint8 tensor of len(frames_host) * sizeof(GsFrame) bytes."""
    b = GsBatch()
    _check(lib().gs_batch_init(frames_host, len(frames_host), num_gaussians, num_cameras, num_trajs, tile,
                               pair_capacity, _ptr(frames_dev, torch.uint8, "frames_dev"), C.byref(b)),
           "gs_batch_init")
    return b


def gs_workspace_size(batch) -> int:
    n = lib().gs_workspace_size(C.byref(batch))
    if n == 0:
        raise GsError("gs_workspace_size: invalid batch")
    return int(n)


def gs_workspace_offsets(batch):
    off = (C.c_size_t * 10)()
    n = lib().gs_workspace_offsets(C.byref(batch), off, 10)
    return [int(off[i]) for i in range(n)]


def gs_read_stats(batch, ws, stream=None) -> GsStats:
    st = GsStats()
    _check(lib().gs_read_stats(C.byref(batch), _ptr(ws, torch.uint8, "ws"), _stream(stream), C.byref(st)),
           "gs_read_stats")
    return st


def gs_reset_status(batch, ws, stream=None):
    _check(lib().gs_reset_status(C.byref(batch), _ptr(ws, torch.uint8, "ws"), _stream(stream)), "gs_reset_status")


def gs_pose_compose(batch, traj_t, traj_pose, traj_offset, ext, delta, ws, stream=None):
    _check(lib().gs_pose_compose(C.byref(batch), _ptr(traj_t, F64, "traj_t"), _ptr(traj_pose, F64, "traj_pose"),
                                 _ptr(traj_offset, I32, "traj_offset"), _ptr(ext, F64, "ext"),
                                 _ptr(delta, F64, "delta"), _ptr(ws, torch.uint8, "ws"), _stream(stream)),
           "gs_pose_compose")


def gs_project(batch, X, quat, log_scale, logit_opacity, opts, ws, stream=None):
    _check(lib().gs_project(C.byref(batch), _ptr(X, F32, "X"), _ptr(quat, F32, "quat"),
                            _ptr(log_scale, F32, "log_scale"), _ptr(logit_opacity, F32, "logit_opacity"),
                            C.byref(opts), _ptr(ws, torch.uint8, "ws"), _stream(stream)), "gs_project")


def gs_bin_sort(batch, opts, ws, stream=None):
    _check(lib().gs_bin_sort(C.byref(batch), C.byref(opts), _ptr(ws, torch.uint8, "ws"), _stream(stream)),
           "gs_bin_sort")


def gs_render_fwd(batch, colors, opts, ws, out_rgb, out_T, out_last, stream=None):
    _check(lib().gs_render_fwd(C.byref(batch), _ptr(colors, F32, "colors"), C.byref(opts),
                               _ptr(ws, torch.uint8, "ws"), _ptr(out_rgb, F32, "out_rgb"), _ptr(out_T, F32, "out_T"),
                               _ptr(out_last, I32, "out_last"), _stream(stream)), "gs_render_fwd")


def gs_loss_l1(batch, rgb, target, scale, out_loss, out_grad, ws, stream=None):
    n = rgb.numel()
    if target.numel() != n or (out_grad is not None and out_grad.numel() != n):
        raise ValueError("gs_loss_l1: size mismatch")
    _check(lib().gs_loss_l1(C.byref(batch), _ptr(rgb, F32, "rgb"), _ptr(target, F32, "target"), n, float(scale),
                            _ptr(out_loss, F64, "out_loss"), _ptr(out_grad, F32, "out_grad", allow_none=True),
                            _ptr(ws, torch.uint8, "ws"), _stream(stream)), "gs_loss_l1")


def gs_loss_photo(batch, rgb, target, lambda1, out_loss, out_grad, ws, scale=1.0, stream=None):
    """out_loss: float64 [3] (L_photo, L1, D-SSIM); out_grad: float32 like rgb or None."""
    n = 3 * batch.num_pixels
    if rgb.numel() != n or target.numel() != n or (out_grad is not None and out_grad.numel() != n):
        raise ValueError("gs_loss_photo: size mismatch")
    if out_loss.numel() < 3:
        raise ValueError("gs_loss_photo: out_loss needs 3 doubles")
    _check(lib().gs_loss_photo(C.byref(batch), _ptr(rgb, F32, "rgb"), _ptr(target, F32, "target"), float(lambda1),
                               float(scale), _ptr(out_loss, F64, "out_loss"),
                               _ptr(out_grad, F32, "out_grad", allow_none=True), _ptr(ws, torch.uint8, "ws"),
                               _stream(stream)), "gs_loss_photo")


def gs_render_bwd(batch, X, quat, log_scale, logit_opacity, colors, opts, ws, out_T, out_last, dL_drgb,
                  d_quat, d_log_scale, d_logit_opacity, d_colors, accumulate=True, stream=None):
    _check(lib().gs_render_bwd(C.byref(batch), _ptr(X, F32, "X"), _ptr(quat, F32, "quat"),
                               _ptr(log_scale, F32, "log_scale"), _ptr(logit_opacity, F32, "logit_opacity"),
                               _ptr(colors, F32, "colors"), C.byref(opts), _ptr(ws, torch.uint8, "ws"),
                               _ptr(out_T, F32, "out_T"), _ptr(out_last, I32, "out_last"),
                               _ptr(dL_drgb, F32, "dL_drgb"), _ptr(d_quat, F32, "d_quat"),
                               _ptr(d_log_scale, F32, "d_log_scale"), _ptr(d_logit_opacity, F32, "d_logit_opacity"),
                               _ptr(d_colors, F32, "d_colors"), int(bool(accumulate)), _stream(stream)),
           "gs_render_bwd")


def gs_pose_grad(batch, ext, ws, d_ext, d_delta, d_xi=None, accumulate=False, stream=None):
    _check(lib().gs_pose_grad(C.byref(batch), _ptr(ext, F64, "ext"), _ptr(ws, torch.uint8, "ws"),
                              _ptr(d_ext, F64, "d_ext"), _ptr(d_delta, F64, "d_delta"),
                              _ptr(d_xi, F64, "d_xi", allow_none=True), int(bool(accumulate)), _stream(stream)),
           "gs_pose_grad")


def gs_ngp_param_count(cfg):
    return int(lib().gs_ngp_param_count(C.byref(cfg)))


def gs_ngp_forward(cfg, theta, X, rgb, logit_opacity, log_scale, quat, stream=None):
    _check(lib().gs_ngp_forward(C.byref(cfg), _ptr(theta, F32, "theta"), _ptr(X, F32, "X"), X.shape[0],
                                _ptr(rgb, F32, "rgb"), _ptr(logit_opacity, F32, "logit_opacity"),
                                _ptr(log_scale, F32, "log_scale"), _ptr(quat, F32, "quat"), _stream(stream)),
           "gs_ngp_forward")


def gs_ngp_backward(cfg, theta, X, d_rgb, d_logit_opacity, d_log_scale, d_quat, d_theta, stream=None):
    _check(lib().gs_ngp_backward(C.byref(cfg), _ptr(theta, F32, "theta"), _ptr(X, F32, "X"), X.shape[0],
                                 _ptr(d_rgb, F32, "d_rgb"), _ptr(d_logit_opacity, F32, "d_logit_opacity"),
                                 _ptr(d_log_scale, F32, "d_log_scale"), _ptr(d_quat, F32, "d_quat"),
                                 _ptr(d_theta, F32, "d_theta"), _stream(stream)), "gs_ngp_backward")


def gs_ngp_set_wait_limit(ns):
    """Bound (ns) on the hash-grid kernels' waits for their MMAs; 0 makes the
    first unfinished wait give up (a test hook); default 10**9."""
    _check(lib().gs_ngp_set_wait_limit(C.c_uint64(int(ns))), "gs_ngp_set_wait_limit")


def gs_ngp_fault():
    """Read and clear the hash-grid kernels' fault word (bit 0: a tensor-core
    wait ran out; that call's outputs are incomplete)."""
    v = C.c_uint32(0)
    _check(lib().gs_ngp_fault(C.byref(v)), "gs_ngp_fault")
    return int(v.value)


def gs_voxel_scratch_size(n):
    return int(lib().gs_voxel_scratch_size(int(n)))


def gs_voxel_downsample(X, voxel, out_index, out_count, scratch, stream=None):
    """X: float32 [n,3]; out_index: int32 [n]; out_count: int64 [1] (as uint64);
    scratch: uint8 tensor of gs_voxel_scratch_size(n) bytes, 256-byte aligned."""
    n = X.shape[0]
    if out_index.numel() < n or out_count.numel() < 1 or scratch.numel() < gs_voxel_scratch_size(n):
        raise ValueError("gs_voxel_downsample: buffer too small")
    _check(lib().gs_voxel_downsample(_ptr(X, F32, "X"), n, float(voxel), _ptr(out_index, torch.int32, "out_index"),
                                     _ptr(out_count, torch.int64, "out_count"), _ptr(scratch, torch.uint8, "scratch"),
                                     _stream(stream)), "gs_voxel_downsample")


def gs_bin_sort_noalloc(batch, opts, rect, depth, keys, vals, ranges, out_pairs, stream=None):
    """Tile binning + depth sort into the caller's buffers, with no device
    allocation and no workspace (for callers that cannot allocate).
    rect: int32/uint32 [R*2]; depth: float32 [R]; keys: int64 [cap];
    vals: int32 [cap]; ranges: int32 [T*2]; out_pairs: int64 [2]."""
    _check(lib().gs_bin_sort_noalloc(C.byref(batch), C.byref(opts), _ptr(rect, None, "rect"),
                                     _ptr(depth, F32, "depth"), _ptr(keys, torch.int64, "keys"),
                                     _ptr(vals, torch.int32, "vals"), _ptr(ranges, torch.int32, "ranges"),
                                     _ptr(out_pairs, torch.int64, "out_pairs"), _stream(stream)),
           "gs_bin_sort_noalloc")
