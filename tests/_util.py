"""Helpers shared by the GPU tests: build the library, move seeded problems to
the device, run the CUDA path through the C-ABI and compare with the oracle."""
import numpy as np
import torch

import oracle
from paper_2403_11577_gb300 import build, capi, render, scenes


def ensure_built():
    build.build()
    capi.lib()


def ext_delta(problem, which="current", device="cuda"):
    ext = problem.ext if which == "current" else problem.ext_target
    delta = problem.delta if which == "current" else problem.delta_target
    return (torch.tensor(np.asarray(ext, np.float64), device=device),
            torch.tensor(np.asarray(delta, np.float64), device=device))


def setup(problem, opts=None, pair_capacity=None, frame_ids=None):
    scene = render.DeviceScene.from_problem(problem)
    opts = opts or render.RenderOptions(tile=problem.tile)
    plan = render.Plan.for_problem(problem, scene, opts, pair_capacity, frame_ids)
    ext, delta = ext_delta(problem)
    return scene, plan, ext, delta


def oracle_opts(opts: render.RenderOptions) -> oracle.Opts:
    return oracle.Opts(near_z=opts.near_z, lowpass=opts.lowpass, alpha_min=opts.alpha_min,
                       alpha_max=opts.alpha_max, t_min=opts.t_min, scale_max=opts.scale_max,
                       bg=tuple(opts.bg), frustum_margin=opts.frustum_margin)


def last_gaussian_ids(plan, frame_i):
    """Gaussian id (within the scene) of each pixel's last composited
    Gaussian, -1 if none, as [H*W] from the GPU's sorted pairs."""
    fr = plan.frame(frame_i)
    H, W, T = fr.height - fr.row0, fr.width, plan.opts.tile  # rows of the (cropped) image
    last = plan.image(plan.last, frame_i).cpu().numpy().reshape(-1)
    P = int(plan.stats().num_pairs)
    vals = plan.ws_view(capi.WS_VALS, torch.int32, max(P, 1)).cpu().numpy().view(np.uint32)
    ranges = plan.ws_view(capi.WS_RANGES, torch.int32, 2 * plan.batch.num_tiles).cpu().numpy().view(np.uint32)
    ranges = ranges.reshape(-1, 2)
    v, u = np.divmod(np.arange(H * W), W)  # v counted from the first rendered row
    tile = fr.tile_offset + (v // T) * fr.tiles_x + (u // T)
    out = np.full(H * W, -1, np.int64)
    has = last > 0
    out[has] = vals[ranges[tile[has], 0] + last[has] - 1]
    return out


def sample_pixels(rng, cam, n):
    u = rng.integers(0, cam.width, n)
    v = rng.integers(0, cam.height, n)
    return np.stack([u, v], 1)


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def oracle_outcomes(scene, frame, ext, delta, opts, pixels=None):
    """The oracle's render of a frame's pixels together with every outcome of
    their ambiguous float32 decisions (oracle.render(..., alternatives=True))."""
    return oracle.render(scene, frame, ext, delta, oracle_opts(opts), pixels, alternatives=True)


def match_outcomes(rgb_g, T_g, last_g, ref, tol):
    """Compare the GPU's colour, transmittance and last Gaussian per pixel
    with the oracle's outcomes: the FP64 one and, where a skip or stop
    decision is ambiguous in float32, each alternative (every one is a
    correct float32 result).  Returns (decided, matched): decided = the
    oracle gives the pixel an outcome set (no undecided depth order, near
    plane culling or branch overflow); matched = the GPU equals one outcome
    within tol, with the same last Gaussian."""
    rgb_o, T_o, last_o, flags, (nalt, alt) = ref
    rgb_g = np.asarray(rgb_g, np.float64).reshape(-1, 3)
    T_g = np.asarray(T_g, np.float64).reshape(-1)
    last_g = np.asarray(last_g).reshape(-1)
    matched = (np.abs(rgb_g - rgb_o).max(1) <= tol) & (np.abs(T_g - T_o) <= tol) & (last_g == last_o)
    for k in range(alt.shape[1]):
        a = alt[:, k]
        matched |= (nalt > k) & (np.abs(rgb_g - a[:, :3]).max(1) <= tol) & (np.abs(T_g - a[:, 3]) <= tol) & \
                   (last_g == a[:, 4].astype(np.int64))
    decided = (flags & oracle.FLAGS_UNDECIDED) == 0
    return decided, matched
