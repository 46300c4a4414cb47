"""Autotuner for the tile edge and the shared-memory batch of the renderer.

For every (tile, batch) in {8, 16, 32} x {64, 128, 256} it plans the
workload, captures one calibration iteration in a CUDA graph and times
replays with CUDA events; the fastest setting is cached in a JSON file keyed
by the GPU name and a signature of the workload (Gaussians, frame sizes).
The image does not depend on the setting (the same Gaussians meet each pixel
in the same order), so the choice is purely a speed choice.
"""
from __future__ import annotations

import json
import os

import torch

from . import render

TILES = (8, 16, 32)
BATCHES = (64, 128, 256)
CACHE = os.environ.get("GS3DCALIB_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache",
                                    "autotune.json"))


def signature(problem, scene) -> str:
    sizes = sorted({(f.camera.width, f.camera.height) for f in problem.frames})
    return "N%d_F%d_%s" % (scene.n, len(problem.frames), "_".join("%dx%d" % s for s in sizes))


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    json.dump(d, open(tmp, "w"), indent=1)
    os.replace(tmp, CACHE)


def plan_with_capacity(problem, scene, opts, ext, delta, cap=None):
    """A plan whose pair capacity holds the batch at (ext, delta): the
    capacity is doubled until the binning reports no overflow."""
    frames = render.Plan.frames_from_problem(problem, scene)
    cap = cap or render.default_pair_capacity(frames, opts.tile)
    while True:
        plan = render.Plan(frames, scene.n, problem.num_cameras, len(problem.scenes), opts, cap, scene.X.device)
        plan.forward(scene, ext, delta)
        if not plan.stats().status & 1 or cap >= (1 << 32) - 1:
            return plan
        cap = int(min(2 * cap, (1 << 32) - 1))


def time_setting(problem, scene, target, ext, delta, tile, batch, reps=5, base=None):
    opts = render.RenderOptions(tile=tile, batch=batch, **(base or {}))
    plan = plan_with_capacity(problem, scene, opts, ext, delta)
    step = render.CalibStep(plan, scene, target, ext, delta, graph=True)
    for _ in range(2):
        step()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    st = plan.stats()
    del step, plan
    return ms, st.status


def tune(problem, scene, reps=5, use_cache=True, verbose=False):
    """Return {"tile", "batch", "ms", "table"} for this GPU and workload."""
    key = "%s|%s" % (torch.cuda.get_device_name(), signature(problem, scene))
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    dev = scene.X.device
    ext = torch.tensor(problem.ext, dtype=torch.float64, device=dev)
    delta = torch.tensor(problem.delta, dtype=torch.float64, device=dev)
    t_ext = problem.ext_target if problem.ext_target is not None else problem.ext
    t_del = problem.delta_target if problem.delta_target is not None else problem.delta
    ref = render.Plan.for_problem(problem, scene, render.RenderOptions(tile=16, batch=128))
    ref.forward(scene, torch.tensor(t_ext, dtype=torch.float64, device=dev),
                torch.tensor(t_del, dtype=torch.float64, device=dev))
    target = ref.rgb.clone()
    del ref
    table = {}
    for tile in TILES:
        for batch in BATCHES:
            ms, status = time_setting(problem, scene, target, ext, delta, tile, batch, reps)
            table["%d/%d" % (tile, batch)] = ms if status == 0 else None
            if verbose:
                print("tile %2d batch %3d: %.3f ms/iter (status %d)" % (tile, batch, ms, status))
    ok = {k: v for k, v in table.items() if v is not None}
    best = min(ok, key=ok.get)
    tile, batch = (int(x) for x in best.split("/"))
    res = {"tile": tile, "batch": batch, "ms": ok[best], "table": table}
    cache[key] = res
    _save(cache)
    return res
