"""The allocation-free binning entry point (gs_bin_sort_noalloc), for
callers that cannot allocate device memory and so cannot provide a
workspace, against the workspace entry point gs_bin_sort on the same
records: values, tile ranges and pair counts must be identical, and the
full 64-bit keys must be the workspace's tile keys over the depth bits of
each pair's record (the sort is integer work, compared bit for bit), on two
calls in a row with different inputs.  Requests beyond the pair capacity and
rectangles outside their frame write nothing and report it, and the shared
scratch serves the next call.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2403_11577_gb300 import capi, render, scenes

from _util import ensure_built

pytestmark = pytest.mark.gpu


def _plan(frames_wh, counts, cap):
    frames = [dict(width=w, height=h, fx=100.0, fy=100.0, cx=w / 2, cy=h / 2, camera_id=0, traj_id=0,
                   gauss_offset=0, gauss_count=c, timestamp=0.0) for (w, h), c in zip(frames_wh, counts)]
    # the allocation-free entry point bins whole rectangles (it is passed no splat records)
    return render.Plan(frames, max(counts), 1, 1, render.RenderOptions(tile=16, exact_tiles=False), cap)


def _records(plan, seed, frames_wh, counts):
    tiles = [((w + 15) // 16, (h + 15) // 16) for w, h in frames_wh]
    rect, depth = scenes.random_splat_records(seed, tiles, counts, tie_fraction=0.3, max_extent_tiles=6)
    n = len(depth)
    packed = np.zeros((n, 2), np.uint32)
    packed[:, 0] = (rect[:, 0].astype(np.uint32) & 0xFFFF) | ((rect[:, 1].astype(np.uint32) & 0xFFFF) << 16)
    packed[:, 1] = (rect[:, 2].astype(np.uint32) & 0xFFFF) | ((rect[:, 3].astype(np.uint32) & 0xFFFF) << 16)
    plan.ws_view(capi.WS_RECT, torch.int32, 2 * n).copy_(torch.from_numpy(packed.view(np.int32).ravel()))
    plan.ws_view(capi.WS_DEPTH, torch.float32, n).copy_(torch.from_numpy(depth))
    return n


def test_bin_sort_noalloc_matches_workspace_entry_point():
    ensure_built()
    frames_wh = [(1408, 376), (300, 200), (77, 50)]
    counts = [20000, 4000, 600]
    cap = 1 << 20
    plan = _plan(frames_wh, counts, cap)
    T = plan.batch.num_tiles
    keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    vals = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * T, dtype=torch.int32, device="cuda")
    counts_out = torch.empty(2, dtype=torch.int64, device="cuda")
    for call, seed in enumerate((11, 12)):
        n = _records(plan, seed, frames_wh, counts)
        plan.bin_sort()
        st = plan.stats()
        P = int(st.num_pairs)
        assert P > 0 and st.status == 0
        rect = plan.ws_view(capi.WS_RECT, torch.int32, 2 * n)
        depth = plan.ws_view(capi.WS_DEPTH, torch.float32, n)
        keys.fill_(-1)
        vals.fill_(-1)
        capi.gs_bin_sort_noalloc(plan.batch, plan.copts, rect, depth, keys, vals, ranges, counts_out)
        torch.cuda.synchronize()
        assert counts_out.tolist() == [P, P], (call, counts_out.tolist(), P)
        # same order: vals and ranges bit for bit; the full 64-bit keys are the
        # workspace's tile keys over the depth bits of each pair's record
        assert torch.equal(vals[:P], plan.ws_view(capi.WS_VALS, torch.int32, P)), call
        assert torch.equal(ranges, plan.ws_view(capi.WS_RANGES, torch.int32, 2 * T)), call
        k = keys[:P].cpu().numpy().view(np.uint64)
        tile = plan.ws_view(capi.WS_KEYS, torch.int32, P).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal((k >> np.uint64(32)).astype(np.uint32), tile)
        v = vals[:P].cpu().numpy().view(np.uint32).astype(np.int64)
        rec_off = np.array([plan.frame(i).record_offset for i in range(len(frames_wh))])
        tile_off = np.array([plan.frame(i).tile_offset for i in range(len(frames_wh))])
        fr = np.searchsorted(tile_off, tile, side="right") - 1
        dbits = depth.cpu().numpy().view(np.uint32)[rec_off[fr] + v]
        np.testing.assert_array_equal((k & np.uint64(0xFFFFFFFF)).astype(np.uint32), dbits)


def test_bin_sort_noalloc_rejects_oversized_batches():
    ensure_built()
    plan = _plan([(64, 64)], [10], (1 << 20) + 1)
    x = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(capi.GsError, match="status 2"):
        capi.gs_bin_sort_noalloc(plan.batch, plan.copts, x.view(torch.int32), x.view(torch.float32)[:1], x,
                                 x.view(torch.int32), x.view(torch.int32), x[:2])


def _run_noalloc(plan, n, cap):
    T = plan.batch.num_tiles
    keys = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    vals = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((2 * T,), 7, dtype=torch.int32, device="cuda")
    out = torch.full((2,), 5, dtype=torch.int64, device="cuda")
    capi.gs_bin_sort_noalloc(plan.batch, plan.copts, plan.ws_view(capi.WS_RECT, torch.int32, 2 * n),
                             plan.ws_view(capi.WS_DEPTH, torch.float32, n), keys, vals, ranges, out)
    torch.cuda.synchronize()
    return keys, vals, ranges, out.cpu().numpy().view(np.uint64)


def _check_against_workspace(plan, n, cap):
    plan.bin_sort()
    P = int(plan.stats().num_pairs)
    keys, vals, ranges, out = _run_noalloc(plan, n, cap)
    assert out.tolist() == [P, P]
    assert torch.equal(vals[:P], plan.ws_view(capi.WS_VALS, torch.int32, P))
    assert torch.equal(ranges, plan.ws_view(capi.WS_RANGES, torch.int32, 2 * plan.batch.num_tiles))


def test_bin_sort_noalloc_overflow_writes_nothing_then_recovers():
    """More pairs requested than batch->pair_capacity (itself within the
    fixed scratch): nothing is written, out_pairs = [0, requested] and every
    range is empty; a call within capacity right after it is exact again."""
    ensure_built()
    frames_wh, counts = [(640, 480)], [3000]
    small = _plan(frames_wh, counts, 1000)
    n = _records(small, 21, frames_wh, counts)
    r = small.ws_view(capi.WS_RECT, torch.int32, 2 * n).cpu().numpy().view(np.uint32).reshape(n, 2)
    w = (r[:, 1] & 0xFFFF).astype(np.int64) - (r[:, 0] & 0xFFFF) + 1
    h = (r[:, 1] >> 16).astype(np.int64) - (r[:, 0] >> 16) + 1
    requested = int((np.where((w > 0) & (h > 0), w * h, 0)).sum())
    assert requested > 1000
    keys, vals, ranges, out = _run_noalloc(small, n, 1000)
    assert out.tolist() == [0, requested]
    assert int(ranges.abs().sum()) == 0
    assert bool((vals == -1).all()) and bool((keys == -1).all())
    big = _plan(frames_wh, counts, requested + 10)
    n = _records(big, 21, frames_wh, counts)
    _check_against_workspace(big, n, requested + 10)


def test_bin_sort_noalloc_rejects_rectangles_outside_their_frame():
    """A rectangle reaching past its frame's last tile column (or row) would
    name tiles of the next row or frame: the call writes nothing, reports
    out_pairs = [0, UINT64_MAX] with every range empty, and the next call
    with valid rectangles is exact again."""
    ensure_built()
    frames_wh, counts = [(300, 200), (160, 96)], [500, 300]
    cap = 1 << 16
    for bad_field in ("x1", "y1"):
        plan = _plan(frames_wh, counts, cap)
        n = _records(plan, 31, frames_wh, counts)
        rect_t = plan.ws_view(capi.WS_RECT, torch.int32, 2 * n)
        r = rect_t.cpu().numpy().view(np.uint32).reshape(n, 2).copy()
        good = r.copy()
        i = int(np.nonzero(((r[:, 0] & 0xFFFF) <= (r[:, 1] & 0xFFFF)) &
                           ((r[:, 0] >> 16) <= (r[:, 1] >> 16)))[0][0])  # a non-empty record of frame 0
        tiles_x, tiles_y = plan.frame(0).tiles_x, plan.frame(0).tiles_y
        if bad_field == "x1":
            r[i, 1] = (r[i, 1] & 0xFFFF0000) | np.uint32(tiles_x)
        else:
            r[i, 1] = (r[i, 1] & 0xFFFF) | (np.uint32(tiles_y) << 16)
        rect_t.copy_(torch.from_numpy(r.view(np.int32).ravel()))
        keys, vals, ranges, out = _run_noalloc(plan, n, cap)
        assert out.tolist() == [0, 2 ** 64 - 1], bad_field
        assert int(ranges.abs().sum()) == 0
        assert bool((vals == -1).all())
        rect_t.copy_(torch.from_numpy(good.view(np.int32).ravel()))
        _check_against_workspace(plan, n, cap)
