"""The allocation-free binning entry point (gs_bin_sort_noalloc), for
callers that cannot allocate device memory and so cannot provide a
workspace, against the workspace entry point gs_bin_sort on the same
records: values, tile ranges and pair counts must be identical, and the
full 64-bit keys must be the workspace's tile keys over the depth bits of
each pair's record (the sort is integer work, compared bit for bit), on two
calls in a row with different inputs.  This file is collected last on
purpose."""
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
