"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/gs3dcalib.h declares, and its host-only planning entry
points behave (no kernel is launched here)."""
import ctypes as C
import re

import pytest

from paper_2403_11577_gb300 import build, capi


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.lib()


def _no_device():
    import torch
    return not torch.cuda.is_available()


# the validation tests pass pointers that are never meant to be dereferenced;
# they run only where no device can be reached, so that a check removed by
# mistake cannot turn into a kernel launch on a fake address
host_only = pytest.mark.skipif(not _no_device(), reason="fake pointers: host-only validation test")


def test_exports_every_declared_symbol(lib):
    declared = capi.declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    # and the binding wraps every one of them under the same name
    for name in declared:
        assert hasattr(capi, name), name


def test_struct_layout_and_version(lib):
    assert capi.gs_version().startswith("gs3dcalib")
    sizes = (C.c_size_t * 4)()
    assert lib.gs_struct_sizes(sizes, 4) == 4
    assert list(sizes) == [C.sizeof(capi.GsFrame), C.sizeof(capi.GsOpts), C.sizeof(capi.GsBatch),
                           C.sizeof(capi.GsStats)]


def test_batch_init_rejects_bad_frames_without_device(lib):
    frames = (capi.GsFrame * 1)()
    frames[0].width, frames[0].height = 0, 10  # invalid size
    b = capi.GsBatch()
    code = lib.gs_batch_init(frames, 1, 10, 1, 1, 16, 1000, C.c_void_p(0x1000), C.byref(b))
    assert code == capi.GS_ERR_INVALID_ARG
    frames[0].width = 64
    for tile in (7, 12, 64):
        assert lib.gs_batch_init(frames, 1, 10, 1, 1, tile, 1000, C.c_void_p(0x1000), C.byref(b)) == \
            capi.GS_ERR_INVALID_ARG
    frames[0].camera_id = 3  # beyond num_cameras
    assert lib.gs_batch_init(frames, 1, 10, 1, 1, 16, 1000, C.c_void_p(0x1000), C.byref(b)) == \
        capi.GS_ERR_INVALID_ARG


def test_workspace_size_is_host_only(lib):
    b = capi.GsBatch()
    b.frames_dev = 0x1000
    b.num_frames, b.num_cameras, b.num_trajs, b.num_gaussians = 8, 1, 1, 1_000_000
    b.tile, b.num_tiles = 16, 8 * 88 * 24
    b.num_records, b.num_pixels, b.pair_capacity = 8_000_000, 8 * 1408 * 376, 100_000_000
    n = capi.gs_workspace_size(b)
    # records (rect 8, depth 4, splat 32, grad2d 48, two key/value buffers of
    # the record sort 2 x 8 B) and pairs (two key/value buffers, 2 x 8 B) dominate
    assert n >= 8_000_000 * (92 + 16) + 100_000_000 * 16
    offs = capi.gs_workspace_offsets(b)
    assert len(offs) == 10 and offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    b.num_frames = 0
    assert lib.gs_workspace_size(C.byref(b)) == 0


def test_header_documents_each_entry_point():
    text = open(build.INCLUDE + "/gs3dcalib.h").read()
    for name in capi.declared_symbols():
        # a comment block directly precedes every declaration
        m = re.search(r"\*/\s*\n(?:[^\n]*\n)?[^\n]*\b%s\s*\(" % name, text)
        assert m, name


@host_only
def test_ngp_entry_points_validate_on_the_host(lib):
    """The hash-grid entry points check their configuration and pointers
    before any device work: the parameter count matches the oracle's layout,
    and bad configurations, NULL outputs and misaligned gradients are
    rejected (the pointers below are never dereferenced)."""
    from oracle import ngp as ongp
    from paper_2403_11577_gb300 import ngp
    cfg = ngp.HashGridConfig([-10.0, -8.0, -1.0], [30.0, 12.0, 9.0], levels=6, log2_table=12)
    o = ongp.NgpConfig(cfg.aabb_min, cfg.aabb_max, levels=6, log2_table=12)
    assert capi.gs_ngp_param_count(cfg.c()) == o.count()
    bad = cfg.c()
    bad.levels = 17
    assert capi.gs_ngp_param_count(bad) == -1
    bad = cfg.c()
    bad.aabb_max[0] = bad.aabb_min[0]  # empty box
    assert capi.gs_ngp_param_count(bad) == -1
    p = C.c_void_p
    ok16, ok8 = p(0x10000), p(0x10008)
    args = [p(0x20000)] * 4
    assert lib.gs_ngp_backward(C.byref(cfg.c()), ok16, ok16, C.c_int64(5), *args, ok8, None) == \
        capi.GS_ERR_INVALID_ARG  # d_theta only 8-byte aligned
    assert lib.gs_ngp_backward(C.byref(bad), ok16, ok16, C.c_int64(5), *args, ok16, None) == capi.GS_ERR_INVALID_ARG
    assert lib.gs_ngp_forward(C.byref(cfg.c()), ok16, ok16, C.c_int64(5), None, *args[:3], None) == \
        capi.GS_ERR_INVALID_ARG  # NULL rgb
    assert lib.gs_ngp_forward(C.byref(cfg.c()), ok16, ok16, C.c_int64(-1), *args, None) == capi.GS_ERR_INVALID_ARG
    assert lib.gs_ngp_fault(None) == capi.GS_ERR_INVALID_ARG


@host_only
def test_entry_points_validate_on_the_host(lib):
    """Every batch entry point rejects a missing batch, a misaligned
    workspace, options that disagree with the batch or lie outside their
    documented ranges, and NULL required pointers with GS_ERR_INVALID_ARG
    before any device work; the allocation-free sort answers exact tiles with
    GS_ERR_UNSUPPORTED, an oversized batch with GS_ERR_CAPACITY and a
    misaligned buffer with GS_ERR_INVALID_ARG.  The pointers below are never
    dereferenced."""
    from paper_2403_11577_gb300 import render
    P = C.c_void_p
    INV = capi.GS_ERR_INVALID_ARG
    b = capi.GsBatch()
    b.frames_dev = 0x1000
    b.num_frames, b.num_cameras, b.num_trajs, b.num_gaussians = 2, 1, 1, 100
    b.tile, b.num_tiles = 16, 2 * 4 * 3
    b.num_records, b.num_pixels, b.pair_capacity = 200, 2 * 64 * 48, 10_000
    ws, bad_ws, ptr = P(0x100000), P(0x100008), P(0x200000)

    def opts(**kw):
        o = render.RenderOptions().c()
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    ok = opts()
    B, O = C.byref(b), C.byref(ok)
    # batch and workspace
    assert lib.gs_reset_status(None, ws, None) == INV
    assert lib.gs_reset_status(B, bad_ws, None) == INV
    assert lib.gs_read_stats(B, ws, None, None) == INV
    nb = capi.GsBatch.from_buffer_copy(b)
    nb.frames_dev = None
    assert lib.gs_bin_sort(C.byref(nb), O, ws, None) == INV
    # options
    for bad in (opts(tile=8), opts(batch=100), opts(exact_tiles=2), opts(alpha_max=1.0), opts(alpha_min=0.0),
                opts(near_z=0.0), opts(scale_max=0.0), opts(t_min=-1.0)):
        assert lib.gs_bin_sort(B, C.byref(bad), ws, None) == INV
        assert lib.gs_project(B, ptr, ptr, ptr, ptr, C.byref(bad), ws, None) == INV
    assert lib.gs_project(B, ptr, ptr, ptr, ptr, None, ws, None) == INV
    # required pointers
    assert lib.gs_pose_compose(B, None, ptr, ptr, ptr, ptr, ws, None) == INV
    assert lib.gs_pose_compose(B, ptr, ptr, ptr, ptr, ptr, bad_ws, None) == INV
    assert lib.gs_project(B, None, ptr, ptr, ptr, O, ws, None) == INV
    assert lib.gs_render_fwd(B, ptr, O, ws, ptr, ptr, None, None) == INV
    assert lib.gs_render_fwd(B, None, O, ws, ptr, ptr, ptr, None) == INV
    assert lib.gs_loss_l1(B, ptr, ptr, -1, 1.0, ptr, ptr, ws, None) == INV
    assert lib.gs_loss_l1(B, ptr, None, 10, 1.0, ptr, ptr, ws, None) == INV
    assert lib.gs_loss_photo(B, ptr, ptr, 1.5, 1.0, ptr, ptr, ws, None) == INV
    assert lib.gs_loss_photo(B, ptr, ptr, 0.2, 1.0, None, ptr, ws, None) == INV
    # X, quat, log_scale, logit_opacity, colors, opts, ws, out_T, out_last, dL_drgb, d_quat, d_log_scale,
    # d_logit_opacity, d_colors
    bwd = [ptr] * 5 + [O, ws, ptr, ptr, ptr] + [ptr] * 4
    for i in (0, 4, 7, 8, 9, 10, 13):
        args = list(bwd)
        args[i] = None
        assert lib.gs_render_bwd(B, *args, 0, None) == INV, i
    assert lib.gs_pose_grad(B, ptr, ws, ptr, None, None, 0, None) == INV
    assert lib.gs_pose_grad(B, None, ws, ptr, ptr, None, 0, None) == INV
    assert lib.gs_profile_events(99, None, None) == INV
    assert lib.gs_profile_events(capi.GS_PROF_RENDER_BWD, None, None) == INV
    # voxel downsampling
    scratch = P(0x300000)
    for n, v, s in ((-1, 0.1, scratch), (10, 0.0, scratch), (10, float("nan"), scratch), (10, float("inf"), scratch),
                    (10, 0.1, P(0x300010))):
        assert lib.gs_voxel_downsample(ptr, n, v, ptr, ptr, s, None) == INV, (n, v)
    assert lib.gs_voxel_downsample(ptr, 10, 0.1, ptr, None, scratch, None) == INV
    # allocation-free sort
    assert lib.gs_bin_sort_noalloc(B, O, ptr, ptr, None, ptr, ptr, ptr, None) == INV
    assert lib.gs_bin_sort_noalloc(B, C.byref(opts(exact_tiles=1)), ptr, ptr, ptr, ptr, ptr, ptr, None) == \
        capi.GS_ERR_UNSUPPORTED
    big = capi.GsBatch.from_buffer_copy(b)
    big.pair_capacity = 1 << 22
    assert lib.gs_bin_sort_noalloc(C.byref(big), C.byref(opts(exact_tiles=0)), ptr, ptr, ptr, ptr, ptr, ptr,
                                   None) == capi.GS_ERR_CAPACITY
    # rect, keys, ranges and out_pairs are read or written as 8-byte words,
    # depth and vals as 4-byte words: a pointer off that boundary is refused
    o0 = C.byref(opts(exact_tiles=0))
    args = [ptr] * 6  # rect, depth, keys, vals, ranges, out_pairs
    for i, off in ((0, 4), (1, 2), (2, 4), (3, 2), (4, 4), (5, 4)):
        a = list(args)
        a[i] = P(0x200000 + off)
        assert lib.gs_bin_sort_noalloc(B, o0, *a, None) == INV, i
