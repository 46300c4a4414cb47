// extern "C" entry points of libgs3dcalib.so: argument checks, batch
// planning, workspace layout and kernel dispatch.  Declarations and the
// contract of every call are in include/gs3dcalib.h.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gs {

cudaError_t launch_pose_compose(const gs_batch *, const double *, const double *, const int32_t *,
                                const double *, const double *, float *, double *, cudaStream_t);
cudaError_t launch_pose_grad(const gs_batch *, int, const double *, double *, double *, const double *,
                             const double *, double *, double *, double *, bool, cudaStream_t);
cudaError_t launch_project(const gs_batch *, const float *, const float *, const float *, const float *,
                           const float *, const gs_opts *, uint2 *, float *, float4 *, float4 *, Stats *,
                           cudaStream_t);
int project_bwd_parts(const gs_batch *);
cudaError_t launch_project_bwd(const gs_batch *, const float *, const float *, const float *, const float *,
                               const float *, const gs_opts *, const uint2 *, const float4 *, float *, float *,
                               float *, float *, double *, bool, cudaStream_t);
cudaError_t launch_bin_sort(const gs_batch *, const gs_opts *, const Layout &, unsigned char *, cudaStream_t, int);
cudaError_t launch_render_fwd(const gs_batch *, const gs_opts *, const uint32_t *, const uint2 *, const uint32_t *,
                              const float4 *, const float *, Stats *, float *, float *, int32_t *, uint32_t *,
                              long long, cudaStream_t);
cudaError_t launch_render_bwd(const gs_batch *, const gs_opts *, const uint32_t *, const uint2 *, const uint32_t *,
                              const float4 *, const float *, Stats *, const float *, const int32_t *, const float *,
                              float4 *, const uint32_t *, long long, cudaStream_t);
cudaError_t launch_l1(const float *, const float *, long long, float, double *, float *, double *, cudaStream_t);
cudaError_t launch_photo(const gs_batch *, const float *, const float *, float, float, double *, float *, float *,
                         double *, cudaStream_t);
size_t voxel_scratch_bytes(long long n, int *sort_blocks);
long long ngp_param_count(const gs_ngp *c);
cudaError_t launch_ngp_fwd(const gs_ngp *c, const float *theta, const float *X, long long n, float *rgb,
                           float *logit_o, float *log_s, float *quat, cudaStream_t s);
cudaError_t ngp_fault(unsigned int *out);
cudaError_t ngp_set_wait_limit(unsigned long long ns);
cudaError_t launch_ngp_bwd(const gs_ngp *c, const float *theta, const float *X, long long n, const float *d_rgb,
                           const float *d_logit_o, const float *d_log_s, const float *d_quat, float *d_theta,
                           cudaStream_t s);
cudaError_t launch_voxel(const float *X, long long n, float v, int32_t *out_index, unsigned long long *out_count,
                         unsigned char *scratch, cudaStream_t s);

constexpr int kSortBlocksMax = 304;  // two per SM on a 152-SM GB300

bool make_layout(const gs_batch *b, Layout *L) {
    if (!b || b->num_frames <= 0 || b->num_records < 0 || b->num_tiles <= 0 || b->pair_capacity < 0) return false;
    const size_t F = (size_t)b->num_frames, R = (size_t)b->num_records, T = (size_t)b->num_tiles;
    const size_t cap = (size_t)b->pair_capacity;
    L->emit_blocks = (int)((R + kEmitItems - 1) / kEmitItems);
    long long st = ((long long)cap + kSortTile - 1) / kSortTile;
    L->sort_blocks = (int)std::max(1ll, std::min(st, (long long)kSortBlocksMax));
    long long rt = ((long long)R + kSortTile - 1) / kSortTile;
    L->rec_sort_blocks = (int)std::max(1ll, std::min(rt, (long long)kSortBlocksMax));
    L->twist_parts = std::max(1, project_bwd_parts(b));
    L->passes = radix_passes(b->num_tiles);
    L->first_buffer = L->passes & 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L->stats = take(sizeof(Stats));
    L->pose32 = take(F * kPose32Stride * sizeof(float));
    L->pose64 = take(F * kPose64Stride * sizeof(double));
    L->rect = take(R * 8);
    L->depth = take(R * 4);
    L->splat = take(R * 32);
    L->grad2d = take(R * 48);
    L->keys[0] = take(cap * 4);
    L->vals[0] = take(cap * 4);
    L->keys[1] = take(cap * 4);
    L->vals[1] = take(cap * 4);
    L->rec_keys[0] = take(R * 4);
    L->rec_vals[0] = take(R * 4);
    L->rec_keys[1] = take(R * 4);
    L->rec_vals[1] = take(R * 4);
    L->ranges = take(T * 8);
    L->order = take(T * 4);
    L->emit_sums = take((size_t)std::max(1, L->emit_blocks) * 8);
    L->rec_pairs = take(R * 8);  // exact tiles: pairs and non-empty rows per sorted record
    // render: per forward band slot, one bit per tile-list entry (each tile's
    // bits start on a word: word (range start / 32) + tile)
    L->band_words = (long long)(cap / 32 + T + 2);
    L->band_masks = take((size_t)render_band_slots(b->tile) * (size_t)L->band_words * 4);
    L->sort_hist = take((size_t)kRadix * (std::max(L->sort_blocks, L->rec_sort_blocks) + 1) * 4);  // counts + totals
    L->twist_part = take(F * (size_t)L->twist_parts * 6 * 8);
    L->twist_mid = take(F * 32 * 6 * 8);  // 32 slices per frame of the twist reduction
    L->twist_frame = take(F * 6 * 8);
    L->loss_part = take((size_t)kLossBlocks * 8);
    L->photo_maps = take((size_t)b->num_pixels * 9 * 4);  // 3 SSIM maps per channel
    L->photo_part = take(T * 2 * 8);
    L->total = o;
    return true;
}

}  // namespace gs

using namespace gs;

namespace {

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline unsigned char *W(void *ws) { return reinterpret_cast<unsigned char *>(ws); }

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool opts_ok(const gs_batch *b, const gs_opts *o) {
    if (!o) return false;
    if (o->tile != b->tile) return false;
    if (!(o->tile == 8 || o->tile == 16 || o->tile == 32)) return false;
    if (!(o->batch == 64 || o->batch == 128 || o->batch == 256)) return false;
    if (!(o->alpha_min > 0.f) || !(o->alpha_max > o->alpha_min) || !(o->alpha_max < 1.f)) return false;
    if (!(o->t_min >= 0.f) || !(o->near_z > 0.f) || !(o->lowpass >= 0.f) || !(o->scale_max > 0.f)) return false;
    if (o->exact_tiles != 0 && o->exact_tiles != 1) return false;
    return true;
}

bool batch_ok(const gs_batch *b, const void *ws) {
    return b && b->frames_dev && ws && aligned(ws, 256) && b->num_frames > 0 && b->num_tiles > 0;
}

gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

int g_prof_kernel = GS_PROF_NONE;
cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

// Records the timing hook's start (or stop) event before (after) `kernel`.
// Captured launches get an external event-record node; eager ones a plain record.
cudaError_t prof_mark(int kernel, bool start, cudaStream_t s) {
    if (g_prof_kernel != kernel || kernel == GS_PROF_NONE) return cudaSuccess;
    cudaEvent_t ev = start ? g_prof_start : g_prof_stop;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    return cudaEventRecord(ev, s);
}

}  // namespace

extern "C" {

const char *gs_version(void) { return "gs3dcalib 0.1.0 (sm_103a)"; }

gs_status gs_profile_events(int32_t kernel, void *start_event, void *stop_event) {
    if (kernel < GS_PROF_NONE || kernel > GS_PROF_LOSS) return GS_ERR_INVALID_ARG;
    if (kernel != GS_PROF_NONE && (!start_event || !stop_event)) return GS_ERR_INVALID_ARG;
    g_prof_kernel = kernel;
    g_prof_start = reinterpret_cast<cudaEvent_t>(start_event);
    g_prof_stop = reinterpret_cast<cudaEvent_t>(stop_event);
    return GS_OK;
}

int32_t gs_struct_sizes(size_t *out, int32_t n) {
    const size_t v[4] = {sizeof(gs_frame), sizeof(gs_opts), sizeof(gs_batch), sizeof(gs_stats)};
    int32_t k = n < 4 ? n : 4;
    for (int32_t i = 0; out && i < k; i++) out[i] = v[i];
    return out ? k : 0;
}

gs_status gs_batch_init(gs_frame *frames, int32_t F, int32_t num_gaussians, int32_t num_cameras,
                        int32_t num_trajs, int32_t tile, int64_t pair_capacity, gs_frame *frames_dev,
                        gs_batch *out) {
    if (!frames || !frames_dev || !out || F <= 0 || F > kMaxFrames || num_gaussians < 0 || num_cameras <= 0 ||
        num_trajs <= 0 || pair_capacity < 0 || pair_capacity >= (1ll << 32))
        return GS_ERR_INVALID_ARG;
    if (!(tile == 8 || tile == 16 || tile == 32)) return GS_ERR_INVALID_ARG;
    int64_t rec = 0, pix = 0, tiles = 0;
    for (int f = 0; f < F; f++) {
        gs_frame &fr = frames[f];
        if (fr.width <= 0 || fr.height <= 0 || fr.camera_id < 0 || fr.camera_id >= num_cameras ||
            fr.traj_id < 0 || fr.traj_id >= num_trajs || fr.gauss_offset < 0 || fr.gauss_count < 0 ||
            (int64_t)fr.gauss_offset + fr.gauss_count > num_gaussians || !std::isfinite(fr.fx) ||
            !std::isfinite(fr.fy) || !std::isfinite(fr.cx) || !std::isfinite(fr.cy) ||
            !std::isfinite(fr.timestamp) || fr.row0 < 0 || fr.row0 >= fr.height)
            return GS_ERR_INVALID_ARG;
        fr.tiles_x = (fr.width + tile - 1) / tile;
        fr.tiles_y = (fr.height - fr.row0 + tile - 1) / tile;
        if (fr.tiles_x >= 65536 || fr.tiles_y >= 65536) return GS_ERR_INVALID_ARG;
        fr.record_offset = rec;
        fr.pixel_offset = pix;
        fr.tile_offset = (int32_t)tiles;
        rec += fr.gauss_count;
        pix += (int64_t)fr.width * (fr.height - fr.row0);
        tiles += (int64_t)fr.tiles_x * fr.tiles_y;
        if (tiles >= (1ll << 31) || rec >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    }
    if (cudaMemcpy(frames_dev, frames, sizeof(gs_frame) * F, cudaMemcpyHostToDevice) != cudaSuccess)
        return GS_ERR_CUDA;
    out->frames_dev = frames_dev;
    out->num_frames = F;
    out->num_cameras = num_cameras;
    out->num_trajs = num_trajs;
    out->num_gaussians = num_gaussians;
    out->tile = tile;
    out->num_tiles = (int32_t)tiles;
    out->num_records = rec;
    out->num_pixels = pix;
    out->pair_capacity = pair_capacity;
    return GS_OK;
}

size_t gs_workspace_size(const gs_batch *b) {
    Layout L;
    return make_layout(b, &L) ? L.total : 0;
}

int32_t gs_workspace_offsets(const gs_batch *b, size_t *off, int32_t max_entries) {
    Layout L;
    if (!off || !make_layout(b, &L)) return 0;
    const size_t v[10] = {L.stats, L.pose32, L.pose64, L.rect, L.depth, L.splat, L.grad2d, L.keys[0], L.vals[0],
                          L.ranges};
    int n = max_entries < 10 ? max_entries : 10;
    for (int i = 0; i < n; i++) off[i] = v[i];
    return n;
}

gs_status gs_read_stats(const gs_batch *b, const void *ws, void *stream, gs_stats *out) {
    Layout L;
    if (!out || !batch_ok(b, ws) || !make_layout(b, &L)) return GS_ERR_INVALID_ARG;
    Stats st;
    cudaError_t e = cudaMemcpyAsync(&st, (const unsigned char *)ws + L.stats, sizeof st, cudaMemcpyDeviceToHost,
                                    S(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return GS_ERR_CUDA;
    out->status = st.status;
    out->reserved = 0;
    out->num_pairs = st.num_pairs;
    out->eval_fwd = st.eval_fwd;
    out->eval_bwd = st.eval_bwd;
    return GS_OK;
}

gs_status gs_reset_status(const gs_batch *b, void *ws, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !make_layout(b, &L)) return GS_ERR_INVALID_ARG;
    return cuda_status(cudaMemsetAsync(W(ws) + L.stats, 0, sizeof(Stats), S(stream)));
}

gs_status gs_pose_compose(const gs_batch *b, const double *traj_t, const double *traj_pose,
                          const int32_t *traj_offset, const double *ext, const double *delta, void *ws,
                          void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !traj_t || !traj_pose || !traj_offset || !ext || !delta || !make_layout(b, &L))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_pose_compose(b, traj_t, traj_pose, traj_offset, ext, delta,
                                           (float *)(W(ws) + L.pose32), (double *)(W(ws) + L.pose64), S(stream)));
}

gs_status gs_project(const gs_batch *b, const float *X, const float *quat, const float *log_scale,
                     const float *logit_opacity, const gs_opts *o, void *ws, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !opts_ok(b, o) || !make_layout(b, &L)) return GS_ERR_INVALID_ARG;
    if (b->num_gaussians > 0 && (!X || !quat || !log_scale || !logit_opacity)) return GS_ERR_INVALID_ARG;
    unsigned char *w = W(ws);
    cudaError_t e = prof_mark(GS_PROF_PROJECT, true, S(stream));
    if (e == cudaSuccess)
        e = launch_project(b, (const float *)(w + L.pose32), X, quat, log_scale, logit_opacity, o,
                           (uint2 *)(w + L.rect), (float *)(w + L.depth), (float4 *)(w + L.splat),
                           (float4 *)(w + L.grad2d), (Stats *)(w + L.stats), S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_PROJECT, false, S(stream));
    return cuda_status(e);
}

gs_status gs_bin_sort(const gs_batch *b, const gs_opts *o, void *ws, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !opts_ok(b, o) || !make_layout(b, &L)) return GS_ERR_INVALID_ARG;
    cudaError_t e = prof_mark(GS_PROF_BIN_SORT, true, S(stream));
    if (e == cudaSuccess) e = launch_bin_sort(b, o, L, W(ws), S(stream), 0);
    if (e == cudaSuccess) e = prof_mark(GS_PROF_BIN_SORT, false, S(stream));
    return cuda_status(e);
}

gs_status gs_render_fwd(const gs_batch *b, const float *colors, const gs_opts *o, void *ws, float *out_rgb,
                        float *out_T, int32_t *out_last, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !opts_ok(b, o) || !make_layout(b, &L) || !out_rgb || !out_T || !out_last)
        return GS_ERR_INVALID_ARG;
    if (b->num_gaussians > 0 && !colors) return GS_ERR_INVALID_ARG;
    unsigned char *w = W(ws);
    cudaError_t e = cudaMemsetAsync(&((Stats *)(w + L.stats))->eval_fwd, 0, 8, S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_RENDER_FWD, true, S(stream));
    if (e == cudaSuccess)
        e = launch_render_fwd(b, o, (const uint32_t *)(w + L.order), (const uint2 *)(w + L.ranges),
                              (const uint32_t *)(w + L.vals[0]),
                              (const float4 *)(w + L.splat), colors, (Stats *)(w + L.stats), out_rgb, out_T,
                              out_last, (uint32_t *)(w + L.band_masks), L.band_words, S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_RENDER_FWD, false, S(stream));
    return cuda_status(e);
}

gs_status gs_loss_l1(const gs_batch *b, const float *rgb, const float *target, int64_t n, float scale,
                     double *out_loss, float *out_grad, void *ws, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !make_layout(b, &L) || !rgb || !target || !out_loss || n < 0) return GS_ERR_INVALID_ARG;
    cudaError_t e = prof_mark(GS_PROF_LOSS, true, S(stream));
    if (e == cudaSuccess)
        e = launch_l1(rgb, target, n, scale, out_loss, out_grad, (double *)(W(ws) + L.loss_part), S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_LOSS, false, S(stream));
    return cuda_status(e);
}

gs_status gs_loss_photo(const gs_batch *b, const float *rgb, const float *target, float lambda1, float scale,
                        double *out_loss, float *out_grad, void *ws, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !make_layout(b, &L) || !out_loss || !(lambda1 >= 0.f && lambda1 <= 1.f) ||
        !std::isfinite(scale))
        return GS_ERR_INVALID_ARG;
    if (b->num_pixels > 0 && (!rgb || !target)) return GS_ERR_INVALID_ARG;
    unsigned char *w = W(ws);
    cudaError_t e = prof_mark(GS_PROF_LOSS, true, S(stream));
    if (e == cudaSuccess)
        e = launch_photo(b, rgb, target, lambda1, scale, out_loss, out_grad, (float *)(w + L.photo_maps),
                         (double *)(w + L.photo_part), S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_LOSS, false, S(stream));
    return cuda_status(e);
}

int64_t gs_ngp_param_count(const gs_ngp *cfg) { return ngp_param_count(cfg); }

gs_status gs_ngp_set_wait_limit(uint64_t ns) { return cuda_status(ngp_set_wait_limit(ns)); }

gs_status gs_ngp_fault(uint32_t *out) {
    if (!out) return GS_ERR_INVALID_ARG;
    unsigned int v = 0;
    const cudaError_t e = ngp_fault(&v);
    *out = v;
    return cuda_status(e);
}

gs_status gs_ngp_forward(const gs_ngp *cfg, const float *theta, const float *X, int64_t n, float *rgb,
                         float *logit_opacity, float *log_scale, float *quat, void *stream) {
    if (ngp_param_count(cfg) < 0 || n < 0 || !theta || (reinterpret_cast<uintptr_t>(theta) & 7) ||
        (n > 0 && (!X || !rgb || !logit_opacity || !log_scale || !quat)))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_ngp_fwd(cfg, theta, X, n, rgb, logit_opacity, log_scale, quat, S(stream)));
}

gs_status gs_ngp_backward(const gs_ngp *cfg, const float *theta, const float *X, int64_t n, const float *d_rgb,
                          const float *d_logit_opacity, const float *d_log_scale, const float *d_quat,
                          float *d_theta, void *stream) {
    if (ngp_param_count(cfg) < 0 || n < 0 || !theta || !d_theta || (reinterpret_cast<uintptr_t>(theta) & 7) ||
        (reinterpret_cast<uintptr_t>(d_theta) & 15) ||
        (n > 0 && (!X || !d_rgb || !d_logit_opacity || !d_log_scale || !d_quat)))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_ngp_bwd(cfg, theta, X, n, d_rgb, d_logit_opacity, d_log_scale, d_quat, d_theta,
                                      S(stream)));
}

size_t gs_voxel_scratch_size(int64_t n) {
    if (n < 0 || n >= (1ll << 31)) return 0;
    return voxel_scratch_bytes(n, nullptr);
}

gs_status gs_voxel_downsample(const float *X, int64_t n, float voxel, int32_t *out_index, uint64_t *out_count,
                              void *scratch, void *stream) {
    if (n < 0 || n >= (1ll << 31) || !(std::isfinite(voxel) && voxel > 0.f) || !out_count || !scratch ||
        (n > 0 && (!X || !out_index)) || (reinterpret_cast<uintptr_t>(scratch) & 255))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_voxel(X, n, voxel, out_index, reinterpret_cast<unsigned long long *>(out_count),
                                    static_cast<unsigned char *>(scratch), S(stream)));
}

gs_status gs_render_bwd(const gs_batch *b, const float *X, const float *quat, const float *log_scale,
                        const float *logit_opacity, const float *colors, const gs_opts *o, void *ws,
                        const float *out_T, const int32_t *out_last, const float *dL_drgb, float *d_quat,
                        float *d_log_scale, float *d_logit_opacity, float *d_colors, int32_t accumulate,
                        void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !opts_ok(b, o) || !make_layout(b, &L) || !out_T || !out_last || !dL_drgb)
        return GS_ERR_INVALID_ARG;
    if (b->num_gaussians > 0 && (!X || !quat || !log_scale || !logit_opacity || !colors || !d_quat ||
                                 !d_log_scale || !d_logit_opacity || !d_colors))
        return GS_ERR_INVALID_ARG;
    unsigned char *w = W(ws);
    Stats *st = (Stats *)(w + L.stats);
    cudaError_t e = cudaMemsetAsync(&st->eval_bwd, 0, 8, S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_RENDER_BWD, true, S(stream));
    if (e == cudaSuccess)
        e = launch_render_bwd(b, o, (const uint32_t *)(w + L.order), (const uint2 *)(w + L.ranges),
                              (const uint32_t *)(w + L.vals[0]),
                              (const float4 *)(w + L.splat), colors, st, out_T, out_last, dL_drgb,
                              (float4 *)(w + L.grad2d), (const uint32_t *)(w + L.band_masks), L.band_words,
                              S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_RENDER_BWD, false, S(stream));
    if (e != cudaSuccess) return GS_ERR_CUDA;
    if (b->num_gaussians == 0)
        return cuda_status(cudaMemsetAsync(w + L.twist_part, 0, (size_t)b->num_frames * L.twist_parts * 6 * 8,
                                           S(stream)));
    e = prof_mark(GS_PROF_PROJECT_BWD, true, S(stream));
    if (e == cudaSuccess)
        e = launch_project_bwd(b, (const float *)(w + L.pose32), X, quat, log_scale, logit_opacity, o,
                               (const uint2 *)(w + L.rect), (const float4 *)(w + L.grad2d), d_quat, d_log_scale,
                               d_logit_opacity, d_colors, (double *)(w + L.twist_part), accumulate != 0, S(stream));
    if (e == cudaSuccess) e = prof_mark(GS_PROF_PROJECT_BWD, false, S(stream));
    return cuda_status(e);
}

gs_status gs_pose_grad(const gs_batch *b, const double *ext, void *ws, double *d_ext, double *d_delta,
                       double *d_xi, int32_t accumulate, void *stream) {
    Layout L;
    if (!batch_ok(b, ws) || !make_layout(b, &L) || !ext || !d_ext || !d_delta) return GS_ERR_INVALID_ARG;
    unsigned char *w = W(ws);
    return cuda_status(launch_pose_grad(b, L.twist_parts, (const double *)(w + L.twist_part),
                                        (double *)(w + L.twist_mid), (double *)(w + L.twist_frame),
                                        (const double *)(w + L.pose64), ext, d_ext,
                                        d_delta, d_xi, accumulate != 0, S(stream)));
}

}  // extern "C"
