// Phi (Eq. 5): front-to-back alpha compositing of the depth-sorted splats of
// each tile, and its backward (Sec. III-B).
//
// One block per (frame, tile) work item of the whole batch, taken in the
// heavy-first order gs_bin_sort computes (longest lists start first).  Each
// warp owns a compact full-width band of the tile and walks the tile's
// depth-sorted list on its own (no block-wide barrier inside the loop): it
// loads chunks of batch/2 entries (prefetching the next chunk into registers
// while it uses the current one), keeps the entries whose alpha >= alpha_min
// box meets its band -- outside the box alpha is below alpha_min at every
// pixel, so the cull is exact and identical in both directions -- compacts
// them in order into its own shared-memory slot and composites them for its
// PPT pixels per thread.  A warp stops as soon as all its pixels have
// stopped.
//
// Per pixel and Gaussian (both directions use the same arithmetic):
//   dx = u - mean_x, dy = v - mean_y
//   e2 = A dx^2 + B dx dy + C dy^2     (= power * log2 e)
//   skip if e2 > 0;  e = e2 + F (F = log2 opacity); skip if e < log2 alpha_min
//   alpha = min(alpha_max, 2^e)
//
// Backward: walks the pixel's range from its last composited Gaussian back
// to the first, recovering T_i = T_{i+1} / (1 - alpha_i) from the final
// transmittance instead of storing it, with accum = colour composited behind:
//   dL/dc_i     = alpha_i T_i g
//   dL/dalpha_i = T_i (c_i - accum) . g - T_final (bg . g) / (1 - alpha_i)
//   dL/de       = dL/dalpha_i * alpha_i * ln 2   (0 where alpha is clamped)
// giving dL/dF = dL/de, dL/dA = dL/de dx^2, dL/dB = dL/de dx dy,
// dL/dC = dL/de dy^2, dL/dmean = -dL/de (2A dx + B dy, B dx + 2C dy).
// The nine per-pixel values are summed over the thread's pixels, then over
// the warp (skipped when no lane contributes): eight of them by a transposed
// halving exchange that leaves one total per group of four lanes, which the
// group's first lane adds to the record (eight lanes, contiguous addresses),
// the ninth by a plain shuffle reduction.
#include "common.cuh"

namespace gs {

namespace {

// Threads per block: 64 for 8x8 tiles (a pixel each), 128 for 16x16 (two
// vertically adjacent pixels each), 256 for 32x32 (four each).
template <int TILE>
struct Cfg {
    static constexpr int NPIX = TILE * TILE;
    static constexpr int PPT = TILE == 8 ? 1 : (TILE == 16 ? 2 : 4);  // pixels per thread
    static constexpr int NT = NPIX / PPT;
    static constexpr int RPW = 32 * PPT / TILE;    // pixel rows per warp (full tile width)
};

struct RenderParams {
    float lmin;       // log2(alpha_min)
    float amax, tmin;
    float bg0, bg1, bg2;
};

// Exponent e2 = A dx^2 + B dx dy + C dy^2 with a fixed operation order
// (no contraction freedom), shared by the forward and the backward.
__device__ __forceinline__ float exponent2(float dx, float dy, float A, float B, float C) {
    const float bdy = __fmul_rn(B, dy);
    const float t = __fmaf_rn(A, dx, bdy);
    const float cdy = __fmul_rn(C, dy);
    const float q = __fmul_rn(cdy, dy);
    return __fmaf_rn(dx, t, q);
}

// Pixel (lx, ly) of the tile handled by thread `tid` as its k-th pixel.  A
// warp covers RPW consecutive full-width rows, so its pixels form a compact
// TILE x RPW region (used to cull Gaussians per warp).
template <int TILE>
__device__ __forceinline__ void pixel_of(int tid, int k, int &lx, int &ly) {
    lx = tid % TILE;
    ly = (tid / TILE) * Cfg<TILE>::PPT + k;
}

// Whether the Gaussian's alpha >= alpha_min box (centre m, half-widths e)
// meets the warp's pixel region.  Outside that box alpha < alpha_min at
// every pixel, so skipping is exact; forward and backward use this same test.
__device__ __forceinline__ bool box_hits(float4 a, float2 e, float xlo, float xhi, float ylo, float yhi) {
    return (a.x + e.x >= xlo) && (a.x - e.x <= xhi) && (a.y + e.y >= ylo) && (a.y - e.y <= yhi);
}

// One staged Gaussian of a warp's chunk, as loaded from global memory.
struct Entry {
    float4 a;       // mean_x, mean_y, A, B
    float4 b;       // C, F, rx, ry
    float cr, cg, cb;
    uint32_t g;     // Gaussian index within the scene
    bool valid;
};

__device__ __forceinline__ void load_entry(Entry &e, bool valid, const uint32_t *__restrict__ vals, uint32_t at,
                                           long long rec0, const float4 *__restrict__ splat,
                                           const float *__restrict__ col) {
    e.valid = valid;
    if (!valid) return;
    e.g = vals[at];
    const long long r = rec0 + e.g;
    e.a = splat[2 * r];
    e.b = splat[2 * r + 1];
    e.cr = __ldg(col + 3 * e.g);
    e.cg = __ldg(col + 3 * e.g + 1);
    e.cb = __ldg(col + 3 * e.g + 2);
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(Cfg<TILE>::NT)
k_render_fwd(const gs_frame *__restrict__ frames, int F, const uint32_t *__restrict__ order,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
             const float4 *__restrict__ splat, const float *__restrict__ colors, RenderParams rp,
             Stats *__restrict__ stats, float *__restrict__ out_rgb, float *__restrict__ out_T,
             int32_t *__restrict__ out_last) {
    constexpr int NT = Cfg<TILE>::NT, PPT = Cfg<TILE>::PPT, RPW = Cfg<TILE>::RPW;
    constexpr int NW = NT / 32, CH = BATCH / 2, PER = CH / 32;
    __shared__ float4 s0[NW][CH];  // mean_x, mean_y, A, B
    __shared__ float4 s1[NW][CH];  // C, F, r, g
    __shared__ float s2[NW][CH];   // b
    __shared__ int spos[NW][CH];   // position in the tile's sorted range
    __shared__ unsigned long long s_eval;
    const int t = (int)order[blockIdx.x];  // heavy tiles first
    const int f = frame_of_tile(frames, F, t);
    const gs_frame &fr = frames[f];
    const int W = fr.width, H = fr.height;
    const int lt = t - fr.tile_offset;
    const int tx = lt % fr.tiles_x, ty = lt / fr.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float xlo = (float)(tx * TILE), xhi = xlo + (float)(TILE - 1);
    const float ylo = (float)(ty * TILE + warp * RPW), yhi = ylo + (float)(RPW - 1);
    float px[PPT], py[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT];
    int last[PPT];
    bool done[PPT], inside[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        int lx, ly;
        pixel_of<TILE>(threadIdx.x, k, lx, ly);
        const int u = tx * TILE + lx, v = ty * TILE + ly;
        px[k] = (float)u;
        py[k] = (float)v;
        inside[k] = u < W && v < H;
        done[k] = !inside[k];
        T[k] = 1.f;
        c0[k] = c1[k] = c2[k] = 0.f;
        last[k] = 0;
    }
    if (threadIdx.x == 0) s_eval = 0;
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    const long long rec0 = fr.record_offset;
    const float *col = colors + 3 * (size_t)fr.gauss_offset;
    unsigned evals = 0;
    // each warp walks the tile's list on its own: it loads a chunk of CH
    // entries (the next one is prefetched while the current one is used),
    // keeps those whose alpha box meets its band, compacts them in order into
    // its shared-memory slot and composites them
    Entry nx[PER];
#pragma unroll
    for (int p = 0; p < PER; p++) load_entry(nx[p], p * 32 + lane < n, vals, range.x + p * 32 + lane, rec0, splat, col);
    for (int cb0 = 0; cb0 < n; cb0 += CH) {
        bool mine_done = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) mine_done &= done[k];
        if (__all_sync(0xffffffffu, mine_done)) break;
        Entry cu[PER];
#pragma unroll
        for (int p = 0; p < PER; p++) cu[p] = nx[p];
        if (cb0 + CH < n) {
#pragma unroll
            for (int p = 0; p < PER; p++) {
                const int i = cb0 + CH + p * 32 + lane;
                load_entry(nx[p], i < n, vals, range.x + i, rec0, splat, col);
            }
        }
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const bool hit = cu[p].valid && box_hits(cu[p].a, make_float2(cu[p].b.z, cu[p].b.w), xlo, xhi, ylo, yhi);
            const uint32_t msk = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int at = cnt + __popc(msk & lt_mask);
                s0[warp][at] = cu[p].a;
                s1[warp][at] = make_float4(cu[p].b.x, cu[p].b.y, cu[p].cr, cu[p].cg);
                s2[warp][at] = cu[p].cb;
                spos[warp][at] = cb0 + p * 32 + lane;
            }
            cnt += __popc(msk);
        }
        __syncwarp();
        for (int j = 0; j < cnt; j++) {
            const float4 a = s0[warp][j], b = s1[warp][j];
            const float cb = s2[warp][j];
            const int pos = spos[warp][j];
            // every lane evaluates the exponent; one warp vote decides
            // whether any pixel composites this Gaussian, and the
            // compositing itself runs predicated (no divergence)
            float e[PPT];
            bool ct[PPT];
            bool anyc = false;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                evals += !done[k];
                const float dx = px[k] - a.x, dy = py[k] - a.y;
                const float e2 = exponent2(dx, dy, a.z, a.w, b.x);
                e[k] = e2 + b.y;
                ct[k] = !done[k] && !(e2 > 0.f) && !(e[k] < rp.lmin);
                anyc |= ct[k];
            }
            if (!__any_sync(0xffffffffu, anyc)) continue;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const float alpha = fminf(rp.amax, ex2_approx(e[k]));
                const float nT = T[k] * (1.f - alpha);
                const bool stop = ct[k] && nT < rp.tmin;
                const bool blend = ct[k] && !stop;
                done[k] = done[k] || stop;
                const float w = blend ? alpha * T[k] : 0.f;
                c0[k] = fmaf(b.z, w, c0[k]);
                c1[k] = fmaf(b.w, w, c1[k]);
                c2[k] = fmaf(cb, w, c2[k]);
                T[k] = blend ? nT : T[k];
                last[k] = blend ? pos + 1 : last[k];
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!inside[k]) continue;
        int lx, ly;
        pixel_of<TILE>(threadIdx.x, k, lx, ly);
        const long long pix = fr.pixel_offset + (long long)(ty * TILE + ly) * W + (tx * TILE + lx);
        out_rgb[3 * pix] = c0[k] + T[k] * rp.bg0;
        out_rgb[3 * pix + 1] = c1[k] + T[k] * rp.bg1;
        out_rgb[3 * pix + 2] = c2[k] + T[k] * rp.bg2;
        out_T[pix] = T[k];
        out_last[pix] = last[k];
    }
    // evaluation counter (for the roofline): warp sums, one atomic per warp
    unsigned long long ev = evals;
    for (int s = 16; s > 0; s >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, s);
    __syncthreads();
    if (lane == 0) atomicAdd(&s_eval, ev);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&stats->eval_fwd, s_eval);
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Sum eight per-lane values over the warp by halving exchanges: at each step
// a lane keeps half of its values and sends the other half to its partner,
// so the exchanges shrink 4, 2, 1, 1, 1 (8 shuffles instead of 40).  On
// return every lane holds the warp total of component
// c = 4*bit4(lane) + 2*bit3(lane) + bit2(lane).
__device__ __forceinline__ float warp_sum8_transposed(const float (&v)[8], int lane) {
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float send = u16 ? v[i] : v[i + 4];
        const float keep = u16 ? v[i + 4] : v[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = u8 ? w[i] : w[i + 2];
        const float keep = u8 ? w[i + 2] : w[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const float send = u4 ? x[0] : x[1];
    float y = (u4 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    return y;
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(Cfg<TILE>::NT)
k_render_bwd(const gs_frame *__restrict__ frames, int F, const uint32_t *__restrict__ order,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
             const float4 *__restrict__ splat, const float *__restrict__ colors, RenderParams rp,
             Stats *__restrict__ stats, const float *__restrict__ in_T, const int32_t *__restrict__ in_last,
             const float *__restrict__ dL_drgb, float4 *__restrict__ grad2d) {
    constexpr int NT = Cfg<TILE>::NT, PPT = Cfg<TILE>::PPT, RPW = Cfg<TILE>::RPW;
    constexpr int NW = NT / 32, CH = BATCH / 2, PER = CH / 32;
    __shared__ float4 s0[NW][CH];
    __shared__ float4 s1[NW][CH];
    __shared__ float s2[NW][CH];
    __shared__ int spos[NW][CH];
    __shared__ uint32_t sg[NW][CH];
    __shared__ unsigned long long s_eval;
    const int t = (int)order[blockIdx.x];  // heavy tiles first
    const int f = frame_of_tile(frames, F, t);
    const gs_frame &fr = frames[f];
    const int W = fr.width, H = fr.height;
    const int lt = t - fr.tile_offset;
    const int tx = lt % fr.tiles_x, ty = lt / fr.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float xlo = (float)(tx * TILE), xhi = xlo + (float)(TILE - 1);
    const float ylo = (float)(ty * TILE + warp * RPW), yhi = ylo + (float)(RPW - 1);
    float px[PPT], py[PPT], T[PPT], Tf[PPT], g0[PPT], g1[PPT], g2[PPT], bgd[PPT];
    float a0[PPT], a1[PPT], a2[PPT];
    int last[PPT];
    if (threadIdx.x == 0) s_eval = 0;
    // the range of this tile; a pixel's start position never exceeds it
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        int lx, ly;
        pixel_of<TILE>(threadIdx.x, k, lx, ly);
        const int u = tx * TILE + lx, v = ty * TILE + ly;
        px[k] = (float)u;
        py[k] = (float)v;
        a0[k] = a1[k] = a2[k] = 0.f;
        if (u < W && v < H) {
            const long long pix = fr.pixel_offset + (long long)v * W + u;
            Tf[k] = in_T[pix];
            last[k] = min(max(in_last[pix], 0), n);
            g0[k] = dL_drgb[3 * pix];
            g1[k] = dL_drgb[3 * pix + 1];
            g2[k] = dL_drgb[3 * pix + 2];
        } else {
            Tf[k] = 1.f;
            last[k] = 0;
            g0[k] = g1[k] = g2[k] = 0.f;
        }
        T[k] = Tf[k];
        bgd[k] = rp.bg0 * g0[k] + rp.bg1 * g1[k] + rp.bg2 * g2[k];
        mylast = max(mylast, last[k]);
    }
    // each warp walks its own part of the list backwards, from the largest
    // start position of its pixels, in chunks of CH (the next one prefetched)
    const int warp_last = __reduce_max_sync(0xffffffffu, mylast);
    const long long rec0 = fr.record_offset;
    const float *col = colors + 3 * (size_t)fr.gauss_offset;
    unsigned evals = 0;
    Entry nx[PER];
    {
        const int c0 = max(0, warp_last - CH);
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const int i = c0 + p * 32 + lane;
            load_entry(nx[p], i < warp_last, vals, range.x + i, rec0, splat, col);
        }
    }
    for (int c_end = warp_last; c_end > 0; c_end -= CH) {
        const int c0 = max(0, c_end - CH);
        Entry cu[PER];
#pragma unroll
        for (int p = 0; p < PER; p++) cu[p] = nx[p];
        if (c0 > 0) {
            const int n0 = max(0, c0 - CH);
#pragma unroll
            for (int p = 0; p < PER; p++) {
                const int i = n0 + p * 32 + lane;
                load_entry(nx[p], i < c0, vals, range.x + i, rec0, splat, col);
            }
        }
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const bool hit = cu[p].valid && box_hits(cu[p].a, make_float2(cu[p].b.z, cu[p].b.w), xlo, xhi, ylo, yhi);
            const uint32_t msk = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int at = cnt + __popc(msk & lt_mask);
                s0[warp][at] = cu[p].a;
                s1[warp][at] = make_float4(cu[p].b.x, cu[p].b.y, cu[p].cr, cu[p].cg);
                s2[warp][at] = cu[p].cb;
                spos[warp][at] = c0 + p * 32 + lane;
                sg[warp][at] = cu[p].g;
            }
            cnt += __popc(msk);
        }
        __syncwarp();
        for (int j = cnt - 1; j >= 0; j--) {
            const float4 a = s0[warp][j], b = s1[warp][j];
            const float cb = s2[warp][j];
            const int pos = spos[warp][j];
            // every lane evaluates the exponent; one warp vote decides
            // whether any pixel composited this Gaussian; the gradient
            // math then runs predicated (zero where a pixel did not)
            float e[PPT], dxs[PPT], dys[PPT];
            bool ct[PPT];
            bool anyc = false;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const bool act = pos < last[k];
                evals += act;
                dxs[k] = px[k] - a.x;
                dys[k] = py[k] - a.y;
                const float e2 = exponent2(dxs[k], dys[k], a.z, a.w, b.x);
                e[k] = e2 + b.y;
                ct[k] = act && !(e2 > 0.f) && !(e[k] < rp.lmin);
                anyc |= ct[k];
            }
            if (!__any_sync(0xffffffffu, anyc)) continue;
            float dmx = 0.f, dmy = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dF = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const float G = ex2_approx(e[k]);
                const float alpha = ct[k] ? fminf(rp.amax, G) : 0.f;
                const float inv = rcp_approx(1.f - alpha);
                T[k] = ct[k] ? T[k] * inv : T[k];  // T before this Gaussian
                const float w = alpha * T[k];
                dr = fmaf(w, g0[k], dr);
                dg = fmaf(w, g1[k], dg);
                db = fmaf(w, g2[k], db);
                const float dalpha = T[k] * ((b.z - a0[k]) * g0[k] + (b.w - a1[k]) * g1[k] + (cb - a2[k]) * g2[k]) -
                                     Tf[k] * bgd[k] * inv;
                a0[k] = fmaf(alpha, b.z - a0[k], a0[k]);
                a1[k] = fmaf(alpha, b.w - a1[k], a1[k]);
                a2[k] = fmaf(alpha, cb - a2[k], a2[k]);
                const float de = (ct[k] && !(G > rp.amax)) ? dalpha * alpha * kLn2 : 0.f;
                const float dx = dxs[k], dy = dys[k];
                dF += de;
                dA = fmaf(de * dx, dx, dA);
                dB = fmaf(de * dx, dy, dB);
                dC = fmaf(de * dy, dy, dC);
                dmx -= de * (2.f * a.z * dx + a.w * dy);
                dmy -= de * (a.w * dx + 2.f * b.x * dy);
            }
            // record layout: (dmx, dmy, dA, dB), (dC, dF, dr, dg), (db, -, -, -)
            const float v8[8] = {dmx, dmy, dA, dB, dC, dF, dr, dg};
            const float tot = warp_sum8_transposed(v8, lane);
            db = warp_sum_f(db);
            float *rec = reinterpret_cast<float *>(grad2d + 3 * (rec0 + sg[warp][j]));
            if ((lane & 3) == 0) atomicAdd(rec + (lane >> 2), tot);
            if (lane == 0) atomicAdd(rec + 8, db);
        }
        __syncwarp();
    }
    unsigned long long ev = evals;
    for (int s = 16; s > 0; s >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, s);
    __syncthreads();
    if (lane == 0) atomicAdd(&s_eval, ev);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&stats->eval_bwd, s_eval);
}

template <int TILE, int BATCH>
cudaError_t run_fwd(const gs_batch *b, const uint32_t *order, const uint2 *ranges, const uint32_t *vals,
                    const float4 *splat,
                    const float *colors, RenderParams rp, Stats *stats, float *out_rgb, float *out_T,
                    int32_t *out_last, cudaStream_t s) {
    k_render_fwd<TILE, BATCH><<<b->num_tiles, Cfg<TILE>::NT, 0, s>>>(
        b->frames_dev, b->num_frames, order, ranges, vals, splat, colors, rp, stats, out_rgb, out_T, out_last);
    return cudaGetLastError();
}

template <int TILE, int BATCH>
cudaError_t run_bwd(const gs_batch *b, const uint32_t *order, const uint2 *ranges, const uint32_t *vals,
                    const float4 *splat,
                    const float *colors, RenderParams rp, Stats *stats, const float *in_T, const int32_t *in_last,
                    const float *dL, float4 *grad2d, cudaStream_t s) {
    k_render_bwd<TILE, BATCH><<<b->num_tiles, Cfg<TILE>::NT, 0, s>>>(
        b->frames_dev, b->num_frames, order, ranges, vals, splat, colors, rp, stats, in_T, in_last, dL, grad2d);
    return cudaGetLastError();
}

RenderParams make_params(const gs_opts *o) {
    RenderParams rp;
    rp.lmin = log2f(o->alpha_min);
    rp.amax = o->alpha_max;
    rp.tmin = o->t_min;
    rp.bg0 = o->bg[0];
    rp.bg1 = o->bg[1];
    rp.bg2 = o->bg[2];
    return rp;
}

}  // namespace

#define GS_DISPATCH(TILE_, BATCH_, CALL)                          \
    switch (TILE_ * 1000 + BATCH_) {                               \
    case 8064: return CALL(8, 64);                                 \
    case 8128: return CALL(8, 128);                                \
    case 8256: return CALL(8, 256);                                \
    case 16064: return CALL(16, 64);                               \
    case 16128: return CALL(16, 128);                              \
    case 16256: return CALL(16, 256);                              \
    case 32064: return CALL(32, 64);                               \
    case 32128: return CALL(32, 128);                              \
    case 32256: return CALL(32, 256);                              \
    default: return cudaErrorInvalidValue;                         \
    }

cudaError_t launch_render_fwd(const gs_batch *b, const gs_opts *o, const uint32_t *order, const uint2 *ranges,
                              const uint32_t *vals,
                              const float4 *splat, const float *colors, Stats *stats, float *out_rgb,
                              float *out_T, int32_t *out_last, cudaStream_t s) {
    if (b->num_tiles == 0) return cudaSuccess;
    const RenderParams rp = make_params(o);
#define GS_FWD(T_, B_) run_fwd<T_, B_>(b, order, ranges, vals, splat, colors, rp, stats, out_rgb, out_T, out_last, s)
    GS_DISPATCH(o->tile, o->batch, GS_FWD)
#undef GS_FWD
}

cudaError_t launch_render_bwd(const gs_batch *b, const gs_opts *o, const uint32_t *order, const uint2 *ranges,
                              const uint32_t *vals,
                              const float4 *splat, const float *colors, Stats *stats, const float *in_T,
                              const int32_t *in_last, const float *dL, float4 *grad2d, cudaStream_t s) {
    if (b->num_tiles == 0) return cudaSuccess;
    const RenderParams rp = make_params(o);
#define GS_BWD(T_, B_) run_bwd<T_, B_>(b, order, ranges, vals, splat, colors, rp, stats, in_T, in_last, dL, grad2d, s)
    GS_DISPATCH(o->tile, o->batch, GS_BWD)
#undef GS_BWD
}

}  // namespace gs
