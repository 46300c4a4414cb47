// Phi (Eq. 5): front-to-back alpha compositing of the depth-sorted splats of
// each tile, and its backward (Sec. III-B).
//
// The (frame, tile) work items of the whole batch are taken in the
// heavy-first order gs_bin_sort computes (longest lists first).  A work item
// is cut into compact, near-square bands, and each band is one block of one
// warp, which walks the tile's depth-sorted list on its own: it loads chunks
// of batch/2 entries (prefetching the next chunk into registers while it
// uses the current one), keeps the entries that can reach alpha >= alpha_min
// somewhere in its band, compacts them in order into its shared-memory slot
// and composites them.  A warp stops as soon as all its pixels have stopped,
// and its block ends there (no wait for the tile's other bands).
//
// The heaviest tiles (up to four per SM, the head of the heavy-first order)
// bound the kernel's duration: a band of a tile near the vanishing point
// walks tens of thousands of entries alone.  Each of them is split into two
// work items (upper and lower half) with bands of half the pixels (half the
// pixels per thread), which halves the Gaussians a warp composites and so
// that tile's critical path.  The work items of one launch are: the halves
// of the heavy tiles first (blocks are dispatched in index order, so their
// bands start first), then every other tile whole.  The image does not depend on
// the band shape (see the culling below).
//
// Culling per band is exact: a Gaussian is kept when its alpha box meets the
// band and the minimum of its quadratic form over the band rectangle is
// within reach of alpha_min (the minimum of a convex quadratic over a
// rectangle lies at the centre or on a side the centre is outside of; a
// margin above the rounding of both this test and the per-pixel exponent
// keeps it conservative).
//
// Per pixel and Gaussian (both directions use the same arithmetic):
//   dx = u - mean_x, dy = v - mean_y
//   e2 = A dx^2 + B dx dy + C dy^2     (= power * log2 e)
//   skip if e2 > 0;  e = e2 + F (F = log2 opacity); skip if e < log2 alpha_min
//   alpha = min(alpha_max, 2^e)
//
// The forward also records, per band and per 32 entries of the tile's list,
// a mask of the entries that some pixel of the band composited (one bit
// per entry; each tile's bits start on a word of its own, word
// range.start / 32 + tile, in one array per band slot).  The backward's
// band is the union of one or two forward bands; at batch 64 it loads and
// stages only the entries of the OR of their masks, which skips the band
// test and every entry that no pixel of the band composites (on the
// 1M-Gaussian drive, 12.7M kept (band, Gaussian) entries of the band test
// against 10.5M composited).  At the other batches it keeps its band test.
//
// Backward: walks the pixel's range from its last composited Gaussian back
// to the first, recovering T_i = T_{i+1} / (1 - alpha_i) from the final
// transmittance instead of storing it, with S = light composited behind,
// projected on the pixel's colour gradient g:
//   S_i = sum_{j>i} alpha_j T_j (c_j . g) + T_final (bg . g)
//   dL/dc_i     = alpha_i T_i g
//   dL/dalpha_i = T_i (c_i . g) - S_i / (1 - alpha_i)
//   dL/de       = dL/dalpha_i * alpha_i * ln 2   (0 where alpha is clamped)
// giving dL/dF = dL/de, dL/dA = dL/de dx^2, dL/dB = dL/de dx dy,
// dL/dC = dL/de dy^2, and, as A, B, C are per Gaussian,
// dL/dmean = -(2A sum(dL/de dx) + B sum(dL/de dy), B sum(dL/de dx) + 2C sum(dL/de dy)).
// The nine per-pixel sums are added over the thread's pixels, then over the
// warp (skipped when no lane contributes): eight of them by a transposed
// halving exchange that leaves one total per group of four lanes, which the
// group's first lane adds to the record (eight lanes, contiguous addresses),
// the ninth by a plain shuffle reduction.  The factor ln 2 is applied to the
// warp totals.
#include <algorithm>

#include "common.cuh"

namespace gs {

namespace {

// Pixels per thread: 2 at tiles 8 and 16, 4 at 32; half of that in the
// halves of heavy tiles.
// The forward's pixels per thread: two at tiles 8 and 16 (8x8 bands), four at
// tile 32.  GS_FWD_PPT16 overrides tile 16's value (2 or 4) at build time.
#ifndef GS_FWD_PPT16
#define GS_FWD_PPT16 2
#endif
__host__ __device__ constexpr int pix_per_thread(int tile) { return tile == 32 ? 4 : (tile == 16 ? GS_FWD_PPT16 : 2); }

// The backward's pixels per thread: four at tiles 16 and 32 (16x8 bands, 8x8
// in the halves of heavy tiles), which spreads each kept Gaussian's 9-value
// warp reduction over twice the pixels of the forward's 8x8 bands; two at
// tile 8.  GS_BWD_PPT16 overrides tile 16's value (2 or 4) at build time.
#ifndef GS_BWD_PPT16
#define GS_BWD_PPT16 4
#endif
__host__ __device__ constexpr int bwd_pix_per_thread(int tile) {
    return tile == 8 ? 2 : (tile == 16 ? GS_BWD_PPT16 : 4);
}

// A work item of TILE-wide rows for NT threads at PPT pixels per thread.
// A warp's band holds 32 * PPT pixels in the squarest shape the tile allows:
// 8x4 (32 pixels), 8x8 (64) or 16x8 (128).  Of two bands of equal area the
// squarer one has the shorter border, so fewer Gaussians reach it without
// compositing any of its pixels (on the 1M-Gaussian drive frames, 8x8 keeps
// 6-7% fewer (band, Gaussian) pairs than 16x4, and 8x4 12% fewer than 16x2).
// Lane l holds column l mod BW of its band and the PPT vertically adjacent
// rows from (l / BW) * PPT; the bands fill the item row of bands by row.
template <int TILE, int PPT, int NT>
struct Cfg {
    static constexpr int NW = NT / 32;                   // warps per block
    static constexpr int BW = 32 * PPT >= 128 ? 16 : 8;  // band width
    static constexpr int BH = 32 * PPT / BW;             // band height
    static constexpr int BPR = TILE / BW;                // bands per row of bands
    static constexpr int ROWS = NW / BPR * BH;           // pixel rows of the item
    static_assert(NT % 32 == 0 && TILE % BW == 0 && 32 % BW == 0 && NW % BPR == 0 && ROWS <= TILE,
                  "the bands tile the work item");
};

// The forward bands that tile backward band wb of a work item of the same
// kind (whole tile or heavy half), as forward band indices: the backward's
// bands are unions of NX x NY forward bands (two 8x8 bands for a 16x8 band at
// tile 16; the same band at tiles 8 and 32).
template <int TILE, int PPTF, int NTF, int PPTB, int NTB>
struct BandMap {
    using Cf = Cfg<TILE, PPTF, NTF>;
    using Cb = Cfg<TILE, PPTB, NTB>;
    static constexpr int NX = Cb::BW / Cf::BW, NY = Cb::BH / Cf::BH, N = NX * NY;
    static_assert(Cb::BW % Cf::BW == 0 && Cb::BH % Cf::BH == 0 && N >= 1 && N <= 2 && Cf::ROWS == Cb::ROWS,
                  "backward bands are unions of at most two forward bands");
    __device__ static int fwd_band(int wb, int k) {
        const int bx = (wb % Cb::BPR) * Cb::BW + (k % NX) * Cf::BW;
        const int by = (wb / Cb::BPR) * Cb::BH + (k / NX) * Cf::BH;
        return (by / Cf::BH) * Cf::BPR + bx / Cf::BW;
    }
};

template <int TILE>
struct Threads {
    static constexpr int NT = TILE * TILE / pix_per_thread(TILE);
};


template <int TILE>
struct BwdThreads {
    static constexpr int NT = TILE * TILE / bwd_pix_per_thread(TILE);
};

struct RenderParams {
    float lmin;       // log2(alpha_min)
    float amax, tmin;
    float bg0, bg1, bg2;
};

// Exponent e2 = A dx^2 + B dx dy + C dy^2 with a fixed operation order (no
// contraction freedom), shared by the forward and the backward and by every
// band shape.
__device__ __forceinline__ float exponent2(float dx, float dy, float A, float B, float C) {
    const float bdy = __fmul_rn(B, dy);
    const float t = __fmaf_rn(A, dx, bdy);
    const float cdy = __fmul_rn(C, dy);
    const float q = __fmul_rn(cdy, dy);
    return __fmaf_rn(dx, t, q);
}

// exponent2 for two vertically adjacent pixels of a thread (offsets dx and
// dy.x, dy.y) in packed f32x2 arithmetic: each element is rounded exactly as
// the scalar operations of exponent2 round it, so both give the same bits.
__device__ __forceinline__ float2 exponent2x2(float dx, float2 dy, float A, float B, float C) {
    const float2 dx2 = make_float2(dx, dx);
    const float2 bdy = __fmul2_rn(make_float2(B, B), dy);
    const float2 t = __ffma2_rn(make_float2(A, A), dx2, bdy);
    const float2 cdy = __fmul2_rn(make_float2(C, C), dy);
    const float2 q = __fmul2_rn(cdy, dy);
    return __ffma2_rn(dx2, t, q);
}

// Whether a Gaussian with centre m, exponent coefficients (A, B, C), F =
// log2 opacity and alpha box half-widths (rx, ry) can reach alpha >=
// alpha_min at some point of the band [xlo, xhi] x [ylo, yhi].
// With P(d) = -(A dx^2 + B dx dy + C dy^2) (positive definite), a pixel can
// pass only where P <= F - lmin.  The minimum of P over the band is 0 with
// the centre inside; otherwise it lies on a side that the centre is outside
// of, where P restricted to the side is a parabola minimised at a clamped
// point.  The margin 2^-10 (F - lmin) + 2^-16 (|A| Dx^2 + |B| Dx Dy + |C| Dy^2)
// (Dx, Dy the largest offsets within the band) exceeds the rounding error
// of this test and of exponent2 by more than an order of magnitude, so a
// Gaussian that the per-pixel test would composite is never dropped.
__device__ __forceinline__ bool band_hits(float mx, float my, float A, float B, float C, float F, float rx,
                                          float ry, float lmin, float xlo, float xhi, float ylo, float yhi) {
    if (!((mx + rx >= xlo) && (mx - rx <= xhi) && (my + ry >= ylo) && (my - ry <= yhi))) return false;
    const float a = -A, b = -B, c = -C;
    const float x0 = xlo - mx, x1 = xhi - mx, y0 = ylo - my, y1 = yhi - my;
    const bool out_x = x0 > 0.f || x1 < 0.f, out_y = y0 > 0.f || y1 < 0.f;
    float pmin = 0.f;
    if (out_x || out_y) {
        float px = INFINITY, py = INFINITY;
        if (out_x) {
            const float dx = x0 > 0.f ? x0 : x1;
            const float dy = fminf(fmaxf(__fdividef(-b * dx, 2.f * c), y0), y1);
            px = dx * (a * dx + b * dy) + c * dy * dy;
        }
        if (out_y) {
            const float dy = y0 > 0.f ? y0 : y1;
            const float dx = fminf(fmaxf(__fdividef(-b * dy, 2.f * a), x0), x1);
            py = dx * (a * dx + b * dy) + c * dy * dy;
        }
        pmin = fminf(px, py);
    }
    const float lim = F - lmin;
    const float Dx = fmaxf(fabsf(x0), fabsf(x1)), Dy = fmaxf(fabsf(y0), fabsf(y1));
    const float mag = a * Dx * Dx + fabsf(b) * Dx * Dy + c * Dy * Dy;
    return pmin <= lim + fabsf(lim) * 0x1p-10f + mag * 0x1p-16f;
}

// One Gaussian of a warp's chunk, as loaded from global memory.
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

// A kept Gaussian in the warp's shared-memory slot.
struct alignas(16) Staged {
    float4 a;  // mean_x, mean_y, A, B
    float4 b;  // C, F, r, g
    uint4 z;   // bits of b, position in the tile's range, Gaussian index, 0
};

// Band of warp `warp` in the work item starting at row rbase of the tile
// whose first image row is y_tile, clipped to the image, and the image
// column u and first image row v0 of the lane's pixels.
template <int TILE, class C, int PPT>
__device__ __forceinline__ void band_of(int tx, int y_tile, int rbase, int warp, int lane, int W, int H, float &xlo,
                                        float &xhi, float &ylo, float &yhi, int &u, int &v0) {
    const int x0 = tx * TILE + (warp % C::BPR) * C::BW;
    const int y0 = y_tile + rbase + (warp / C::BPR) * C::BH;
    xlo = (float)x0;
    xhi = (float)min(x0 + C::BW - 1, W - 1);
    ylo = (float)y0;
    yhi = (float)min(y0 + C::BH - 1, H - 1);
    u = x0 + lane % C::BW;
    v0 = y0 + (lane / C::BW) * PPT;
}

// Compact the chunk's kept entries, in order, into the warp's slot; returns
// how many were kept.  pos0 + p * 32 + lane is entry p's position.
template <int PER>
__device__ __forceinline__ int compact(Staged *st, const Entry (&cu)[PER], int pos0, int lane, float lmin, float xlo,
                                       float xhi, float ylo, float yhi) {
    const uint32_t lt_mask = (1u << lane) - 1u;
    int cnt = 0;
#pragma unroll
    for (int p = 0; p < PER; p++) {
        const Entry &e = cu[p];
        const bool hit = e.valid && band_hits(e.a.x, e.a.y, e.a.z, e.a.w, e.b.x, e.b.y, e.b.z, e.b.w, lmin, xlo, xhi,
                                              ylo, yhi);
        const uint32_t msk = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            Staged &s = st[cnt + __popc(msk & lt_mask)];
            s.a = e.a;
            s.b = make_float4(e.b.x, e.b.y, e.cr, e.cg);
            s.z = make_uint4(__float_as_uint(e.cb), (uint32_t)(pos0 + p * 32 + lane), e.g, 0u);
        }
        cnt += __popc(msk);
    }
    __syncwarp();
    return cnt;
}

// Forward of one work item: rows [rbase, rbase + ROWS) of tile t.
template <int TILE, int PPT, int NT, int BATCH>
__device__ __forceinline__ void fwd_item(int t, int rbase, int warp, uint32_t *__restrict__ bits, Staged *st,
                                         const gs_frame *__restrict__ frames, int F,
                                         const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                                         const float4 *__restrict__ splat, const float *__restrict__ colors,
                                         const RenderParams &rp, Stats *__restrict__ stats,
                                         float *__restrict__ out_rgb, float *__restrict__ out_T,
                                         int32_t *__restrict__ out_last) {
    using C = Cfg<TILE, PPT, NT>;
    constexpr int CH = BATCH / 2, PER = CH / 32;
    static_assert(C::ROWS * (PPT == pix_per_thread(TILE) ? 1 : 2) == TILE, "a work item is a tile or half of one");
    const int lane = threadIdx.x;
    const int f = frame_of_tile(frames, F, t);
    const gs_frame &fr = frames[f];
    const int W = fr.width, H = fr.height;
    const int lt = t - fr.tile_offset;
    const int tx = lt % fr.tiles_x, ty = lt / fr.tiles_x;
    const int y_tile = fr.row0 + ty * TILE;  // image row of the tile's first row (frames may be cropped)
    float xlo, xhi, ylo, yhi;
    int u, v0;  // the thread's image column and first image row
    band_of<TILE, C, PPT>(tx, y_tile, rbase, warp, lane, W, H, xlo, xhi, ylo, yhi, u, v0);
    const float px = (float)u;
    float py[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT];
    int last[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        py[k] = (float)(v0 + k);
        done[k] = !(u < W && v0 + k < H);
        T[k] = 1.f;
        c0[k] = c1[k] = c2[k] = 0.f;
        last[k] = 0;
    }
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    const long long rec0 = fr.record_offset;
    const float *col = colors + 3 * (size_t)fr.gauss_offset;
    unsigned evals = 0;  // composited (pixel, Gaussian) pairs
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
        const int cnt = compact<PER>(st, cu, cb0, lane, rp.lmin, xlo, xhi, ylo, yhi);
        uint32_t cmask[PER];  // chunk entries that some pixel of the band composites, 32 per word
#pragma unroll
        for (int q = 0; q < PER; q++) cmask[q] = 0u;
        for (int j = 0; j < cnt; j++) {
            const float4 a = st[j].a, b = st[j].b;
            // every lane evaluates the exponent; one warp vote decides
            // whether any pixel composites this Gaussian, and the
            // compositing itself runs predicated (no divergence)
            const float dx = px - a.x;
            float e[PPT];
            bool ct[PPT];
            bool anyc = false;
            if constexpr (PPT % 2 == 0) {
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 e2 = exponent2x2(
                        dx, __fadd2_rn(make_float2(py[k], py[k + 1]), make_float2(-a.y, -a.y)), a.z, a.w, b.x);
                    const float2 ev = __fadd2_rn(e2, make_float2(b.y, b.y));
                    e[k] = ev.x;
                    e[k + 1] = ev.y;
                    ct[k] = !done[k] && !(e2.x > 0.f) && !(ev.x < rp.lmin);
                    ct[k + 1] = !done[k + 1] && !(e2.y > 0.f) && !(ev.y < rp.lmin);
                    anyc = anyc || ct[k] || ct[k + 1];
                }
            } else {
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const float e2 = exponent2(dx, py[k] - a.y, a.z, a.w, b.x);
                e[k] = e2 + b.y;
                ct[k] = !done[k] && !(e2 > 0.f) && !(e[k] < rp.lmin);
                anyc |= ct[k];
            }
            }
            if (!__any_sync(0xffffffffu, anyc)) continue;
            const uint4 z = st[j].z;
            // bit (position mod 32), by a funnel shift that wraps its count
            if constexpr (PER == 1) {
                cmask[0] |= __funnelshift_l(0u, 1u, z.y);
            } else {
                const int q0 = ((int)z.y - cb0) >> 5;
#pragma unroll
                for (int q = 0; q < PER; q++)
                    if (q0 == q) cmask[q] |= __funnelshift_l(0u, 1u, z.y);
            }
            const float cb = __uint_as_float(z.x);
            const int pos1 = (int)z.y + 1;
            if constexpr (PPT % 2 == 0) {
                // the pixels two by two in packed f32x2 arithmetic (each
                // element rounded as the scalar loop below rounds it)
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 al = make_float2(fminf(rp.amax, ex2_approx(e[k])), fminf(rp.amax, ex2_approx(e[k + 1])));
                    const float2 T2 = make_float2(T[k], T[k + 1]);
                    const float2 nT = __fmul2_rn(T2, __ffma2_rn(al, make_float2(-1.f, -1.f), make_float2(1.f, 1.f)));
                    const float2 wa = __fmul2_rn(al, T2);
                    const bool s0 = ct[k] && nT.x < rp.tmin, s1 = ct[k + 1] && nT.y < rp.tmin;
                    const bool b0 = ct[k] && !s0, b1 = ct[k + 1] && !s1;
                    done[k] = done[k] || s0;
                    done[k + 1] = done[k + 1] || s1;
                    evals += (unsigned)b0 + (unsigned)b1;
                    const float2 w = make_float2(b0 ? wa.x : 0.f, b1 ? wa.y : 0.f);
                    const float2 r = __ffma2_rn(make_float2(b.z, b.z), w, make_float2(c0[k], c0[k + 1]));
                    const float2 g = __ffma2_rn(make_float2(b.w, b.w), w, make_float2(c1[k], c1[k + 1]));
                    const float2 bl = __ffma2_rn(make_float2(cb, cb), w, make_float2(c2[k], c2[k + 1]));
                    c0[k] = r.x;
                    c0[k + 1] = r.y;
                    c1[k] = g.x;
                    c1[k + 1] = g.y;
                    c2[k] = bl.x;
                    c2[k + 1] = bl.y;
                    T[k] = b0 ? nT.x : T[k];
                    T[k + 1] = b1 ? nT.y : T[k + 1];
                    last[k] = b0 ? pos1 : last[k];
                    last[k + 1] = b1 ? pos1 : last[k + 1];
                }
            } else {
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const float alpha = fminf(rp.amax, ex2_approx(e[k]));
                const float nT = T[k] * (1.f - alpha);
                const bool stop = ct[k] && nT < rp.tmin;
                const bool blend = ct[k] && !stop;
                done[k] = done[k] || stop;
                evals += blend;
                const float w = blend ? alpha * T[k] : 0.f;
                c0[k] = fmaf(b.z, w, c0[k]);
                c1[k] = fmaf(b.w, w, c1[k]);
                c2[k] = fmaf(cb, w, c2[k]);
                T[k] = blend ? nT : T[k];
                last[k] = blend ? pos1 : last[k];
            }
            }
        }
        if (lane < PER && cb0 + 32 * lane < n) {  // the words of list positions (the tile's own)
            uint32_t word = cmask[0];
#pragma unroll
            for (int q = 1; q < PER; q++) word = lane == q ? cmask[q] : word;
            bits[(long long)(range.x >> 5) + t + (cb0 >> 5) + lane] = word;
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int v = v0 + k;
        if (!(u < W && v < H)) continue;
        const long long pix = fr.pixel_offset + (long long)(v - fr.row0) * W + u;
        out_rgb[3 * pix] = c0[k] + T[k] * rp.bg0;
        out_rgb[3 * pix + 1] = c1[k] + T[k] * rp.bg1;
        out_rgb[3 * pix + 2] = c2[k] + T[k] * rp.bg2;
        out_T[pix] = T[k];
        out_last[pix] = last[k];
    }
    // composited-pair counter (the roofline's unit): warp sums, one atomic per warp
    unsigned long long ev = evals;
    for (int s = 16; s > 0; s >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, s);
    if (lane == 0) atomicAdd(&stats->eval_fwd, ev);
}

// Work item i of a launch: the halves of the `heavy` first tiles of the
// heavy-first order, then the other tiles whole.  Each block is one warp,
// one band of an item (blocks i * NW .. i * NW + NW - 1 are item i's bands),
// so a warp that finishes its band frees its slot for the next block
// instead of waiting for the other bands of its tile.
template <int TILE, int BATCH>
__global__ void __launch_bounds__(32)
k_render_fwd(const gs_frame *__restrict__ frames, int F, const uint32_t *__restrict__ order, int heavy,
             uint32_t *__restrict__ bits, long long band_words,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
             const float4 *__restrict__ splat, const float *__restrict__ colors, RenderParams rp,
             Stats *__restrict__ stats, float *__restrict__ out_rgb, float *__restrict__ out_T,
             int32_t *__restrict__ out_last) {
    constexpr int NT = Threads<TILE>::NT, PL = pix_per_thread(TILE), NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Staged *st = reinterpret_cast<Staged *>(smem_raw);
    const int i = (int)blockIdx.x / NW, warp = (int)blockIdx.x % NW;
    if (i < 2 * heavy)
        fwd_item<TILE, PL / 2, NT, BATCH>((int)order[i >> 1], (i & 1) * (TILE / 2), warp,
                                          bits + band_words * (NW * (1 + (i & 1)) + warp), st, frames, F, ranges,
                                          vals, splat, colors, rp, stats, out_rgb, out_T, out_last);
    else
        fwd_item<TILE, PL, NT, BATCH>((int)order[i - heavy], 0, warp, bits + band_words * warp, st, frames, F, ranges,
                                      vals, splat, colors, rp, stats, out_rgb, out_T, out_last);
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

// Sum eight per-lane values over the warp by halving exchanges: at each step
// a lane keeps half of its values and sends the other half to its partner,
// so the exchanges shrink 4, 2, 1, 1, 1 (8 shuffles instead of 40).  On
// return every lane holds the warp total of component
// c = 4*bit4(lane) + 2*bit3(lane) + bit2(lane) = lane >> 2.
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

// Backward of one work item: rows [rbase, rbase + ROWS) of tile t.
template <int TILE, int PPT, int NT, int BATCH>
__device__ __forceinline__ void bwd_item(int t, int rbase, int warp, const uint32_t *__restrict__ bits,
                                         const uint32_t *__restrict__ bits2, Staged *st_all,
                                         const gs_frame *__restrict__ frames, int F,
                                         const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                                         const float4 *__restrict__ splat, const float *__restrict__ colors,
                                         const RenderParams &rp, Stats *__restrict__ stats,
                                         const float *__restrict__ in_T, const int32_t *__restrict__ in_last,
                                         const float *__restrict__ dL_drgb, float4 *__restrict__ grad2d) {
    using C = Cfg<TILE, PPT, NT>;
    constexpr int CH = BATCH / 2, PER = CH / 32;
    static_assert(C::ROWS * (PPT == bwd_pix_per_thread(TILE) ? 1 : 2) == TILE, "a work item is a tile or half of one");
    const int lane = threadIdx.x & 31;
    // the warp's slot, indexed by its warp in the block (the only one);
    // written this way, ptxas schedules the loop with 92 registers instead
    // of 80, which measured 3.5% faster (2.63 vs 2.73 ms on the 8-frame
    // drive)
    Staged *st = st_all + (threadIdx.x >> 5) * CH;
    const int f = frame_of_tile(frames, F, t);
    const gs_frame &fr = frames[f];
    const int W = fr.width, H = fr.height;
    const int lt = t - fr.tile_offset;
    const int tx = lt % fr.tiles_x, ty = lt / fr.tiles_x;
    const int y_tile = fr.row0 + ty * TILE;
    float xlo, xhi, ylo, yhi;
    int u, v0;
    band_of<TILE, C, PPT>(tx, y_tile, rbase, warp, lane, W, H, xlo, xhi, ylo, yhi, u, v0);
    const float px = (float)u;
    // the range of this tile; a pixel's start position never exceeds it
    const uint2 range = ranges[t];
    const int n = (int)(range.y - range.x);
    float py[PPT], T[PPT], S[PPT], g0[PPT], g1[PPT], g2[PPT];
    int last[PPT];
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int v = v0 + k;
        py[k] = (float)v;
        if (u < W && v < H) {
            const long long pix = fr.pixel_offset + (long long)(v - fr.row0) * W + u;
            T[k] = in_T[pix];
            last[k] = min(max(in_last[pix], 0), n);
            g0[k] = dL_drgb[3 * pix];
            g1[k] = dL_drgb[3 * pix + 1];
            g2[k] = dL_drgb[3 * pix + 2];
        } else {
            T[k] = 1.f;
            last[k] = 0;
            g0[k] = g1[k] = g2[k] = 0.f;
        }
        S[k] = T[k] * (rp.bg0 * g0[k] + rp.bg1 * g1[k] + rp.bg2 * g2[k]);
        mylast = max(mylast, last[k]);
    }
    // each warp walks its own part of the list backwards, from the largest
    // start position of its pixels, in chunks of CH (the next one prefetched)
    const int warp_last = __reduce_max_sync(0xffffffffu, mylast);
    const long long rec0 = fr.record_offset;
    const float *col = colors + 3 * (size_t)fr.gauss_offset;
    unsigned evals = 0;  // composited (pixel, Gaussian) pairs
    // At batch 64 (32-entry chunks) the chunks are aligned to 32 list
    // positions, and only the entries that some pixel of one of the forward
    // bands tiling this band composited (the forward's masks) are loaded and
    // staged, in order.  Every entry the band's pixels composite is among
    // them (the forward composites a superset), so the result is the same as
    // with the band test, which picks the entries at the other batches.
    constexpr bool kBits = CH == 32;
    const long long wbase = (long long)(range.x >> 5) + t;
    const uint32_t lt_mask = (1u << lane) - 1u;
    Entry nx[PER];
    uint32_t mnx = 0;
    {
        const int c0 = kBits ? ((warp_last - 1) & ~31) : max(0, warp_last - CH);
        if (kBits && warp_last > 0) {
            const int k = warp_last - c0;
            mnx = (bits[wbase + (c0 >> 5)] | bits2[wbase + (c0 >> 5)]) & (k >= 32 ? 0xffffffffu : (1u << k) - 1u);
        }
#pragma unroll
        for (int p = 0; p < PER; p++) {
            const int i = c0 + p * 32 + lane;
            const bool want = kBits ? ((mnx >> lane) & 1u) != 0u : i < warp_last;
            load_entry(nx[p], want && warp_last > 0, vals, range.x + i, rec0, splat, col);
        }
    }
    for (int c_end = warp_last; c_end > 0;) {
        const int c0 = kBits ? ((c_end - 1) & ~31) : max(0, c_end - CH);
        Entry cu[PER];
#pragma unroll
        for (int p = 0; p < PER; p++) cu[p] = nx[p];
        const uint32_t m = mnx;
        if (c0 > 0) {
            const int n0 = kBits ? c0 - 32 : max(0, c0 - CH);
            if (kBits) mnx = bits[wbase + (n0 >> 5)] | bits2[wbase + (n0 >> 5)];
#pragma unroll
            for (int p = 0; p < PER; p++) {
                const int i = n0 + p * 32 + lane;
                const bool want = kBits ? ((mnx >> lane) & 1u) != 0u : i < c0;
                load_entry(nx[p], want, vals, range.x + i, rec0, splat, col);
            }
        }
        int cnt;
        if constexpr (kBits) {
            if ((m >> lane) & 1u) {
                Staged &sg = st[__popc(m & lt_mask)];
                sg.a = cu[0].a;
                sg.b = make_float4(cu[0].b.x, cu[0].b.y, cu[0].cr, cu[0].cg);
                sg.z = make_uint4(__float_as_uint(cu[0].cb), (uint32_t)(c0 + lane), cu[0].g, 0u);
            }
            __syncwarp();
            cnt = __popc(m);
        } else {
            cnt = compact<PER>(st, cu, c0, lane, rp.lmin, xlo, xhi, ylo, yhi);
        }
        for (int j = cnt - 1; j >= 0; j--) {
            const float4 a = st[j].a, b = st[j].b;
            const uint4 z = st[j].z;  // b, pos, g
            const int pos = (int)z.y;
            // every lane evaluates the exponent; one warp vote decides
            // whether any pixel composited this Gaussian; the gradient
            // math then runs predicated (zero where a pixel did not)
            const float dx = px - a.x;
            float e[PPT], dy[PPT];
            bool ct[PPT];
            bool anyc = false;
            if constexpr (PPT % 2 == 0) {
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float2 d2 = __fadd2_rn(make_float2(py[k], py[k + 1]), make_float2(-a.y, -a.y));
                    dy[k] = d2.x;
                    dy[k + 1] = d2.y;
                    const float2 e2 = exponent2x2(dx, d2, a.z, a.w, b.x);
                    const float2 ev = __fadd2_rn(e2, make_float2(b.y, b.y));
                    e[k] = ev.x;
                    e[k + 1] = ev.y;
                    ct[k] = pos < last[k] && !(e2.x > 0.f) && !(ev.x < rp.lmin);
                    ct[k + 1] = pos < last[k + 1] && !(e2.y > 0.f) && !(ev.y < rp.lmin);
                    anyc = anyc || ct[k] || ct[k + 1];
                }
            } else {
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                dy[k] = py[k] - a.y;
                const float e2 = exponent2(dx, dy[k], a.z, a.w, b.x);
                e[k] = e2 + b.y;
                ct[k] = pos < last[k] && !(e2 > 0.f) && !(e[k] < rp.lmin);
                anyc |= ct[k];
            }
            }
            if (!__any_sync(0xffffffffu, anyc)) continue;
            const float cb = __uint_as_float(z.x);
            // per-thread sums: sum de dx, sum de dy, dA, dB, dC, dF, dr, dg, db
            float sx = 0.f, sy = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dF = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
            if constexpr (PPT % 2 == 0) {
                // the thread's pixels two by two in packed f32x2 arithmetic
                // (the same terms as the scalar loop below)
                float2 sxv, syv, dAv, dBv, dCv, dFv, drv, dgv, dbv;
#pragma unroll
                for (int k = 0; k < PPT; k += 2) {
                    const float G0 = ex2_approx(ct[k] ? e[k] : -INFINITY);
                    const float G1 = ex2_approx(ct[k + 1] ? e[k + 1] : -INFINITY);
                    const float2 al = make_float2(fminf(rp.amax, G0), fminf(rp.amax, G1));
                    const float2 om = __ffma2_rn(al, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));  // 1 - alpha
                    const float2 inv = make_float2(ct[k] ? rcp_approx(om.x) : 1.f, ct[k + 1] ? rcp_approx(om.y) : 1.f);
                    const float2 T2 = __fmul2_rn(make_float2(T[k], T[k + 1]), inv);  // T before this Gaussian
                    T[k] = T2.x;
                    T[k + 1] = T2.y;
                    const float2 w = __fmul2_rn(al, T2);
                    const float2 gr = make_float2(g0[k], g0[k + 1]), gg = make_float2(g1[k], g1[k + 1]),
                                 gb = make_float2(g2[k], g2[k + 1]);
                    const float2 cd = __ffma2_rn(make_float2(b.z, b.z), gr,
                                                 __ffma2_rn(make_float2(b.w, b.w), gg,
                                                            __fmul2_rn(make_float2(cb, cb), gb)));
                    const float2 S2 = make_float2(S[k], S[k + 1]);
                    const float2 dal = __ffma2_rn(T2, cd, __fmul2_rn(make_float2(-S2.x, -S2.y), inv));
                    const float2 Sn = __ffma2_rn(w, cd, S2);
                    S[k] = Sn.x;
                    S[k + 1] = Sn.y;
                    float2 de = __fmul2_rn(dal, al);  // dL/de / ln 2
                    de.x = G0 > rp.amax ? 0.f : de.x;
                    de.y = G1 > rp.amax ? 0.f : de.y;
                    const float2 dx2 = make_float2(dx, dx), dy2 = make_float2(dy[k], dy[k + 1]);
                    const float2 tx2 = __fmul2_rn(de, dx2), ty2 = __fmul2_rn(de, dy2);
                    if (k == 0) {
                        sxv = tx2;
                        syv = ty2;
                        dAv = __fmul2_rn(tx2, dx2);
                        dBv = __fmul2_rn(tx2, dy2);
                        dCv = __fmul2_rn(ty2, dy2);
                        dFv = de;
                        drv = __fmul2_rn(w, gr);
                        dgv = __fmul2_rn(w, gg);
                        dbv = __fmul2_rn(w, gb);
                    } else {
                        sxv = __fadd2_rn(sxv, tx2);
                        syv = __fadd2_rn(syv, ty2);
                        dAv = __ffma2_rn(tx2, dx2, dAv);
                        dBv = __ffma2_rn(tx2, dy2, dBv);
                        dCv = __ffma2_rn(ty2, dy2, dCv);
                        dFv = __fadd2_rn(dFv, de);
                        drv = __ffma2_rn(w, gr, drv);
                        dgv = __ffma2_rn(w, gg, dgv);
                        dbv = __ffma2_rn(w, gb, dbv);
                    }
                    evals += (unsigned)ct[k] + (unsigned)ct[k + 1];
                }
                sx = sxv.x + sxv.y;
                sy = syv.x + syv.y;
                dA = dAv.x + dAv.y;
                dB = dBv.x + dBv.y;
                dC = dCv.x + dCv.y;
                dF = dFv.x + dFv.y;
                dr = drv.x + drv.y;
                dg = dgv.x + dgv.y;
                db = dbv.x + dbv.y;
            } else {
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                // a pixel that does not composite this Gaussian gets alpha = 0
                // (2^-inf), so every term below vanishes for it
                const float G = ex2_approx(ct[k] ? e[k] : -INFINITY);
                const float alpha = fminf(rp.amax, G);
                const float inv = ct[k] ? rcp_approx(1.f - alpha) : 1.f;
                T[k] *= inv;  // T before this Gaussian
                const float w = alpha * T[k];
                dr = fmaf(w, g0[k], dr);
                dg = fmaf(w, g1[k], dg);
                db = fmaf(w, g2[k], db);
                const float cd = fmaf(b.z, g0[k], fmaf(b.w, g1[k], cb * g2[k]));
                const float dal = T[k] * cd - S[k] * inv;
                S[k] = fmaf(w, cd, S[k]);
                const float de = G > rp.amax ? 0.f : dal * alpha;  // dL/de / ln 2
                const float tx_ = de * dx, ty_ = de * dy[k];
                dA = fmaf(tx_, dx, dA);
                dB = fmaf(tx_, dy[k], dB);
                dC = fmaf(ty_, dy[k], dC);
                sx += tx_;
                sy += ty_;
                dF += de;
                evals += ct[k];
            }
            }
            // record layout: (dmx, dmy, dA, dB), (dC, dF, dr, dg), (db, -, -, -)
            const float v8[8] = {sx, sy, dA, dB, dC, dF, dr, dg};
            const float tot = warp_sum8_transposed(v8, lane);
            const float dbt = warp_sum_f(db);
            // lanes 0-3 hold sum de dx and lanes 4-7 sum de dy: the mean gradient
            const float oth = __shfl_xor_sync(0xffffffffu, tot, 4);
            const int comp = lane >> 2;
            float val = comp < 6 ? tot * kLn2 : tot;
            val = comp == 0 ? -kLn2 * (2.f * a.z * tot + a.w * oth) : val;
            val = comp == 1 ? -kLn2 * (a.w * oth + 2.f * b.x * tot) : val;
            float *rec = reinterpret_cast<float *>(grad2d + 3 * (rec0 + z.z));
            if ((lane & 3) == 0) atomicAdd(rec + comp, val);
            if (lane == 0) atomicAdd(rec + 8, dbt);
        }
        __syncwarp();
        c_end = c0;
    }
    unsigned long long ev = evals;
    for (int s = 16; s > 0; s >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, s);
    if (lane == 0) atomicAdd(&stats->eval_bwd, ev);
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(32)
k_render_bwd(const gs_frame *__restrict__ frames, int F, const uint32_t *__restrict__ order, int heavy,
             const uint32_t *__restrict__ bits, long long band_words,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
             const float4 *__restrict__ splat, const float *__restrict__ colors, RenderParams rp,
             Stats *__restrict__ stats, const float *__restrict__ in_T, const int32_t *__restrict__ in_last,
             const float *__restrict__ dL_drgb, float4 *__restrict__ grad2d) {
    constexpr int NT = BwdThreads<TILE>::NT, PL = bwd_pix_per_thread(TILE), NW = NT / 32;
    constexpr int NTF = Threads<TILE>::NT, PLF = pix_per_thread(TILE), NWF = NTF / 32;
    using MW = BandMap<TILE, PLF, NTF, PL, NT>;
    using MH = BandMap<TILE, PLF / 2, NTF, PL / 2, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Staged *st = reinterpret_cast<Staged *>(smem_raw);
    const int i = (int)blockIdx.x / NW, warp = (int)blockIdx.x % NW;
    if (i < 2 * heavy)
        bwd_item<TILE, PL / 2, NT, BATCH>((int)order[i >> 1], (i & 1) * (TILE / 2), warp,
                                          bits + band_words * (NWF * (1 + (i & 1)) + MH::fwd_band(warp, 0)),
                                          bits + band_words * (NWF * (1 + (i & 1)) + MH::fwd_band(warp, MH::N - 1)),
                                          st, frames, F, ranges, vals, splat, colors, rp, stats, in_T, in_last,
                                          dL_drgb, grad2d);
    else
        bwd_item<TILE, PL, NT, BATCH>((int)order[i - heavy], 0, warp, bits + band_words * MW::fwd_band(warp, 0),
                                      bits + band_words * MW::fwd_band(warp, MW::N - 1), st, frames, F,
                                      ranges, vals, splat, colors, rp, stats, in_T, in_last, dL_drgb, grad2d);
}

// ---------------------------------------------------------------- launch

// Heavy tiles split in halves: four per SM, at most a quarter of the tiles
// (on the 8-frame drive: 4.98 ms per iteration against 5.00 ms at two per SM,
// 5.01 at one, 5.00 at eight and 6.02 with no split).
int heavy_tiles(long long num_tiles) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int)std::min<long long>(num_tiles / 4, 4ll * sms);
}

// Dynamic shared memory of a render kernel (the warp's staging slot), with
// the opt-in for more than the default 48 KB per block (static shared memory
// included) set before each launch that needs it (a per-device function
// attribute; cheap and legal while capturing).
template <typename K>
cudaError_t smem_opt_in(K kern, size_t bytes) {
    if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int BATCH>
constexpr size_t stage_bytes() {
    return (size_t)(BATCH / 2) * sizeof(Staged);
}

template <int TILE, int BATCH>
cudaError_t run_fwd(const gs_batch *b, const uint32_t *order, const uint2 *ranges, const uint32_t *vals,
                    const float4 *splat, const float *colors, RenderParams rp, Stats *stats, float *out_rgb,
                    float *out_T, int32_t *out_last, uint32_t *masks, long long band_words, cudaStream_t s) {
    constexpr size_t smem = stage_bytes<BATCH>();
    const int heavy = heavy_tiles(b->num_tiles);
    cudaError_t e = smem_opt_in(k_render_fwd<TILE, BATCH>, smem);
    if (e != cudaSuccess) return e;
    k_render_fwd<TILE, BATCH><<<(unsigned)((b->num_tiles + heavy) * (Threads<TILE>::NT / 32)), 32, smem, s>>>(
        b->frames_dev, b->num_frames, order, heavy, masks, band_words, ranges, vals, splat, colors, rp, stats,
        out_rgb, out_T, out_last);
    return cudaGetLastError();
}

template <int TILE, int BATCH>
cudaError_t run_bwd(const gs_batch *b, const uint32_t *order, const uint2 *ranges, const uint32_t *vals,
                    const float4 *splat, const float *colors, RenderParams rp, Stats *stats, const float *in_T,
                    const int32_t *in_last, const float *dL, float4 *grad2d, const uint32_t *masks,
                    long long band_words, cudaStream_t s) {
    constexpr size_t smem = stage_bytes<BATCH>();
    const int heavy = heavy_tiles(b->num_tiles);
    cudaError_t e = smem_opt_in(k_render_bwd<TILE, BATCH>, smem);
    if (e != cudaSuccess) return e;
    k_render_bwd<TILE, BATCH><<<(unsigned)((b->num_tiles + heavy) * (BwdThreads<TILE>::NT / 32)), 32, smem, s>>>(
        b->frames_dev, b->num_frames, order, heavy, masks, band_words, ranges, vals, splat, colors, rp, stats, in_T,
        in_last, dL, grad2d);
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
                              float *out_T, int32_t *out_last, uint32_t *masks, long long band_words,
                              cudaStream_t s) {
    if (b->num_tiles == 0) return cudaSuccess;
    const RenderParams rp = make_params(o);
#define GS_FWD(T_, B_) \
    run_fwd<T_, B_>(b, order, ranges, vals, splat, colors, rp, stats, out_rgb, out_T, out_last, masks, band_words, s)
    GS_DISPATCH(o->tile, o->batch, GS_FWD)
#undef GS_FWD
}

cudaError_t launch_render_bwd(const gs_batch *b, const gs_opts *o, const uint32_t *order, const uint2 *ranges,
                              const uint32_t *vals,
                              const float4 *splat, const float *colors, Stats *stats, const float *in_T,
                              const int32_t *in_last, const float *dL, float4 *grad2d, const uint32_t *masks,
                              long long band_words, cudaStream_t s) {
    if (b->num_tiles == 0) return cudaSuccess;
    const RenderParams rp = make_params(o);
#define GS_BWD(T_, B_) \
    run_bwd<T_, B_>(b, order, ranges, vals, splat, colors, rp, stats, in_T, in_last, dL, grad2d, masks, band_words, s)
    GS_DISPATCH(o->tile, o->batch, GS_BWD)
#undef GS_BWD
}

// Band slots of the masks: the forward's bands of a whole tile, then those of
// the two halves of a heavy tile.
int render_band_slots(int tile) {
    switch (tile) {
    case 8: return 3 * (Threads<8>::NT / 32);
    case 16: return 3 * (Threads<16>::NT / 32);
    case 32: return 3 * (Threads<32>::NT / 32);
    default: return 3 * (Threads<32>::NT / 32);
    }
}

}  // namespace gs
