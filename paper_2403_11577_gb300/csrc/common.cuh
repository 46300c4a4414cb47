// Internal definitions shared by the CUDA translation units of
// libgs3dcalib.so (workspace layout, frame lookup, small device helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs3dcalib.h"

namespace gs {

constexpr int kPose32Stride = 32;   // floats per frame: R_cw hi[9], c_hi[3], c_lo[3], pad, R_cw lo[9], pad[7]
constexpr int kPoseRlo = 16;        // offset of R_cw's low parts within a frame's pose32
constexpr int kPose64Stride = 32;   // doubles per frame, see pose.cu
constexpr int kEmitItems = 1024;    // records per pair-emission block
constexpr int kEmitThreads = 256;
constexpr int kSortThreads = 512;   // radix sort block
constexpr int kSortItems = 8;       // keys per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kProjThreads = 128;
constexpr int kLossBlocks = 608;
constexpr int kLossThreads = 256;
constexpr int kMaxFrames = 1024;    // frames per batch

// Workspace counters; the head of the workspace.
struct Stats {
    unsigned int status;
    unsigned int reserved;
    unsigned long long num_pairs;   // valid pairs (0 after an overflow)
    unsigned long long eval_fwd;
    unsigned long long eval_bwd;
    unsigned long long raw_pairs;   // pairs requested before the capacity check
    unsigned long long num_records; // records that survive culling (count of the record sort)
    unsigned long long pad[2];
};

struct Layout {
    size_t stats, pose32, pose64, rect, depth, splat, grad2d, keys[2], vals[2], rec_keys[2], rec_vals[2], ranges,
        order, emit_sums, rec_pairs, band_masks, sort_hist, twist_part, twist_mid, twist_frame, loss_part, photo_maps, photo_part, total;
    int emit_blocks;     // blocks of the pair count / emit kernels
    int sort_blocks;     // blocks of the radix passes over pairs
    int rec_sort_blocks; // blocks of the radix passes over records
    int twist_parts;     // twist partials per frame (one per warp of the projection backward)
    int passes;          // radix passes over the tile bits of the pairs
    int first_buffer;    // buffer the emission writes (the last pass ends in 0)
    long long band_words; // words per band slot of the render's composited-entry masks
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int radix_passes(int num_tiles);
int render_band_slots(int tile);
int full_key_passes(int num_tiles);
bool make_layout(const gs_batch *b, Layout *L);

// ------------------------------------------------------------ device side

// Frame owning global tile t (binary search over tile offsets).
__device__ __forceinline__ int frame_of_tile(const gs_frame *fr, int F, int t) {
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fr[mid].tile_offset <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Frame owning record r.
__device__ __forceinline__ int frame_of_record(const gs_frame *fr, int F, long long r) {
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fr[mid].record_offset <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Error-free transformations in float (never contracted into FMAs): a + b =
// s + e exactly (two_sum), and a * b = p + e exactly (two_prod).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tiles of a packed rectangle (x0 | y0 << 16, x1 | y1 << 16), 0 if empty.
__device__ __forceinline__ uint32_t rect_count(uint2 rc) {
    uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu, y1 = rc.y >> 16;
    if (x0 > x1 || y0 > y1) return 0u;
    return (x1 - x0 + 1u) * (y1 - y0 + 1u);
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

}  // namespace gs
