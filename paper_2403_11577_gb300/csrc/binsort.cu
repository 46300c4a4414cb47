// Tile binning and depth ordering for Phi (Eq. 5).
//
// The pairs must end up ordered by (global tile, depth, Gaussian index):
// the order of the 64-bit key (global tile << 32) | float bits of the depth,
// value = Gaussian index within its scene, stable in record order.
// gs_bin_sort gets there in two cheap stages instead of one wide sort, with
// 32-bit keys throughout:
// 1. 4 LSD passes over the per-(frame, Gaussian) records keyed by the float
//    bits of their depth: a stable depth order of the records (ties keep
//    record order).  The first pass reads the depths directly and drops the
//    culled records (depth +inf, as gs_project writes for an empty
//    rectangle); it counts the rest, and the later passes and stage 2 visit
//    only those.  (A record with an empty rectangle and a finite depth is
//    sorted like the others and emits no pair.)
// 2. k_pair_count / k_pair_scan / k_pair_emit over the records in that
//    order: every record emits one pair per tile of its rectangle (emission
//    is cooperative: threads stride over the block's output range and find
//    their record by binary search).  With exact tiles (gs_opts.exact_tiles)
//    k_pair_count_exact / k_pair_emit_exact emit only the tiles of each
//    rectangle row that the record's ellipse can meet (spans.cuh).  The
//    pairs are thus already in (depth, record) order; their key is the
//    global tile alone.
// 3. LSD passes over the tile id (2 for up to 65,536 tiles): a stable sort
//    by tile keeps the depth order inside each tile, so the result is the
//    full-key order bit for bit, with a fraction of the traffic.
// 4. k_tile_ranges: [start, end) of every tile; k_tile_order: the tiles
//    sorted heavy-first for the render kernels.
// gs_bin_sort_noalloc sorts 64-bit full keys over all their bits instead
// (one stage, no record buffers).  gs_voxel_downsample (Sec. III-D) uses the
// same 64-bit passes to bin LiDAR points into voxels.
// Each radix pass: k_radix_hist (per-block digit counts) -> k_radix_colscan
// (per-digit prefix over blocks, digit totals) -> k_radix_scatter (stable:
// per-warp ranking in index order, the lanes of equal digit found by one
// ballot per digit bit; per-tile prefix over warps; staging in shared memory
// by digit; coalesced writes; the next tile's keys and values are loaded
// into registers while the current tile is staged and written); each block
// owns one contiguous chunk of the input.
// No kernel waits on another block; there are no spin loops.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "spans.cuh"

namespace gs {

namespace {

template <int NT>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *sh) {
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; w++) t += sh[w];
    return t;  // valid in thread 0
}

// perm (optional): the order in which records are visited; NULL = record order.
// live (optional): the entries of perm to visit (the records that survived
// culling in the record sort), else R.
__device__ __forceinline__ long long visited(long long R, const unsigned long long *live) {
    return live ? min(R, (long long)*live) : R;
}

__global__ void __launch_bounds__(kEmitThreads)
k_pair_count(const uint2 *__restrict__ rect, long long R, const unsigned long long *__restrict__ live,
             const uint32_t *__restrict__ perm, unsigned long long *__restrict__ sums) {
    __shared__ unsigned long long sh[kEmitThreads / 32];
    R = visited(R, live);
    const long long base = (long long)blockIdx.x * kEmitItems;
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < kEmitItems; i += kEmitThreads) {
        long long p = base + i;
        if (p < R) c += rect_count(rect[perm ? (long long)perm[p] : p]);
    }
    unsigned long long t = block_sum_u64<kEmitThreads>(c, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// Exclusive scan of n u64 values in place by one block of 1024 threads.
__device__ void block_exclusive_scan_u64(unsigned long long *a, long long n, unsigned long long *total) {
    __shared__ unsigned long long part[1024];
    const int T = blockDim.x;
    const long long per = (n + T - 1) / T;
    const long long lo = min((long long)threadIdx.x * per, n), hi = min(lo + per, n);
    unsigned long long s = 0;
    for (long long i = lo; i < hi; i++) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        unsigned long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - s;  // exclusive prefix of this thread's segment
    for (long long i = lo; i < hi; i++) {
        unsigned long long x = a[i];
        a[i] = run;
        run += x;
    }
    if (threadIdx.x == T - 1) *total = part[T - 1];
}

__global__ void __launch_bounds__(1024)
k_pair_scan(unsigned long long *__restrict__ sums, int nb, long long capacity, Stats *__restrict__ stats) {
    __shared__ unsigned long long total;
    block_exclusive_scan_u64(sums, nb, &total);
    __syncthreads();
    if (threadIdx.x == 0) {
        stats->raw_pairs = total;
        if (total > (unsigned long long)capacity) {
            stats->num_pairs = 0;
            atomicOr(&stats->status, (unsigned)GS_DEV_PAIR_OVERFLOW);
        } else {
            stats->num_pairs = total;
        }
    }
}

// Pairs of each emission block with exact tiles (as k_pair_count); also
// each record's pairs and non-empty rows, by sorted position, for the
// emission.
__global__ void __launch_bounds__(kEmitThreads)
k_pair_count_exact(const gs_frame *__restrict__ frames, int F, int T, float lmin, const uint2 *__restrict__ rect,
                   const float4 *__restrict__ splat, long long R, const unsigned long long *__restrict__ live,
                   const uint32_t *__restrict__ perm, unsigned long long *__restrict__ sums,
                   uint2 *__restrict__ rec_pairs) {
    __shared__ unsigned long long sh[kEmitThreads / 32];
    R = visited(R, live);
    const long long base = (long long)blockIdx.x * kEmitItems;
    if (base >= R) {  // past the live records: no pairs
        if (threadIdx.x == 0) sums[blockIdx.x] = 0ull;
        return;
    }
    constexpr int PER = kEmitItems / kEmitThreads;
    // the gathers of the thread's records are issued together (records i =
    // threadIdx.x + j * kEmitThreads, coalesced across the block)
    uint32_t r[PER];
    uint2 rc[PER];
    float4 s0[PER], s1[PER];
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const long long p = base + threadIdx.x + j * kEmitThreads;
        r[j] = p < R ? perm[p] : 0u;
    }
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const long long p = base + threadIdx.x + j * kEmitThreads;
        rc[j] = p < R ? rect[r[j]] : make_uint2(1u, 0u);
    }
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const bool any = rect_count(rc[j]) != 0u;
        s0[j] = any ? splat[2 * (long long)r[j]] : make_float4(0.f, 0.f, 0.f, 0.f);
        s1[j] = any ? splat[2 * (long long)r[j] + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    unsigned long long c = 0;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const long long p = base + threadIdx.x + j * kEmitThreads;
        if (p >= R) continue;
        uint32_t np = 0, ns = 0;  // pairs and non-empty rows of the record
        if (rect_count(rc[j]) != 0u) {
            const gs_frame &fr = frames[frame_of_record(frames, F, r[j])];
            const RowSpanner sp = make_spanner(s0[j], s1[j], lmin, rc[j], fr, T);
            const int rx0 = (int)(rc[j].x & 0xffffu), rx1 = (int)(rc[j].y & 0xffffu);
            for (int ty = (int)(rc[j].x >> 16); ty <= (int)(rc[j].y >> 16); ty++) {
                int lo, hi;
                row_span(sp, ty, rx0, rx1, fr, T, lo, hi);
                if (hi >= lo) {
                    np += (uint32_t)(hi - lo + 1);
                    ns++;
                }
            }
        }
        rec_pairs[p] = make_uint2(np, ns);
        c += np;
    }
    const unsigned long long t = block_sum_u64<kEmitThreads>(c, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// Emission with exact tiles (as k_pair_emit<uint32_t>).  A record's pairs
// are its rows' runs of tiles, each a segment (first pair, length, first
// tile, value); the block's segments are staged in shared memory in windows
// of kSegWindow, and the warps expand them into pairs 32 at a time.
constexpr int kSegWindow = 1024;  // 16 KB of segments: eight blocks fit on an SM

struct Segment {
    uint32_t off, len, tile0, val;  // off: first pair, relative to the block's first
};

struct EmitExactSmem {
    Segment seg[kSegWindow];
    unsigned long long wsum[kEmitThreads / 32];
    uint32_t ssum[kEmitThreads / 32];
    uint32_t nseg;
};

__global__ void __launch_bounds__(kEmitThreads)
k_pair_emit_exact(const gs_frame *__restrict__ frames, int F, int T, float lmin, const uint2 *__restrict__ rect,
                  const float4 *__restrict__ splat, long long R, const unsigned long long *__restrict__ live,
                  const uint32_t *__restrict__ perm, const unsigned long long *__restrict__ sums,
                  const uint2 *__restrict__ rec_pairs, const Stats *__restrict__ stats, uint32_t *__restrict__ keys,
                  uint32_t *__restrict__ vals) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EmitExactSmem &S = *reinterpret_cast<EmitExactSmem *>(smem_raw);
    if (stats->num_pairs == 0) return;  // nothing to emit, or overflow
    R = visited(R, live);
    const long long base = (long long)blockIdx.x * kEmitItems;
    if (base >= R) return;
    constexpr int PER = kEmitItems / kEmitThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this thread's records: pairs and non-empty rows (from the count)
    unsigned long long npairs = 0;
    uint32_t nsegs = 0;
    for (int j = 0; j < PER; j++) {
        const long long p = base + threadIdx.x * PER + j;
        if (p >= R) continue;
        const uint2 c = rec_pairs[p];
        npairs += c.x;
        nsegs += c.y;
    }
    // exclusive prefixes of pairs and segments over the block's threads
    unsigned long long pin = npairs;
    uint32_t sin = nsegs;
    for (int sft = 1; sft < 32; sft <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, pin, sft);
        const uint32_t u = __shfl_up_sync(0xffffffffu, sin, sft);
        if (lane >= sft) {
            pin += v;
            sin += u;
        }
    }
    if (lane == 31) {
        S.wsum[warp] = pin;
        S.ssum[warp] = sin;
    }
    __syncthreads();
    unsigned long long pre_p = 0;
    uint32_t pre_s = 0;
    for (int w = 0; w < warp; w++) {
        pre_p += S.wsum[w];
        pre_s += S.ssum[w];
    }
    const unsigned long long my_p = pre_p + pin - npairs;  // first pair of this thread's records
    const uint32_t my_s = pre_s + sin - nsegs;             // and first segment
    if (threadIdx.x == kEmitThreads - 1) S.nseg = pre_s + sin;
    __syncthreads();
    const uint32_t nseg_all = S.nseg;
    const unsigned long long gbase = sums[blockIdx.x], npairs_all = stats->num_pairs;
    for (uint32_t w0 = 0; w0 < nseg_all; w0 += kSegWindow) {
        const uint32_t w1 = min(nseg_all, w0 + (uint32_t)kSegWindow);
        // the owners write their segments that fall in [w0, w1)
        if (nsegs > 0 && my_s < w1 && my_s + nsegs > w0) {
            unsigned long long po = my_p;
            uint32_t si = my_s;
            for (int j = 0; j < PER && si < w1; j++) {
                const long long p = base + threadIdx.x * PER + j;
                if (p >= R || rec_pairs[p].y == 0u) continue;
                const long long r = (long long)perm[p];
                const uint2 rc = rect[r];
                const gs_frame &fr = frames[frame_of_record(frames, F, r)];
                const RowSpanner sp = make_spanner(splat[2 * r], splat[2 * r + 1], lmin, rc, fr, T);
                const int rx0 = (int)(rc.x & 0xffffu), rx1 = (int)(rc.y & 0xffffu);
                const uint32_t val = (uint32_t)(r - fr.record_offset);
                for (int ty = (int)(rc.x >> 16); ty <= (int)(rc.y >> 16) && si < w1; ty++) {
                    int a, b;
                    row_span(sp, ty, rx0, rx1, fr, T, a, b);
                    if (b < a) continue;
                    if (si >= w0)
                        S.seg[si - w0] = {(uint32_t)po, (uint32_t)(b - a + 1),
                                          (uint32_t)fr.tile_offset + (uint32_t)ty * (uint32_t)fr.tiles_x + (uint32_t)a,
                                          val};
                    po += (unsigned long long)(b - a + 1);
                    si++;
                }
            }
        }
        __syncthreads();
        const int n = (int)(w1 - w0);
        const uint32_t o_lo = S.seg[0].off, o_hi = S.seg[n - 1].off + S.seg[n - 1].len;
        // Each warp expands a contiguous run of 32-pair groups.  One binary
        // search finds the segment s0 holding the run's first pair; in every
        // group lane k then checks candidate s0 + 1 + k, whose start lies d
        // pairs after the group's first pair (segments are non-empty and in
        // pair order, so the starts within the next 32 pairs are exactly the
        // first candidates).  The starts with d < 32 form a bit mask, lane l's
        // segment is s0 plus the starts in (0, l], and the next group's s0
        // adds every start with d <= 32.
        constexpr int NW = kEmitThreads / 32;
        const uint32_t ngroups = (o_hi - o_lo + 31u) >> 5;
        const uint32_t per = (ngroups + NW - 1) / NW;
        const uint32_t g0 = min(ngroups, (uint32_t)warp * per), g1 = min(ngroups, g0 + per);
        int s0 = 0;
        if (g0 < g1) {
            const uint32_t o0 = o_lo + (g0 << 5);
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.seg[mid].off <= o0) lo = mid; else hi = mid - 1;
            }
            s0 = lo;
        }
        for (uint32_t g = g0; g < g1; g++) {
            const uint32_t o0 = o_lo + (g << 5);
            const int c = s0 + 1 + lane;
            const uint32_t d = c < n ? S.seg[c].off - o0 : 64u;
            const uint32_t starts = __reduce_or_sync(0xffffffffu, d < 32u ? 1u << d : 0u);
            const bool at32 = __any_sync(0xffffffffu, d == 32u);
            const int sl = s0 + __popc(starts & (0xffffffffu >> (31 - lane)));
            const uint32_t o = o0 + (uint32_t)lane;
            if (o < o_hi) {
                const Segment sg = S.seg[sl];
                if (gbase + o < npairs_all) {  // always true when the count agrees (same arithmetic)
                    keys[gbase + o] = sg.tile0 + (o - sg.off);
                    vals[gbase + o] = sg.val;
                }
            }
            s0 += __popc(starts) + (at32 ? 1 : 0);
        }
        __syncthreads();
    }
}

// Key of a pair: the global tile (K = uint32_t, pairs emitted in depth order)
// or (global tile << 32) | depth bits (K = unsigned long long, full key).
template <typename K>
__device__ __forceinline__ K pair_key(uint32_t tile, uint32_t depth_bits);
template <>
__device__ __forceinline__ uint32_t pair_key<uint32_t>(uint32_t tile, uint32_t) { return tile; }
template <>
__device__ __forceinline__ unsigned long long pair_key<unsigned long long>(uint32_t tile, uint32_t depth_bits) {
    return ((unsigned long long)tile << 32) | depth_bits;
}

// Global tile of a sorted key.
__device__ __forceinline__ uint32_t key_tile(uint32_t k) { return k; }
__device__ __forceinline__ uint32_t key_tile(unsigned long long k) { return (uint32_t)(k >> 32); }

template <typename K>
__global__ void __launch_bounds__(kEmitThreads)
k_pair_emit(const gs_frame *__restrict__ frames, int F, const uint2 *__restrict__ rect,
            const float *__restrict__ depth, long long R, const unsigned long long *__restrict__ live,
            const uint32_t *__restrict__ perm,
            const unsigned long long *__restrict__ sums, const Stats *__restrict__ stats, K *__restrict__ keys,
            uint32_t *__restrict__ vals) {
    __shared__ unsigned long long off[kEmitItems + 1];
    __shared__ uint32_t s_tile0[kEmitItems];   // global tile of the rect's first tile
    __shared__ uint32_t s_w[kEmitItems];       // rect width in tiles
    __shared__ uint32_t s_stride[kEmitItems];  // tiles_x of the frame
    __shared__ uint32_t s_bits[kEmitItems];
    __shared__ uint32_t s_val[kEmitItems];
    __shared__ unsigned long long wsum[kEmitThreads / 32];
    if (stats->num_pairs == 0) return;  // nothing to emit, or overflow
    R = visited(R, live);
    const long long base = (long long)blockIdx.x * kEmitItems;
    if (base >= R) return;
    constexpr int PER = kEmitItems / kEmitThreads;
    // counts of this thread's PER consecutive records
    unsigned long long c[PER];
    unsigned long long mine = 0;
    for (int j = 0; j < PER; j++) {
        const int i = threadIdx.x * PER + j;
        const long long p = base + i;
        c[j] = 0;
        if (p < R) {
            const long long r = perm ? (long long)perm[p] : p;
            uint2 rc = rect[r];
            c[j] = rect_count(rc);
            if (c[j]) {
                const int f = frame_of_record(frames, F, r);
                const gs_frame &fr = frames[f];
                const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
                s_tile0[i] = (uint32_t)fr.tile_offset + y0 * (uint32_t)fr.tiles_x + x0;
                s_w[i] = x1 - x0 + 1u;
                s_stride[i] = (uint32_t)fr.tiles_x;
                s_bits[i] = __float_as_uint(depth[r]);
                s_val[i] = (uint32_t)(r - fr.record_offset);
            }
        }
        mine += c[j];
    }
    // block exclusive scan of the per-thread totals (warp shuffles + warp sums)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = mine;
    for (int s = 1; s < 32; s <<= 1) {
        unsigned long long v = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long wpre = 0;
    for (int w = 0; w < warp; w++) wpre += wsum[w];
    unsigned long long run = wpre + incl - mine;
    for (int j = 0; j < PER; j++) {
        off[threadIdx.x * PER + j] = run;
        run += c[j];
    }
    if (threadIdx.x == kEmitThreads - 1) off[kEmitItems] = run;
    __syncthreads();
    const unsigned long long total = off[kEmitItems];
    const unsigned long long gbase = sums[blockIdx.x];
    for (unsigned long long o = threadIdx.x; o < total; o += kEmitThreads) {
        // record i with off[i] <= o < off[i+1] (records with 0 pairs are skipped)
        int lo = 0, hi = kEmitItems - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= o) lo = mid; else hi = mid - 1;
        }
        const uint32_t k = (uint32_t)(o - off[lo]);
        const uint32_t w = s_w[lo];
        const uint32_t tile = s_tile0[lo] + (k / w) * s_stride[lo] + (k % w);
        keys[gbase + o] = pair_key<K>(tile, s_bits[lo]);
        vals[gbase + o] = s_val[lo];
    }
}

// ------------------------------------------------------------ radix sort

struct Chunk { long long lo, hi; };

__device__ __forceinline__ Chunk sort_chunk(unsigned long long P, int nb, int b) {
    const long long tiles = (long long)((P + kSortTile - 1) / kSortTile);
    const long long per = (tiles + nb - 1) / nb;
    long long lo = min((long long)b * per * kSortTile, (long long)P);
    long long hi = min(lo + per * kSortTile, (long long)P);
    return {lo, hi};
}

// The input of a pass: key/value buffers, or (the first pass over the
// records) the records' depths, each keyed by its float bits (positive, so
// ordered like the depths) and valued by its index; a record of depth +inf
// (what gs_project writes for a culled record) is dropped there, so the
// later passes and the pair emission see only the records that can make
// pairs.
constexpr uint32_t kDropped = 0xffffffffu;       // value of a dropped record (indices are < 2^31)
constexpr uint32_t kCulledDepth = 0x7f800000u;   // +inf

template <typename K>
struct PassInput {
    const K *keys;
    const uint32_t *vals;
    const float *depth;   // non-null: read the records' depths instead
    const unsigned long long *count;  // items (device), or null: count_host
    long long count_host;
    __device__ __forceinline__ unsigned long long n() const {
        return count ? *count : (unsigned long long)count_host;
    }
    // key of item i; false if it is dropped
    __device__ __forceinline__ bool key(long long i, K &k) const {
        if (depth) {
            const uint32_t bits = __float_as_uint(depth[i]);
            k = (K)bits;
            return bits != kCulledDepth;
        }
        k = keys[i];
        return true;
    }
    // key and value of item i; a dropped item gets the value kDropped
    __device__ __forceinline__ void load(long long i, K &k, uint32_t &v) const {
        if (depth) {
            v = key(i, k) ? (uint32_t)i : kDropped;
        } else {
            k = keys[i];
            v = vals[i];
        }
    }
    __device__ __forceinline__ bool live(uint32_t v) const { return !depth || v != kDropped; }
};

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const PassInput<K> in, int shift, int nb, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kSortThreads / 32][kRadix];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const Chunk c = sort_chunk(in.n(), nb, blockIdx.x);
    for (long long i = c.lo + threadIdx.x; i < c.hi; i += kSortThreads) {
        K k;
        if (in.key(i, k)) atomicAdd(&h[warp][(uint32_t)(k >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t s = 0;
        for (int w = 0; w < kSortThreads / 32; w++) s += h[w][d];
        hist[(size_t)d * nb + blockIdx.x] = s;
    }
}

// Column scans of the digit-major count matrix hist[d * nb + b]: block d
// turns its column into exclusive prefixes over blocks and writes the digit's
// total; the scatter adds the exclusive prefix of the totals.  Counts fit in
// u32 (at most the pair capacity, checked on the host to be < 2^32).
constexpr int kColThreads = 512;  // >= the number of sort blocks

__global__ void __launch_bounds__(kColThreads)
k_radix_colscan(uint32_t *__restrict__ hist, int nb, uint32_t *__restrict__ totals) {
    __shared__ uint32_t wsum[kColThreads / 32];
    const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *col = hist + (size_t)d * nb;
    const uint32_t x = threadIdx.x < nb ? col[threadIdx.x] : 0u;
    uint32_t incl = x;
    for (int s = 1; s < 32; s <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
        if (lane >= s) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; w++) pre += wsum[w];
    if (threadIdx.x < nb) col[threadIdx.x] = pre + incl - x;
    if (threadIdx.x == kColThreads - 1) totals[d] = pre + incl;
}

constexpr int kWarps = kSortThreads / 32;

template <typename K>
struct ScatterSmem {
    K skey[kSortTile];
    uint32_t sval[kSortTile];
    uint32_t wcnt[kWarps][kRadix];   // per-warp digit counts, then exclusive prefix over warps
    uint32_t tcnt[kRadix];           // digit counts of the tile
    uint32_t tstart[kRadix];         // exclusive scan of tcnt
    uint32_t run[kRadix];            // next global position of each digit
    uint32_t wtot[kRadix / 32];
};

// ranges (optional, the last pass over tile keys): every tile's [start, end)
// in the output, found from the staged, sorted items (min/max atomics over
// the run boundaries; the ranges start at {UINT32_MAX, 0}).
// count_out (optional): the items written (the sum of the digit totals).
template <typename K>
__global__ void __launch_bounds__(kSortThreads, 2)
k_radix_scatter(const PassInput<K> in, K *__restrict__ kout, uint32_t *__restrict__ vout, int shift, int nb,
                const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals, uint2 *__restrict__ ranges,
                unsigned long long *__restrict__ count_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<K> &S = *reinterpret_cast<ScatterSmem<K> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Chunk c = sort_chunk(in.n(), nb, blockIdx.x);
    // run[d] = (items of digits < d) + (items of digit d in earlier blocks)
    if (threadIdx.x < kRadix) {
        const uint32_t x = totals[threadIdx.x];
        uint32_t incl = x;
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
            if (lane >= s) incl += y;
        }
        if (lane == 31) S.wtot[warp] = incl;
        S.run[threadIdx.x] = incl - x;
    }
    __syncthreads();
    if (threadIdx.x < kRadix) {
        uint32_t pre = 0;
        for (int w = 0; w < warp; w++) pre += S.wtot[w];
        S.run[threadIdx.x] += pre + hist[(size_t)threadIdx.x * nb + blockIdx.x];
        if (count_out && blockIdx.x == 0 && threadIdx.x == kRadix - 1)
            *count_out = (unsigned long long)S.run[threadIdx.x] + totals[threadIdx.x];
    }
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    // warp w owns items [w*32*ITEMS, (w+1)*32*ITEMS) of each tile, in index
    // order; the next tile's keys and values are loaded while this one is
    // staged and written
    K kn[kSortItems];
    uint32_t vn[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const long long idx = c.lo + (long long)warp * 32 * kSortItems + r * 32 + lane;
        kn[r] = K(0);
        vn[r] = kDropped;
        if (idx < c.hi) in.load(idx, kn[r], vn[r]);
    }
    for (long long t0 = c.lo; t0 < c.hi; t0 += kSortTile) {
        for (int i = lane; i < kRadix; i += 32) S.wcnt[warp][i] = 0;
        __syncwarp();
        K k[kSortItems];
        uint32_t v[kSortItems], dg[kSortItems], rk[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; r++) {
            k[r] = kn[r];
            v[r] = vn[r];
        }
#pragma unroll
        for (int r = 0; r < kSortItems; r++) {
            const long long idx = t0 + (long long)warp * 32 * kSortItems + r * 32 + lane;
            const bool valid = idx < c.hi && in.live(v[r]);
            const uint32_t d = (uint32_t)(k[r] >> shift) & (kRadix - 1);
            dg[r] = valid ? d : kRadix;  // kRadix marks an empty slot
            // lanes with the same digit: one ballot per digit bit (cheaper
            // than a match over up to 32 distinct digits)
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < kRadixBits; bit++) {
                const bool set = (d >> bit) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, set);
                peers &= set ? m : ~m;
            }
            const uint32_t before = (uint32_t)__popc(peers & lt_mask);
            uint32_t base = valid ? S.wcnt[warp][d] : 0u;
            __syncwarp();
            if (valid && before == 0) S.wcnt[warp][d] = base + (uint32_t)__popc(peers);
            __syncwarp();
            rk[r] = base + before;
        }
        if (t0 + kSortTile < c.hi) {
#pragma unroll
            for (int r = 0; r < kSortItems; r++) {
                const long long idx = t0 + kSortTile + (long long)warp * 32 * kSortItems + r * 32 + lane;
                kn[r] = K(0);
                vn[r] = kDropped;
                if (idx < c.hi) in.load(idx, kn[r], vn[r]);
            }
        }
        __syncthreads();
        // per digit: exclusive prefix over warps and the tile count
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
            uint32_t s = 0;
            for (int w = 0; w < kWarps; w++) {
                uint32_t x = S.wcnt[w][d];
                S.wcnt[w][d] = s;
                s += x;
            }
            S.tcnt[d] = s;
        }
        __syncthreads();
        // exclusive scan of tcnt over the 256 digits (8 warps of 32)
        if (threadIdx.x < kRadix) {
            const uint32_t x = S.tcnt[threadIdx.x];
            uint32_t incl = x;
            for (int s = 1; s < 32; s <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, incl, s);
                if (lane >= s) incl += y;
            }
            if (lane == 31) S.wtot[warp] = incl;
            S.tstart[threadIdx.x] = incl - x;
        }
        __syncthreads();
        if (threadIdx.x < kRadix) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; w++) pre += S.wtot[w];
            S.tstart[threadIdx.x] += pre;
        }
        __syncthreads();
        // stage by digit
#pragma unroll
        for (int r = 0; r < kSortItems; r++) {
            if (dg[r] < kRadix) {
                const uint32_t pos = S.tstart[dg[r]] + S.wcnt[warp][dg[r]] + rk[r];
                S.skey[pos] = k[r];
                S.sval[pos] = v[r];
            }
        }
        __syncthreads();
        const int n = (int)(S.tstart[kRadix - 1] + S.tcnt[kRadix - 1]);  // staged items
        for (int i = threadIdx.x; i < n; i += kSortThreads) {
            const K key = S.skey[i];
            const uint32_t d = (uint32_t)(key >> shift) & (kRadix - 1);
            const uint32_t pos = S.run[d] + (uint32_t)i - S.tstart[d];
            kout[pos] = key;
            vout[pos] = S.sval[i];
            if (ranges) {
                // within a digit's run the staged keys are in output order, so a
                // tile's items here are contiguous (the items next to a digit
                // run's edges have another digit, hence another key); its
                // neighbours across run edges were staged by other tiles or
                // blocks (min/max settle it)
                const uint32_t t = (uint32_t)key;
                if (i == 0 || S.skey[i - 1] != key) atomicMin(&ranges[t].x, pos);
                if (i + 1 == n || S.skey[i + 1] != key) atomicMax(&ranges[t].y, pos + 1u);
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) S.run[d] += S.tcnt[d];
        __syncthreads();
    }
}

template <typename K>
__global__ void k_tile_ranges(const K *__restrict__ keys, const unsigned long long *__restrict__ count,
                              uint2 *__restrict__ ranges) {
    const long long P = (long long)*count;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = key_tile(keys[i]);
        if (i == 0 || key_tile(keys[i - 1]) != t) ranges[t].x = (uint32_t)i;
        if (i == P - 1 || key_tile(keys[i + 1]) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

// Heavy-first processing order of the tiles (longest pair lists first), so
// that the long tiles start at once and the short ones fill in behind them
// instead of a few long ones running alone at the end.  Tiles are bucketed
// by floor(log2(list length)); the order within a bucket is arbitrary (it
// does not change any result: tiles are independent).
constexpr int kOrderBuckets = 33;

__global__ void __launch_bounds__(1024)
k_tile_order(uint2 *__restrict__ ranges, int T, uint32_t *__restrict__ order) {
    __shared__ uint32_t cnt[kOrderBuckets], base[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [](uint32_t len) { return len == 0 ? 0u : (uint32_t)(32 - __clz(len)); };  // 0..32
    const int lane = threadIdx.x & 31;
    // empty tiles come as {UINT32_MAX, 0} from the sort and leave as {0, 0};
    // warp-aggregated counting: one shared atomic per distinct bucket per warp
    for (int t0 = 0; t0 < T; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        uint2 rg = t < T ? ranges[t] : make_uint2(0u, 0u);
        if (t < T && rg.x > rg.y) {
            rg = make_uint2(0u, 0u);
            ranges[t] = rg;
        }
        const uint32_t k = t < T ? bucket(rg.y - rg.x) : (uint32_t)(kOrderBuckets + lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        if (t < T && (__ffs(peers) - 1) == lane) atomicAdd(&cnt[k], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int k = kOrderBuckets - 1; k >= 0; k--) {  // descending length
            base[k] = s;
            s += cnt[k];
        }
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        const uint32_t k = t < T ? bucket(ranges[t].y - ranges[t].x) : (uint32_t)(kOrderBuckets + lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        uint32_t start = 0;
        if (t < T && leader == lane) start = atomicAdd(&base[k], (uint32_t)__popc(peers));
        start = __shfl_sync(0xffffffffu, start, leader);
        if (t < T) order[start + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)t;
    }
}

}  // namespace

// Radix passes over the tile id (the depth order comes from the record sort).
int radix_passes(int num_tiles) {
    int tb = 0;
    while ((1ll << tb) < (long long)num_tiles) tb++;
    return (tb + kRadixBits - 1) / kRadixBits;
}

// Passes of a sort over the full 64-bit pair key (depth bits, then tile bits).
int full_key_passes(int num_tiles) { return radix_passes(num_tiles) + 32 / kRadixBits; }


namespace {

// One LSD pass (histogram, column scan, scatter) over the input's items;
// with `ranges`, the last pass over tile keys also finds the tile ranges.
template <typename K>
cudaError_t radix_pass(const PassInput<K> &in, K *kout, uint32_t *vout, int shift, int nb, uint32_t *hist,
                       cudaStream_t s, uint2 *ranges = nullptr, unsigned long long *count_out = nullptr) {
    uint32_t *totals = hist + (size_t)kRadix * nb;
    k_radix_hist<K><<<nb, kSortThreads, 0, s>>>(in, shift, nb, hist);
    k_radix_colscan<<<kRadix, kColThreads, 0, s>>>(hist, nb, totals);
    k_radix_scatter<K><<<nb, kSortThreads, sizeof(ScatterSmem<K>), s>>>(in, kout, vout, shift, nb, hist, totals,
                                                                        ranges, count_out);
    return cudaGetLastError();
}

// One pass over key/value buffers of *count items (count_host items if
// count is null).
template <typename K>
cudaError_t radix_pass(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, const unsigned long long *count,
                       int shift, int nb, uint32_t *hist, cudaStream_t s, long long count_host = 0,
                       uint2 *ranges = nullptr) {
    return radix_pass(PassInput<K>{kin, vin, nullptr, count, count_host}, kout, vout, shift, nb, hist, s, ranges);
}

__global__ void k_ranges_init(uint2 *__restrict__ ranges, int T) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) ranges[t] = make_uint2(0xffffffffu, 0u);
}

template <typename K>
cudaError_t scatter_smem_attr() {
    return cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ScatterSmem<K>));
}

}  // namespace

cudaError_t launch_bin_sort(const gs_batch *b, const gs_opts *o, const Layout &L, unsigned char *ws, cudaStream_t s,
                            int sms) {
    (void)sms;
    const bool exact = o->exact_tiles != 0;
    const float lmin = log2f(o->alpha_min);
    const float4 *splat = reinterpret_cast<const float4 *>(ws + L.splat);
    Stats *stats = reinterpret_cast<Stats *>(ws + L.stats);
    const uint2 *rect = reinterpret_cast<const uint2 *>(ws + L.rect);
    const float *depth = reinterpret_cast<const float *>(ws + L.depth);
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(ws + L.emit_sums);
    uint32_t *keys[2] = {reinterpret_cast<uint32_t *>(ws + L.keys[0]), reinterpret_cast<uint32_t *>(ws + L.keys[1])};
    uint32_t *vals[2] = {reinterpret_cast<uint32_t *>(ws + L.vals[0]), reinterpret_cast<uint32_t *>(ws + L.vals[1])};
    uint32_t *rkeys[2] = {reinterpret_cast<uint32_t *>(ws + L.rec_keys[0]),
                          reinterpret_cast<uint32_t *>(ws + L.rec_keys[1])};
    uint32_t *rvals[2] = {reinterpret_cast<uint32_t *>(ws + L.rec_vals[0]),
                          reinterpret_cast<uint32_t *>(ws + L.rec_vals[1])};
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.sort_hist);
    uint2 *ranges = reinterpret_cast<uint2 *>(ws + L.ranges);
    const long long R = b->num_records;
    cudaError_t e = scatter_smem_attr<uint32_t>();
    if (e == cudaSuccess && exact)
        e = cudaFuncSetAttribute(k_pair_emit_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(EmitExactSmem));
    if (e != cudaSuccess) return e;
    if (L.emit_blocks > 0) {
        // stage 1: stable depth order of the records (4 passes, ends in buffer 0;
        // the first reads the records' depths)
        unsigned long long *live = &stats->num_records;  // records that survive culling
        e = radix_pass(PassInput<uint32_t>{nullptr, nullptr, depth, nullptr, R}, rkeys[1], rvals[1], 0,
                       L.rec_sort_blocks, hist, s, nullptr, live);
        for (int p = 1; p < 4 && e == cudaSuccess; p++)
            e = radix_pass(rkeys[p & 1], rvals[p & 1], rkeys[(p + 1) & 1], rvals[(p + 1) & 1], live, 8 * p,
                           L.rec_sort_blocks, hist, s);
        if (e != cudaSuccess) return e;
        // stage 2: pairs emitted in that order (exact tiles or whole rectangles)
        if (exact) {
            uint2 *rec_pairs = reinterpret_cast<uint2 *>(ws + L.rec_pairs);
            k_pair_count_exact<<<L.emit_blocks, kEmitThreads, 0, s>>>(b->frames_dev, b->num_frames, b->tile, lmin,
                                                                      rect, splat, R, live, rvals[0], sums, rec_pairs);
            k_pair_scan<<<1, 1024, 0, s>>>(sums, L.emit_blocks, b->pair_capacity, stats);
            k_pair_emit_exact<<<L.emit_blocks, kEmitThreads, sizeof(EmitExactSmem), s>>>(
                b->frames_dev, b->num_frames, b->tile, lmin, rect, splat, R, live, rvals[0], sums, rec_pairs, stats,
                keys[L.first_buffer], vals[L.first_buffer]);
        } else {
            k_pair_count<<<L.emit_blocks, kEmitThreads, 0, s>>>(rect, R, live, rvals[0], sums);
            k_pair_scan<<<1, 1024, 0, s>>>(sums, L.emit_blocks, b->pair_capacity, stats);
            k_pair_emit<uint32_t><<<L.emit_blocks, kEmitThreads, 0, s>>>(b->frames_dev, b->num_frames, rect, depth,
                                                                         R, live, rvals[0], sums, stats,
                                                                         keys[L.first_buffer], vals[L.first_buffer]);
        }
    } else {
        e = cudaMemsetAsync(&stats->num_pairs, 0, sizeof(unsigned long long), s);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    // stage 3: stable passes over the tile bits only (end in buffer 0); the
    // last one also finds the tile ranges (empty tiles stay {UINT32_MAX, 0}
    // until k_tile_order writes them as {0, 0})
    if (e == cudaSuccess) {
        k_ranges_init<<<(b->num_tiles + 255) / 256, 256, 0, s>>>(ranges, b->num_tiles);
        e = cudaGetLastError();
    }
    int cur = L.first_buffer;
    for (int p = 0; p < L.passes && e == cudaSuccess; p++) {
        e = radix_pass(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], &stats->num_pairs, 8 * p, L.sort_blocks,
                       hist, s, 0, p == L.passes - 1 ? ranges : nullptr);
        cur ^= 1;
    }
    if (e == cudaSuccess && L.passes == 0) {  // a single tile: no pass, its range is every pair
        k_tile_ranges<uint32_t><<<1216, 256, 0, s>>>(keys[0], &stats->num_pairs, ranges);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    k_tile_order<<<1, 1024, 0, s>>>(ranges, b->num_tiles, reinterpret_cast<uint32_t *>(ws + L.order));
    return cudaGetLastError();
}

// ---------------------------------------------------- voxel downsampling
//
// Sec. III-D: one point per occupied voxel of edge v, the point of smallest
// index.  A point's voxel is (floor(x/v), floor(y/v), floor(z/v)), the
// quotients in float32 (IEEE division); the three coordinates, biased by
// 2^20, are packed into 21 bits each.  A stable LSD sort of (key, index)
// over index-ordered input puts every voxel's smallest index first; that
// point is flagged, and the flags are compacted in index order.  Points with
// a non-finite coordinate or a voxel coordinate outside (-2^20, 2^20) get
// the all-ones key, which sorts last and is never flagged.

namespace {

constexpr long long kVoxLimit = 1ll << 20;
constexpr int kVoxItems = 1024;  // flags per compaction block

__global__ void k_set_count(unsigned long long *c, long long n) { *c = (unsigned long long)n; }

__global__ void k_voxel_keys(const float *__restrict__ X, long long n, float v, unsigned long long *__restrict__ keys,
                             uint32_t *__restrict__ vals) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long key = 0;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float q = floorf(__fdiv_rn(X[3 * i + a], v));
        ok = ok && isfinite(q) && fabsf(q) < (float)kVoxLimit;
        key = (key << 21) | (ok ? (unsigned long long)((long long)q + kVoxLimit) : 0ull);
    }
    keys[i] = ok ? key : ~0ull;
    vals[i] = (uint32_t)i;
}

// flag[point] = 1 for the first (smallest index) point of each voxel
__global__ void k_voxel_first(const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ vals,
                              long long n, uint32_t *__restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long k = keys[i];
    flag[vals[i]] = (k != ~0ull && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

__global__ void __launch_bounds__(kEmitThreads)
k_flag_count(const uint32_t *__restrict__ flag, long long n, unsigned long long *__restrict__ sums) {
    __shared__ unsigned long long sh[kEmitThreads / 32];
    const long long base = (long long)blockIdx.x * kVoxItems;
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < kVoxItems; i += kEmitThreads)
        if (base + i < n) c += flag[base + i];
    const unsigned long long t = block_sum_u64<kEmitThreads>(c, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024)
k_flag_scan(unsigned long long *__restrict__ sums, int nb, unsigned long long *__restrict__ total) {
    block_exclusive_scan_u64(sums, nb, total);
}

// kept indices in ascending order: block b's flags go to sums[b] + the
// exclusive count within the block (each thread owns 4 consecutive flags)
__global__ void __launch_bounds__(kEmitThreads)
k_flag_emit(const uint32_t *__restrict__ flag, long long n, const unsigned long long *__restrict__ sums,
            int32_t *__restrict__ out) {
    __shared__ unsigned long long wsum[kEmitThreads / 32];
    constexpr int PER = kVoxItems / kEmitThreads;
    const long long base = (long long)blockIdx.x * kVoxItems + (long long)threadIdx.x * PER;
    uint32_t f[PER];
    unsigned long long mine = 0;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        f[j] = base + j < n ? flag[base + j] : 0u;
        mine += f[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = mine;
    for (int s2 = 1; s2 < 32; s2 <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, s2);
        if (lane >= s2) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned long long pos = sums[blockIdx.x] + incl - mine;
    for (int w = 0; w < warp; w++) pos += wsum[w];
#pragma unroll
    for (int j = 0; j < PER; j++)
        if (f[j]) out[pos++] = (int32_t)(base + j);
}

}  // namespace

size_t voxel_scratch_bytes(long long n, int *sort_blocks) {
    const long long st = (n + kSortTile - 1) / kSortTile;
    const int nb = (int)std::max(1ll, std::min(st, 304ll));
    if (sort_blocks) *sort_blocks = nb;
    const long long fb = (n + kVoxItems - 1) / kVoxItems;
    return align256((size_t)n * 8) * 2 + align256((size_t)n * 4) * 3 + align256((size_t)kRadix * (nb + 1) * 4) +
           align256((size_t)std::max(fb, 1ll) * 8) + 256;
}

cudaError_t launch_voxel(const float *X, long long n, float v, int32_t *out_index, unsigned long long *out_count,
                         unsigned char *scratch, cudaStream_t s) {
    int nb = 1;
    voxel_scratch_bytes(n, &nb);
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char *p = scratch + o; o += align256(bytes); return p; };
    unsigned long long *kb[2] = {(unsigned long long *)take((size_t)n * 8), (unsigned long long *)take((size_t)n * 8)};
    uint32_t *vb[2] = {(uint32_t *)take((size_t)n * 4), (uint32_t *)take((size_t)n * 4)};
    uint32_t *flag = (uint32_t *)take((size_t)n * 4);
    uint32_t *hist = (uint32_t *)take((size_t)kRadix * (nb + 1) * 4);
    const long long fb = (n + kVoxItems - 1) / kVoxItems;
    unsigned long long *sums = (unsigned long long *)take((size_t)std::max(fb, 1ll) * 8);
    unsigned long long *count = (unsigned long long *)take(8);
    if (n == 0) return cudaMemsetAsync(out_count, 0, 8, s);
    cudaError_t e = scatter_smem_attr<unsigned long long>();
    if (e != cudaSuccess) return e;
    k_set_count<<<1, 1, 0, s>>>(count, n);
    const int g = (int)((n + 255) / 256);
    k_voxel_keys<<<g, 256, 0, s>>>(X, n, v, kb[0], vb[0]);
    for (int p = 0; p < 8 && e == cudaSuccess; p++)  // 63 key bits
        e = radix_pass(kb[p & 1], vb[p & 1], kb[(p + 1) & 1], vb[(p + 1) & 1], count, 8 * p, nb, hist, s);
    if (e != cudaSuccess) return e;
    k_voxel_first<<<g, 256, 0, s>>>(kb[0], vb[0], n, flag);
    k_flag_count<<<(int)fb, kEmitThreads, 0, s>>>(flag, n, sums);
    k_flag_scan<<<1, 1024, 0, s>>>(sums, (int)fb, out_count);
    k_flag_emit<<<(int)fb, kEmitThreads, 0, s>>>(flag, n, sums, out_index);
    return cudaGetLastError();
}

}  // namespace gs

// ------------------------------------------------- allocation-free variant
//
// gs_bin_sort_noalloc: the same kernels as gs_bin_sort, with the caller's
// rect/depth as inputs and the caller's keys/vals/ranges as outputs; the
// scratch (counters, emission sums, radix histograms and the second key/value
// buffer of the ping-pong) lives in the fixed file-scope array below instead
// of a caller-allocated workspace.

namespace gs {

constexpr long long kNoAllocMaxPairs = 1ll << 20;
constexpr long long kNoAllocMaxRecords = 1ll << 22;
constexpr int kNoAllocSortBlocks = (int)(kNoAllocMaxPairs / kSortTile);  // 256

struct NoAllocScratch {
    Stats stats;
    unsigned long long alt_keys[kNoAllocMaxPairs];
    uint32_t alt_vals[kNoAllocMaxPairs];
    unsigned long long emit_sums[kNoAllocMaxRecords / kEmitItems];
    uint32_t hist[kRadix * (kNoAllocSortBlocks + 1)];  // counts, then digit totals
};

// The size the header documents (12.9 MB).
static_assert(sizeof(NoAllocScratch) == 12878912, "update the documented scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {

constexpr int kMaxDevices = 64;
// Per-device cache of the array's device address.  Host threads may call
// concurrently: a lookup is idempotent (every thread finds the same address),
// so racing first calls only repeat it, and the atomics make the publication
// itself well defined.
std::atomic<void *> g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in for it).
cudaError_t noalloc_scratch(NoAllocScratch **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
    *out = reinterpret_cast<NoAllocScratch *>(p);
    return cudaSuccess;
}

// Rectangles come from the caller here: a non-empty one must lie within its
// frame's tiles (x1 < tiles_x, y1 < tiles_y), else its pairs would name
// tiles of the next tile row or frame, or none at all.  Counts the offenders
// into st->reserved (zeroed before the call).
__global__ void k_noalloc_check_rects(const gs_frame *__restrict__ frames, int F, const uint2 *__restrict__ rect,
                                      long long R, Stats *__restrict__ st) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (r < R) {
        const uint2 rc = rect[r];
        if (rect_count(rc)) {
            const gs_frame &fr = frames[frame_of_record(frames, F, r)];
            bad = (rc.y & 0xffffu) >= (uint32_t)fr.tiles_x || (rc.y >> 16) >= (uint32_t)fr.tiles_y;
        }
    }
    const unsigned n = __popc(__ballot_sync(0xffffffffu, bad));
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&st->reserved, n);
}

// After the pair scan: with any rectangle outside its frame the call writes
// no pair (as after an overflow) and reports UINT64_MAX pairs requested.
__global__ void k_noalloc_gate(Stats *__restrict__ st) {
    if (st->reserved) {
        st->num_pairs = 0;
        st->raw_pairs = ~0ull;
    }
}

__global__ void k_noalloc_counts(const Stats *__restrict__ st, unsigned long long *__restrict__ out) {
    out[0] = st->num_pairs;
    out[1] = st->raw_pairs;
}

}  // namespace

}  // namespace gs

extern "C" gs_status gs_bin_sort_noalloc(const gs_batch *b, const gs_opts *o, const uint32_t *rect,
                                         const float *depth, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                                         uint64_t *out_pairs, void *stream) {
    using namespace gs;
    if (!b || !o || !b->frames_dev || b->num_frames <= 0 || b->num_tiles <= 0 || o->tile != b->tile || !keys ||
        !vals || !ranges || !out_pairs || (b->num_records > 0 && (!rect || !depth)))
        return GS_ERR_INVALID_ARG;
    // the kernels read rect and write ranges as uint2 and keys as uint64
    auto mis = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; };
    if (mis(rect, 8) || mis(ranges, 8) || mis(keys, 8) || mis(out_pairs, 8) || mis(depth, 4) || mis(vals, 4))
        return GS_ERR_INVALID_ARG;
    if (o->exact_tiles != 0) return GS_ERR_UNSUPPORTED;  // only rectangles are passed in
    if (b->pair_capacity > kNoAllocMaxPairs || b->num_records > kNoAllocMaxRecords) return GS_ERR_CAPACITY;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    NoAllocScratch *sc = nullptr;
    if (noalloc_scratch(&sc) != cudaSuccess) return GS_ERR_CUDA;
    const int emit_blocks = (int)((b->num_records + kEmitItems - 1) / kEmitItems);
    const long long st = (b->pair_capacity + kSortTile - 1) / kSortTile;
    const int sort_blocks = (int)std::max(1ll, std::min(st, (long long)kNoAllocSortBlocks));
    const int passes = full_key_passes(b->num_tiles);
    const uint2 *r2 = reinterpret_cast<const uint2 *>(rect);
    unsigned long long *kb[2] = {reinterpret_cast<unsigned long long *>(keys), sc->alt_keys};
    uint32_t *vb[2] = {vals, sc->alt_vals};
    int cur = passes & 1;  // the last pass ends in the caller's buffers
    cudaError_t e = cudaMemsetAsync(&sc->stats, 0, sizeof(Stats), s);  // counters start at zero
    if (e == cudaSuccess && emit_blocks > 0) {
        k_noalloc_check_rects<<<(unsigned)((b->num_records + 255) / 256), 256, 0, s>>>(
            b->frames_dev, b->num_frames, r2, b->num_records, &sc->stats);
        k_pair_count<<<emit_blocks, kEmitThreads, 0, s>>>(r2, b->num_records, nullptr, nullptr, sc->emit_sums);
        k_pair_scan<<<1, 1024, 0, s>>>(sc->emit_sums, emit_blocks, b->pair_capacity, &sc->stats);
        k_noalloc_gate<<<1, 1, 0, s>>>(&sc->stats);
        k_pair_emit<unsigned long long><<<emit_blocks, kEmitThreads, 0, s>>>(
            b->frames_dev, b->num_frames, r2, depth, b->num_records, nullptr, nullptr, sc->emit_sums, &sc->stats, kb[cur],
            vb[cur]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scatter_smem_attr<unsigned long long>();
    for (int p = 0; e == cudaSuccess && p < passes; p++) {
        e = radix_pass(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], &sc->stats.num_pairs, p * kRadixBits,
                       sort_blocks, sc->hist, s);
        cur ^= 1;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)b->num_tiles, s);
    if (e == cudaSuccess) {
        k_tile_ranges<unsigned long long><<<1216, 256, 0, s>>>(kb[0], &sc->stats.num_pairs,
                                                               reinterpret_cast<uint2 *>(ranges));
        k_noalloc_counts<<<1, 1, 0, s>>>(&sc->stats, reinterpret_cast<unsigned long long *>(out_pairs));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
