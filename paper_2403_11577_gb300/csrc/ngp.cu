// F(X | Theta) (Sec. III-C): the Instant-NGP multiresolution hash encoding of
// a Gaussian's centre followed by an MLP whose four heads give the Gaussian's
// colour, opacity, scale and rotation; forward and backward.
//
// Encoding: L <= 16 levels of 2 features, T = 2^log2_table entries per level.
// A point maps to p in [0, 1]^3 (clamped) through the bounding box; at level
// l its coordinates are q = p N_l, its cell c = min(floor(q), N_l - 1), and
// its two features are the trilinear interpolation of the cell's 8 vertices
// (weights from q - c).  A vertex v indexes the level's table densely,
// x + y (N_l + 1) + z (N_l + 1)^2, when the (N_l + 1)^3 vertices fit,
// otherwise by the spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861)
// mod 2^32 mod T.
// MLP: 2L -> 64 -> 64 -> 11 with ReLU after the hidden layers; heads
// rgb = sigmoid(o0..2), logit opacity o3, log scale o4..6, quaternion o7..10
// (the renderer's raw inputs).
// Parameters (theta, float): the L tables [L][T][2], then W1 [64][2L],
// b1 [64], W2 [64][64], b2 [64], W3 [11][64], b3 [11].
//
// The layers are dense contractions over tiles of 128 points and run on the
// 5th-generation tensor cores (tcgen05.mma, kind::f16 with bf16 operands,
// FP32 accumulators in tensor memory).  Every operand x is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi), and each product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi: the dropped A_lo B_lo term and the
// rounding of the low parts are below 2^-16 relative, so the layers keep
// close to FP32 accuracy.  Operands sit in shared memory as 8 x 8 core
// matrices (8 rows of 16 bytes, no swizzle).  One thread issues the MMAs and
// a commit to an mbarrier; every thread waits on it (bounded in time), and
// the epilogues read the accumulators with tcgen05.ld (warp w reads the 32
// rows of lane quarter w % 4, column half w / 4).
//
// Backward: per tile the forward is recomputed, dO = dL/do goes back through
// the heads, dH2 = dO W3, dH1 = dA2 W2 and dENC = dA1 W1 (dA = dH masked by
// the ReLU), and the table gradient is scattered with float2 atomics per
// (point, level, vertex), one float4 atomic where two x-neighbours of a cell
// are adjacent table entries.  The weight gradients are contractions over the
// points.  They accumulate in tensor memory over all tiles of a block as two
// stacked 128-row MMAs whose operands are the tile buffers read transposed
// (MN-major):
//   [H2 | dA2]^T [dO | H1 | ENC | 1]  ->  dW3^T, dW2, db2
//   [dA2 | dA1]^T [ENC | 1]           ->  dW1, db1
// and are added to d_theta once per block; db3 is a warp reduction.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gs {

namespace {

constexpr int kH = 64, kO = 11, kMaxLevels = 16;
constexpr int kTile = 128;     // points per tile: the MMA's M
constexpr int kThreads = 256;  // 8 warps
constexpr int kK1 = 32;        // encoding columns (2L, zero padded)
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound on every mbarrier wait

// Byte offsets of an MN-major operand: true when the descriptor's leading
// byte offset is the stride along M/N and its stride byte offset the stride
// along K, false for the reverse (the reading the kernels use).
constexpr bool kMnLboIsMn = false;

__device__ unsigned int g_ngp_fault;  // bit 0: an mbarrier wait ran out

struct NgpArgs {
    float lo[3], inv_ext[3];
    int L, D;            // levels, encoding width 2L
    uint32_t T, tmask;   // table entries (a power of two) and T - 1
    int res[kMaxLevels];
    int dense[kMaxLevels];
    long long w1;        // offset of W1 in theta; b1, W2, b2, W3, b3 follow
};

// Offsets, within the MLP block, of b1, W2, b2, W3, b3 and the block size.
__host__ __device__ constexpr int off_b1(int D) { return kH * D; }
__host__ __device__ constexpr int off_w2(int D) { return kH * D + kH; }
__host__ __device__ constexpr int off_b2(int D) { return kH * D + kH + kH * kH; }
__host__ __device__ constexpr int off_w3(int D) { return kH * D + 2 * kH + kH * kH; }
__host__ __device__ constexpr int off_b3(int D) { return kH * D + 2 * kH + kH * kH + kO * kH; }
__host__ __device__ constexpr int mlp_size(int D) { return kH * D + 2 * kH + kH * kH + kO * kH + kO; }

// The 8 vertices of a point's cell at level l: table slots and weights.
__device__ __forceinline__ void cell_taps(const NgpArgs &a, int l, float px, float py, float pz, uint32_t (&slot)[8],
                                          float (&w)[8]) {
    const float r = (float)a.res[l];
    const float qx = px * r, qy = py * r, qz = pz * r;
    const float cx = fminf(floorf(qx), r - 1.f), cy = fminf(floorf(qy), r - 1.f), cz = fminf(floorf(qz), r - 1.f);
    const float fx = qx - cx, fy = qy - cy, fz = qz - cz;
    const uint32_t ix = (uint32_t)cx, iy = (uint32_t)cy, iz = (uint32_t)cz;
    const uint32_t n1 = (uint32_t)a.res[l] + 1u;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const uint32_t dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const uint32_t vx = ix + dx, vy = iy + dy, vz = iz + dz;
        w[c] = ((dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy)) * (dz ? fz : 1.f - fz);
        slot[c] = a.dense[l] ? vx + vy * n1 + vz * n1 * n1
                             : ((vx * 1u) ^ (vy * 2654435761u) ^ (vz * 805459861u)) & a.tmask;
    }
}

__device__ __forceinline__ void unit_point(const NgpArgs &a, const float *__restrict__ X, long long i, float &px,
                                           float &py, float &pz) {
    px = fminf(fmaxf((X[3 * i] - a.lo[0]) * a.inv_ext[0], 0.f), 1.f);
    py = fminf(fmaxf((X[3 * i + 1] - a.lo[1]) * a.inv_ext[1], 0.f), 1.f);
    pz = fminf(fmaxf((X[3 * i + 2] - a.lo[2]) * a.inv_ext[2], 0.f), 1.f);
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

// ------------------------------------------------------------ tcgen05 helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (each >> 4 in 14 bits), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, each
// K-major (0) or MN-major (1), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier for at most kWaitNs; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// 32 lanes x 16 consecutive FP32 columns of tensor memory (waits for the load).
// Every lane of the warp executes it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// ------------------------------------------------------------ operands

// A bf16 matrix of R rows x C columns (C a multiple of 8) in shared memory,
// high and low parts at hi and lo: element (r, c) at byte
// (r / 8) (C / 8) 128 + (c / 8) 128 + (r % 8) 16 + (c % 8) 2.
struct Mat {
    unsigned char *hi, *lo;
    int C;
};

__device__ __forceinline__ int mat_off(int C, int r, int c) {
    return (r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2;
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &h, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void put(const Mat &m, int r, int c, float x) {
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    const int o = mat_off(m.C, r, c);
    *reinterpret_cast<__nv_bfloat16 *>(m.hi + o) = h;
    *reinterpret_cast<__nv_bfloat16 *>(m.lo + o) = l;
}

// Columns c, c + 1 (c even) of row r: one 4-byte store per part.
__device__ __forceinline__ void put2(const Mat &m, int r, int c, float x0, float x1) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(x0, h0, l0);
    split_bf16(x1, h1, l1);
    const int o = mat_off(m.C, r, c);
    *reinterpret_cast<uint32_t *>(m.hi + o) = pack2(h0, h1);
    *reinterpret_cast<uint32_t *>(m.lo + o) = pack2(l0, l1);
}

// Columns c0 .. c0 + 7 (c0 % 8 == 0) of row r: one 16-byte store per part.
__device__ __forceinline__ void put8(const Mat &m, int r, int c0, const float *x) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(x[2 * j], h0, l0);
        split_bf16(x[2 * j + 1], h1, l1);
        h[j] = pack2(h0, h1);
        l[j] = pack2(l0, l1);
    }
    const int o = mat_off(m.C, r, c0);
    *reinterpret_cast<uint4 *>(m.hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(m.lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// One MMA operand: descriptor fields of both parts and the start advance per
// 16 elements of K.
struct Op {
    uint32_t hi, lo, lbo, sbo, kstep;
};

// Rows are the MMA's M (or N) index, columns c0.. its K index.
__device__ __forceinline__ Op kmajor(const Mat &m, int c0) {
    const uint32_t off = (uint32_t)(c0 >> 3) * 128u;
    return {smem_addr(m.hi) + off, smem_addr(m.lo) + off, 128u, (uint32_t)(m.C >> 3) * 128u, 256u};
}

// Columns c0.. are the MMA's M (or N) index, rows (points) its K index.
__device__ __forceinline__ Op mnmajor(const Mat &m, int c0) {
    const uint32_t off = (uint32_t)(c0 >> 3) * 128u, kdir = (uint32_t)(m.C >> 3) * 128u, mndir = 128u;
    return {smem_addr(m.hi) + off, smem_addr(m.lo) + off, kMnLboIsMn ? mndir : kdir, kMnLboIsMn ? kdir : mndir,
            2u * kdir};
}

// D (+)= A B^T over ksteps x 16 of K with the three-term split product.
__device__ __forceinline__ void mma3(uint32_t d, const Op &A, const Op &B, int ksteps, uint32_t idesc, bool acc) {
    for (int s = 0; s < ksteps; s++) {
        const uint64_t ah = sdesc(A.hi + s * A.kstep, A.lbo, A.sbo), al = sdesc(A.lo + s * A.kstep, A.lbo, A.sbo);
        const uint64_t bh = sdesc(B.hi + s * B.kstep, B.lbo, B.sbo), bl = sdesc(B.lo + s * B.kstep, B.lbo, B.sbo);
        mma_bf16(d, ah, bh, idesc, (acc || s > 0) ? 1u : 0u);
        mma_bf16(d, ah, bl, idesc, 1u);
        mma_bf16(d, al, bh, idesc, 1u);
    }
}

// ------------------------------------------------------------ shared memory

// Byte size of one part of each matrix.
constexpr int kW1 = kH * kK1 * 2, kW2 = kH * kH * 2, kW3 = 16 * kH * 2;
constexpr int kFwdF = kTile * 96 * 2;           // [ENC (32) | H (64)]
constexpr int kBwdX = kTile * 192 * 2;          // [H2 | dA2 | dA1]
constexpr int kBwdY = kTile * 128 * 2;          // [dO (16) | H1 (64) | ENC (32) | 1 (16)]
constexpr int kBias = (kH + kH + 16 + 16) * 4;  // b1, b2, b3 (16), db3 (16)

constexpr size_t fwd_smem() { return 2 * (kW1 + kW2 + kW3 + kFwdF) + kBias + 64; }
constexpr size_t bwd_smem() { return 2 * (2 * (kW1 + kW2 + kW3) + kBwdX + kBwdY) + kBias + 64 + 4 * kTile; }
static_assert(bwd_smem() <= 227 * 1024, "backward shared memory");

struct Carve {
    unsigned char *p;
    __device__ Mat mat(int bytes, int C) {
        Mat m{p, p + bytes, C};
        p += 2 * bytes;
        return m;
    }
};

// Weights of the forward (B operands, rows = outputs) and, with the
// transposes, of the backward, as bf16 hi/lo parts from theta; biases FP32.
__device__ void stage_weights(const NgpArgs &a, const float *__restrict__ theta, const Mat &W1, const Mat &W2,
                              const Mat &W3, const Mat *W1t, const Mat *W2t, const Mat *W3t, float *bias) {
    const int D = a.D;
    const float *m = theta + a.w1;
    for (int e = threadIdx.x; e < kH * kK1; e += kThreads) {
        const int j = e / kK1, i = e % kK1;
        const float v = i < D ? m[j * D + i] : 0.f;
        put(W1, j, i, v);
        if (W1t) put(*W1t, i, j, v);
    }
    for (int e = threadIdx.x; e < kH * kH; e += kThreads) {
        const int j = e / kH, k = e % kH;
        const float v = m[off_w2(D) + e];
        put(W2, j, k, v);
        if (W2t) put(*W2t, k, j, v);
    }
    for (int e = threadIdx.x; e < 16 * kH; e += kThreads) {
        const int k = e / kH, j = e % kH;
        const float v = k < kO ? m[off_w3(D) + k * kH + j] : 0.f;
        put(W3, k, j, v);
        if (W3t) put(*W3t, j, k, v);
    }
    for (int e = threadIdx.x; e < kH; e += kThreads) {
        bias[e] = m[off_b1(D) + e];
        bias[kH + e] = m[off_b2(D) + e];
    }
    for (int e = threadIdx.x; e < 16; e += kThreads) bias[2 * kH + e] = (e < kO) ? m[off_b3(D) + e] : 0.f;
}

// Encoding of the tile's points into columns c0 + 2l, c0 + 2l + 1 of E
// (zero for points beyond n).  Thread t: point t % 128, levels t / 128 + 2k.
__device__ __forceinline__ void encode_tile(const NgpArgs &a, const float *__restrict__ theta,
                                            const float *__restrict__ X, long long n, long long base, const Mat &E,
                                            int c0) {
    const int p = threadIdx.x & (kTile - 1);
    const long long i = base + p;
    float px = 0.f, py = 0.f, pz = 0.f;
    const bool valid = i < n;
    if (valid) unit_point(a, X, i, px, py, pz);
#pragma unroll 2
    for (int l = threadIdx.x >> 7; l < a.L; l += 2) {
        float e0 = 0.f, e1 = 0.f;
        if (valid) {
            uint32_t slot[8];
            float w[8];
            cell_taps(a, l, px, py, pz, slot, w);
            const float2 *tab = reinterpret_cast<const float2 *>(theta) + (size_t)l * a.T;
            float2 v[8];
#pragma unroll
            for (int c = 0; c < 8; c++) v[c] = __ldg(tab + slot[c]);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                e0 = fmaf(w[c], v[c].x, e0);
                e1 = fmaf(w[c], v[c].y, e1);
            }
        }
        put2(E, p, c0 + 2 * l, e0, e1);
    }
}

// Thread role for reading an accumulator: row (point) and column half.
struct Lane {
    int row, half;
    uint32_t lane_base;  // tensor-memory lane field of the warp's quarter
};

__device__ __forceinline__ Lane lane_role() {
    const int w = threadIdx.x >> 5;
    return {32 * (w & 3) + (int)(threadIdx.x & 31), w >> 2, (uint32_t)(32 * (w & 3)) << 16};
}

// Hidden-layer epilogue: columns [32 half, 32 half + 32) of a 64-wide
// accumulator, + bias, ReLU, into columns c0.. of M; returns the ReLU mask.
__device__ __forceinline__ uint32_t epi_relu(uint32_t tacc, const Lane &ln, const float *bias, const Mat &M, int c0) {
    uint32_t mask = 0;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        float v[16];
        const int col = 32 * ln.half + 16 * g;
        tmem_ld16(tacc + ln.lane_base + (uint32_t)col, v);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            v[j] += bias[col + j];
            if (v[j] > 0.f) mask |= 1u << (16 * g + j);
            else v[j] = 0.f;
        }
        put8(M, ln.row, c0 + col, v);
        put8(M, ln.row, c0 + col + 8, v + 8);
    }
    return mask;
}

// Backward epilogue: the same columns of dH masked by the forward's ReLU.
__device__ __forceinline__ void epi_mask(uint32_t tacc, const Lane &ln, uint32_t mask, const Mat &M, int c0) {
#pragma unroll
    for (int g = 0; g < 2; g++) {
        float v[16];
        const int col = 32 * ln.half + 16 * g;
        tmem_ld16(tacc + ln.lane_base + (uint32_t)col, v);
#pragma unroll
        for (int j = 0; j < 16; j++)
            if (!((mask >> (16 * g + j)) & 1u)) v[j] = 0.f;
        put8(M, ln.row, c0 + col, v);
        put8(M, ln.row, c0 + col + 8, v + 8);
    }
}

struct Sync {
    uint32_t bar, phase;
    // Every thread waits until the issuing thread's MMAs are done; false (for
    // all threads) when any thread's wait ran out.
    __device__ bool wait_all() {
        const bool ok = mbar_wait(bar, phase);
        if (ok) phase ^= 1u;
        const bool bad = __syncthreads_or(!ok);
        fence_after_sync();
        return !bad;
    }
};

// The threads' shared-memory writes become visible to the tensor core, and
// earlier tensor-memory reads are ordered before the next MMAs.
__device__ __forceinline__ void publish() {
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t cols) {
    fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
    }
}

__device__ __forceinline__ void init_bar(uint32_t bar) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// After a timeout: record it and give the MMAs still in flight a bounded
// time to finish before the tensor memory is released.
__device__ __forceinline__ void on_timeout(const Sync &s) {
    if (threadIdx.x == 0) {
        atomicOr(&g_ngp_fault, 1u);
        mbar_wait(s.bar, s.phase);
    }
}

// Tensor-memory columns.
constexpr uint32_t kFwdCols = 256, kF_D1 = 0, kF_D2 = 64, kF_D3 = 128;
constexpr uint32_t kBwdCols = 512, kB_ACCA = 0, kB_ACCB = 128, kB_D1 = 192, kB_D2 = 256, kB_D3 = 320, kB_DH2 = 336,
                   kB_DH1 = 400, kB_DENC = 464;

// Two blocks per SM (2 x 256 tensor-memory columns).
__global__ void __launch_bounds__(kThreads, 2)
k_ngp_fwd(NgpArgs a, const float *__restrict__ theta, const float *__restrict__ X, long long n,
          float *__restrict__ rgb, float *__restrict__ logit_o, float *__restrict__ log_s, float *__restrict__ quat) {
    extern __shared__ __align__(1024) unsigned char smem[];
    Carve cv{smem};
    const Mat W1 = cv.mat(kW1, kK1), W2 = cv.mat(kW2, kH), W3 = cv.mat(kW3, kH), F = cv.mat(kFwdF, 96);
    float *bias = reinterpret_cast<float *>(cv.p);
    uint64_t *bar = reinterpret_cast<uint64_t *>(cv.p + kBias);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(cv.p + kBias + 16);
    stage_weights(a, theta, W1, W2, W3, nullptr, nullptr, nullptr, bias);
    // encoding columns 2L .. 31 stay zero
    const int pad = kK1 - a.D;
    for (int e = threadIdx.x; e < kTile * pad; e += kThreads) put(F, e / pad, a.D + e % pad, 0.f);
    Sync s{smem_addr(bar), 0u};
    init_bar(s.bar);
    tmem_alloc(tslot, kFwdCols);
    publish();
    fence_after_sync();
    const uint32_t tm = *tslot;
    const Lane ln = lane_role();
    const long long tiles = (n + kTile - 1) / kTile;
    bool ok = true;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long base = t * kTile;
        encode_tile(a, theta, X, n, base, F, 0);
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kF_D1, kmajor(F, 0), kmajor(W1, 0), kK1 / 16, idesc_bf16(128, 64, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        epi_relu(tm + kF_D1, ln, bias, F, 32);
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kF_D2, kmajor(F, 32), kmajor(W2, 0), kH / 16, idesc_bf16(128, 64, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        epi_relu(tm + kF_D2, ln, bias + kH, F, 32);  // H2 replaces H1 (layer 2 is done)
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kF_D3, kmajor(F, 32), kmajor(W3, 0), kH / 16, idesc_bf16(128, 16, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        if (ln.half == 0) {
            float o[16];
            tmem_ld16(tm + kF_D3 + ln.lane_base, o);
            const long long i = base + ln.row;
            if (i < n) {
                const float *b3 = bias + 2 * kH;
#pragma unroll
                for (int k = 0; k < 3; k++) rgb[3 * i + k] = sigmoidf(o[k] + b3[k]);
                logit_o[i] = o[3] + b3[3];
#pragma unroll
                for (int k = 0; k < 3; k++) log_s[3 * i + k] = o[4 + k] + b3[4 + k];
#pragma unroll
                for (int k = 0; k < 4; k++) quat[4 * i + k] = o[7 + k] + b3[7 + k];
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok) on_timeout(s);
    tmem_free(tm, kFwdCols);
}

__global__ void __launch_bounds__(kThreads, 1)
k_ngp_bwd(NgpArgs a, const float *__restrict__ theta, const float *__restrict__ X, long long n,
          const float *__restrict__ d_rgb, const float *__restrict__ d_logit_o, const float *__restrict__ d_log_s,
          const float *__restrict__ d_quat, float *__restrict__ d_theta) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int D = a.D;
    Carve cv{smem};
    const Mat W1 = cv.mat(kW1, kK1), W2 = cv.mat(kW2, kH), W3 = cv.mat(kW3, kH);
    const Mat W1t = cv.mat(kW1, kH), W2t = cv.mat(kW2, kH), W3t = cv.mat(kW3, 16);
    const Mat Xb = cv.mat(kBwdX, 192), Yb = cv.mat(kBwdY, 128);
    float *bias = reinterpret_cast<float *>(cv.p);
    float *db3 = bias + 2 * kH + 16;
    uint64_t *bar = reinterpret_cast<uint64_t *>(cv.p + kBias);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(cv.p + kBias + 16);
    unsigned int *live = reinterpret_cast<unsigned int *>(cv.p + kBias + 64);  // [128]: point has a gradient
    stage_weights(a, theta, W1, W2, W3, &W1t, &W2t, &W3t, bias);
    for (int e = threadIdx.x; e < 16; e += kThreads) db3[e] = 0.f;
    // Y columns 80 + 2L .. 111 stay zero, column 112 is one, 113 .. 127 zero
    for (int e = threadIdx.x; e < kTile * 48; e += kThreads) {
        const int r = e / 48, c = 80 + e % 48;
        if (c >= 80 + D) put(Yb, r, c, c == 112 ? 1.f : 0.f);
    }
    Sync s{smem_addr(bar), 0u};
    init_bar(s.bar);
    tmem_alloc(tslot, kBwdCols);
    publish();
    fence_after_sync();
    const uint32_t tm = *tslot;
    const Lane ln = lane_role();
    const long long tiles = (n + kTile - 1) / kTile;
    bool ok = true, started = false;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long base = t * kTile;
        const long long i = base + ln.row;
        encode_tile(a, theta, X, n, base, Yb, 80);
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_D1, kmajor(Yb, 80), kmajor(W1, 0), kK1 / 16, idesc_bf16(128, 64, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        const uint32_t mask1 = epi_relu(tm + kB_D1, ln, bias, Yb, 16);  // H1
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_D2, kmajor(Yb, 16), kmajor(W2, 0), kH / 16, idesc_bf16(128, 64, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        const uint32_t mask2 = epi_relu(tm + kB_D2, ln, bias + kH, Xb, 0);  // H2
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_D3, kmajor(Xb, 0), kmajor(W3, 0), kH / 16, idesc_bf16(128, 16, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        // heads: dO = dL/do (zero beyond the 11 outputs and for points beyond n)
        if (ln.half == 0) {
            float o[16], g[16];
            tmem_ld16(tm + kB_D3 + ln.lane_base, o);
#pragma unroll
            for (int k = 0; k < 16; k++) g[k] = 0.f;
            if (i < n) {
                const float *b3 = bias + 2 * kH;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float sg = sigmoidf(o[k] + b3[k]);
                    g[k] = d_rgb[3 * i + k] * sg * (1.f - sg);
                }
                g[3] = d_logit_o[i];
#pragma unroll
                for (int k = 0; k < 3; k++) g[4 + k] = d_log_s[3 * i + k];
#pragma unroll
                for (int k = 0; k < 4; k++) g[7 + k] = d_quat[4 * i + k];
            }
            put8(Yb, ln.row, 0, g);
            put8(Yb, ln.row, 8, g + 8);
            bool any = false;
#pragma unroll
            for (int k = 0; k < kO; k++) any |= g[k] != 0.f;
            live[ln.row] = any ? 1u : 0u;
#pragma unroll
            for (int k = 0; k < kO; k++) {
                float v = g[k];
#pragma unroll
                for (int sft = 16; sft > 0; sft >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sft);
                if ((threadIdx.x & 31) == 0) atomicAdd(db3 + k, v);
            }
        }
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_DH2, kmajor(Yb, 0), kmajor(W3t, 0), 1, idesc_bf16(128, 64, 0, 0), false);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        epi_mask(tm + kB_DH2, ln, mask2, Xb, 64);  // dA2
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_DH1, kmajor(Xb, 64), kmajor(W2t, 0), kH / 16, idesc_bf16(128, 64, 0, 0), false);
            // [H2 | dA2]^T [dO | H1 | ENC | 1]
            mma3(tm + kB_ACCA, mnmajor(Xb, 0), mnmajor(Yb, 0), kTile / 16, idesc_bf16(128, 128, 1, 1), started);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        epi_mask(tm + kB_DH1, ln, mask1, Xb, 128);  // dA1
        publish();
        if (threadIdx.x == 0) {
            fence_after_sync();
            mma3(tm + kB_DENC, kmajor(Xb, 128), kmajor(W1t, 0), kH / 16, idesc_bf16(128, 32, 0, 0), false);
            // [dA2 | dA1]^T [ENC | 1]
            mma3(tm + kB_ACCB, mnmajor(Xb, 64), mnmajor(Yb, 80), kTile / 16, idesc_bf16(128, 48, 1, 1), started);
            mma_commit(s.bar);
        }
        if (!(ok = s.wait_all())) break;
        started = true;
        const bool point_live = live[ln.row] != 0u;
        // encoding gradient into the tables: this thread's levels 8 half .. 8 half + 7
        // (a point without upstream gradient adds exact zeros: skipped)
        {
            float g[16];
            tmem_ld16(tm + kB_DENC + ln.lane_base + (uint32_t)(16 * ln.half), g);
            if (i < n && point_live) {
                float px, py, pz;
                unit_point(a, X, i, px, py, pz);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int l = 8 * ln.half + q;
                    if (l >= a.L) continue;
                    uint32_t slot[8];
                    float w[8];
                    cell_taps(a, l, px, py, pz, slot, w);
                    float2 *tab = reinterpret_cast<float2 *>(d_theta) + (size_t)l * a.T;
                    // corners c and c + 1 differ in x only; when the first slot is
                    // even the two entries form one aligned float4
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        const float2 v0 = make_float2(w[c] * g[2 * q], w[c] * g[2 * q + 1]);
                        const float2 v1 = make_float2(w[c + 1] * g[2 * q], w[c + 1] * g[2 * q + 1]);
                        if ((slot[c] & 1u) == 0u && slot[c + 1] == slot[c] + 1u) {
                            atomicAdd(reinterpret_cast<float4 *>(tab + slot[c]), make_float4(v0.x, v0.y, v1.x, v1.y));
                        } else {
                            atomicAdd(tab + slot[c], v0);
                            atomicAdd(tab + slot[c + 1], v1);
                        }
                    }
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok) {
        on_timeout(s);
        if (threadIdx.x == 0) atomicAdd(d_theta, __int_as_float(0x7fc00000));  // poison: the gradient is incomplete
    } else if (started) {
        // the block's weight gradients: this thread's row of the accumulators
        float *g1 = d_theta + a.w1;
        const int r = ln.row;
#pragma unroll 1
        for (int c0 = 64 * ln.half; c0 < 64 * ln.half + 64; c0 += 16) {
            float v[16];
            tmem_ld16(tm + kB_ACCA + ln.lane_base + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int c = c0 + j;
                if (r < 64) {
                    if (c < kO) atomicAdd(g1 + off_w3(D) + c * kH + r, v[j]);  // dW3[c][r]
                } else if (c >= 16 && c < 80) {
                    atomicAdd(g1 + off_w2(D) + (r - 64) * kH + (c - 16), v[j]);  // dW2[r - 64][c - 16]
                } else if (c == 112) {
                    atomicAdd(g1 + off_b2(D) + (r - 64), v[j]);  // db2[r - 64]
                }
            }
        }
        if (r >= 64) {  // uniform per warp (lane quarters 2 and 3)
            float v[16];
            tmem_ld16(tm + kB_ACCB + ln.lane_base + (uint32_t)(16 * ln.half), v);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int c = 16 * ln.half + j;
                if (c < D) atomicAdd(g1 + (r - 64) * D + c, v[j]);  // dW1[r - 64][c]
            }
            if (ln.half == 0) {
                tmem_ld16(tm + kB_ACCB + ln.lane_base + 32u, v);
                atomicAdd(g1 + off_b1(D) + (r - 64), v[0]);  // db1[r - 64]
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kO; k += kThreads) atomicAdd(g1 + off_b3(D) + k, db3[k]);
    }
    tmem_free(tm, kBwdCols);
}

}  // namespace

static bool ngp_args(const gs_ngp *c, NgpArgs *a) {
    if (!c || c->levels < 1 || c->levels > kMaxLevels || c->log2_table < 4 || c->log2_table > 26) return false;
    a->L = c->levels;
    a->D = 2 * c->levels;
    a->T = 1u << c->log2_table;
    a->tmask = a->T - 1u;
    for (int d = 0; d < 3; d++) {
        const float ext = c->aabb_max[d] - c->aabb_min[d];
        if (!(ext > 0.f) || !std::isfinite(ext)) return false;
        a->lo[d] = c->aabb_min[d];
        a->inv_ext[d] = 1.f / ext;
    }
    for (int l = 0; l < kMaxLevels; l++) {
        a->res[l] = l < c->levels ? c->res[l] : 1;
        if (l < c->levels && (c->res[l] < 1 || c->res[l] > (1 << 20))) return false;
        const double n1 = (double)a->res[l] + 1.0;
        a->dense[l] = n1 * n1 * n1 <= (double)a->T;
    }
    a->w1 = (long long)c->levels * a->T * 2;
    return true;
}

long long ngp_param_count(const gs_ngp *c) {
    NgpArgs a;
    return ngp_args(c, &a) ? a.w1 + mlp_size(a.D) : -1;
}

// Blocks: at most per_sm per SM, and no more than the tiles.
static cudaError_t ngp_grid(const void *kernel, size_t smem, long long n, int per_sm, int *grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long tiles = (n + kTile - 1) / kTile;
    *grid = (int)std::min<long long>(tiles, (long long)per_sm * sms);
    return cudaSuccess;
}

cudaError_t launch_ngp_fwd(const gs_ngp *c, const float *theta, const float *X, long long n, float *rgb,
                           float *logit_o, float *log_s, float *quat, cudaStream_t s) {
    NgpArgs a;
    if (!ngp_args(c, &a)) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    int grid = 0;
    cudaError_t e = ngp_grid((const void *)k_ngp_fwd, fwd_smem(), n, 2, &grid);
    if (e != cudaSuccess) return e;
    k_ngp_fwd<<<grid, kThreads, fwd_smem(), s>>>(a, theta, X, n, rgb, logit_o, log_s, quat);
    return cudaGetLastError();
}

cudaError_t launch_ngp_bwd(const gs_ngp *c, const float *theta, const float *X, long long n, const float *d_rgb,
                           const float *d_logit_o, const float *d_log_s, const float *d_quat, float *d_theta,
                           cudaStream_t s) {
    NgpArgs a;
    if (!ngp_args(c, &a)) return cudaErrorInvalidValue;
    if (n == 0) return cudaSuccess;
    int grid = 0;
    cudaError_t e = ngp_grid((const void *)k_ngp_bwd, bwd_smem(), n, 1, &grid);
    if (e != cudaSuccess) return e;
    k_ngp_bwd<<<grid, kThreads, bwd_smem(), s>>>(a, theta, X, n, d_rgb, d_logit_o, d_log_s, d_quat, d_theta);
    return cudaGetLastError();
}

cudaError_t ngp_fault(unsigned int *out) {
    unsigned int v = 0, z = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_ngp_fault, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ngp_fault, &z, sizeof(z));
    *out = v;
    return e;
}

}  // namespace gs
