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
constexpr unsigned long long kWaitNs = 1000000000ull;  // default bound of the waits; the drain wait's bound

// Byte offsets of an MN-major operand: true when the descriptor's leading
// byte offset is the stride along M/N and its stride byte offset the stride
// along K, false for the reverse (the reading the kernels use).
constexpr bool kMnLboIsMn = false;

__device__ unsigned int g_ngp_fault;  // bit 0: an mbarrier wait ran out
// Bound, in ns, on the waits for the tensor cores' MMAs (gs_ngp_set_wait_limit);
// 0: a wait gives up as soon as one non-blocking test finds its phase open.
__device__ unsigned long long g_ngp_wait_ns = kWaitNs;

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

// Wait for phase `parity` of the mbarrier for at most limit_ns; false on
// timeout.  With limit 0 one non-blocking test decides.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
    if (limit_ns == 0) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    }
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
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// After a timeout: the wait for the MMAs still in flight before the tensor
// memory is released (always the fixed one-second bound).
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) { return mbar_wait(bar, parity, kWaitNs); }

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
constexpr int kBias = (kH + kH + 16 + 16) * 4;  // b1, b2, b3 (16), db3 (16)

constexpr size_t fwd_smem() { return 2 * (kW1 + kW2 + kW3 + kFwdF) + kBias + 64; }

struct Carve {
    unsigned char *p;
    __device__ Mat mat(int bytes, int C) {
        Mat m{p, p + bytes, C};
        p += 2 * bytes;
        return m;
    }
};

// Weights (B operands, rows = outputs; the backward reads them MN-major as
// their transposes) as bf16 hi/lo parts from theta; biases in FP32.
__device__ void stage_weights(const NgpArgs &a, const float *__restrict__ theta, const Mat &W1, const Mat &W2,
                              const Mat &W3, float *bias) {
    const int D = a.D, nt = (int)blockDim.x;
    const float *m = theta + a.w1;
    for (int e = threadIdx.x; e < kH * kK1; e += nt) {
        const int j = e / kK1, i = e % kK1;
        put(W1, j, i, i < D ? m[j * D + i] : 0.f);
    }
    for (int e = threadIdx.x; e < kH * kH; e += nt) put(W2, e / kH, e % kH, m[off_w2(D) + e]);
    for (int e = threadIdx.x; e < 16 * kH; e += nt) {
        const int k = e / kH, j = e % kH;
        put(W3, k, j, k < kO ? m[off_w3(D) + k * kH + j] : 0.f);
    }
    for (int e = threadIdx.x; e < kH; e += nt) {
        bias[e] = m[off_b1(D) + e];
        bias[kH + e] = m[off_b2(D) + e];
    }
    for (int e = threadIdx.x; e < 16; e += nt) bias[2 * kH + e] = (e < kO) ? m[off_b3(D) + e] : 0.f;
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
    unsigned long long limit_ns;  // the settable bound on a wait for the MMAs, read once per kernel
    // Every thread waits until the issuing thread's MMAs are done; false (for
    // all threads) when any thread's wait ran out.
    __device__ bool wait_all() {
        const bool ok = mbar_wait(bar, phase, limit_ns);
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
        mbar_drain(s.bar, s.phase);
    }
}

// Tensor-memory columns.
constexpr uint32_t kFwdCols = 256, kF_D1 = 0, kF_D2 = 64, kF_D3 = 128;

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
    stage_weights(a, theta, W1, W2, W3, bias);
    // encoding columns 2L .. 31 stay zero
    const int pad = kK1 - a.D;
    for (int e = threadIdx.x; e < kTile * pad; e += kThreads) put(F, e / pad, a.D + e % pad, 0.f);
    Sync s{smem_addr(bar), 0u, *(volatile unsigned long long *)&g_ngp_wait_ns};
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

// ------------------------------------------------------------ backward

// The backward block: 8 consumer warps (warps 0-7) run the MMA chain of tile
// k while 4 producer warps (warps 8-11, one per tensor-memory lane quarter)
// gather the encoding of tile k + 1 into the other encoding buffer and
// scatter the table gradient of tile k - 1 from the other dENC columns.
// The roles meet once per tile at a block barrier; inside the chain the
// consumers synchronise among themselves (named barrier 1).
constexpr int kBwdThreads = 384, kConsumers = 256;
// Table-gradient levels the consumers add for their own tile (after the last
// MMA round, where they would otherwise wait for the producers); the
// producers add the rest.
constexpr int kConsumerLevels = 4;
constexpr int kBwdX = kTile * 128 * 2;  // [H2, later dA1 (64) | dA2 (64)]
constexpr int kBwdY = kTile * 96 * 2;   // [dO (16) | H1 (64) | 1 (16)]
constexpr int kBwdE = kTile * 48 * 2;   // [ENC (32) | 1 (16)], two of them
constexpr size_t bwd_smem() {
    return 2 * (kW1 + kW2 + kW3 + kBwdX + kBwdY + 2 * kBwdE) + kBias + 64 + 2 * 4 * kTile;
}
static_assert(bwd_smem() <= 227 * 1024, "backward shared memory");

// Tensor-memory columns of the backward (dENC double-buffered).
constexpr uint32_t kB_ACCA = 0, kB_ACCB = 128, kB_T1 = 192, kB_T2 = 256, kB_DENC = 320;

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void consumer_publish() {
    fence_async_smem();
    fence_before_sync();
    consumer_sync();
}

// The consumers wait for the issuing thread's MMAs; a timeout in any of them
// sets *abort (read by all consumers after their barrier).
__device__ __forceinline__ bool consumer_wait(Sync &s, volatile int *abort) {
    const bool ok = mbar_wait(s.bar, s.phase, s.limit_ns);
    if (ok) s.phase ^= 1u;
    else *abort = 1;
    consumer_sync();
    fence_after_sync();
    return *abort == 0;
}

// Producer: the encoding of the tile's points (thread pt: point pt, every
// level) into columns 2l, 2l + 1 of E.
__device__ __forceinline__ void produce_encoding(const NgpArgs &a, const float *__restrict__ theta,
                                                 const float *__restrict__ X, long long n, long long base,
                                                 const Mat &E, int pt) {
    const long long i = base + pt;
    const bool valid = i < n;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (valid) unit_point(a, X, i, px, py, pz);
#pragma unroll 2
    for (int l = 0; l < a.L; l++) {
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
        put2(E, pt, 2 * l, e0, e1);
    }
}

// The table gradient of levels l_begin, l_begin + l_step, .. < l_end of the
// warp's 32 points (one per lane, in input order) from their dENC rows (32 columns of tensor memory at tdenc,
// the warp's lane quarter).  Per level, lanes whose point lies in the same
// cell as the previous lane's form a run (coherent inputs such as LiDAR
// sweeps put many consecutive points in one coarse cell); a segmented scan
// over the run sums its 8 vertex contributions and the run's last lane adds
// them, so that one atomic per vertex replaces up to 32 on the same table
// entry.  A warp without such runs at a level adds per lane.  Entries are
// added as float2, or as one float4 where two x-neighbours of the cell are
// adjacent table entries (the first slot even).
__device__ __forceinline__ void add_vertex_pairs(float2 *tab, const uint32_t (&slot)[8], const float (&v)[16]) {
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
        if ((slot[c] & 1u) == 0u && slot[c + 1] == slot[c] + 1u) {
            atomicAdd(reinterpret_cast<float4 *>(tab + slot[c]),
                      make_float4(v[2 * c], v[2 * c + 1], v[2 * c + 2], v[2 * c + 3]));
        } else {
            atomicAdd(tab + slot[c], make_float2(v[2 * c], v[2 * c + 1]));
            atomicAdd(tab + slot[c + 1], make_float2(v[2 * c + 2], v[2 * c + 3]));
        }
    }
}

__device__ __forceinline__ void produce_table_grad(const NgpArgs &a, const float *__restrict__ X, long long i,
                                                   bool live, uint32_t tdenc, float *__restrict__ d_theta,
                                                   int l_begin, int l_end, int l_step) {
    float g[32];
    tmem_ld16(tdenc, *reinterpret_cast<float(*)[16]>(g));
    tmem_ld16(tdenc + 16u, *reinterpret_cast<float(*)[16]>(g + 16));
    const uint32_t live_mask = __ballot_sync(0xffffffffu, live);
    if (live_mask == 0u) return;
    const int lane = (int)(threadIdx.x & 31);
    float px = 0.f, py = 0.f, pz = 0.f;
    if (live) unit_point(a, X, i, px, py, pz);
#pragma unroll
    for (int l = 0; l < kMaxLevels; l++) {
        if (l >= a.L) break;
        if (l < l_begin || l >= l_end || (l - l_begin) % l_step != 0) continue;
        uint32_t slot[8];
        float w[8];
        cell_taps(a, l, px, py, pz, slot, w);
        const float g0 = live ? g[2 * l] : 0.f, g1 = live ? g[2 * l + 1] : 0.f;
        float v[16];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            v[2 * c] = w[c] * g0;
            v[2 * c + 1] = w[c] * g1;
        }
        // the cell's integer coordinates (as in cell_taps): equal cells have equal slots
        const float r = (float)a.res[l];
        const uint32_t cx = (uint32_t)fminf(floorf(px * r), r - 1.f), cy = (uint32_t)fminf(floorf(py * r), r - 1.f),
                       cz = (uint32_t)fminf(floorf(pz * r), r - 1.f);
        const uint32_t qx = __shfl_up_sync(0xffffffffu, cx, 1), qy = __shfl_up_sync(0xffffffffu, cy, 1),
                       qz = __shfl_up_sync(0xffffffffu, cz, 1);
        const bool head = lane == 0 || cx != qx || cy != qy || cz != qz;
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        float2 *tab = reinterpret_cast<float2 *>(d_theta) + (size_t)l * a.T;
        if (heads == 0xffffffffu) {
            if (live) add_vertex_pairs(tab, slot, v);
            continue;
        }
        // segmented inclusive scan over runs of lanes in the same cell
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const float t = __shfl_up_sync(0xffffffffu, v[q], d);
                if (lane - d >= start) v[q] += t;
            }
        }
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
        const uint32_t run = (0xffffffffu >> (31 - lane)) & ~((1u << start) - 1u);  // lanes start .. lane
        if (tail && (live_mask & run)) add_vertex_pairs(tab, slot, v);
    }
}

__global__ void __launch_bounds__(kBwdThreads, 1)
k_ngp_bwd(NgpArgs a, const float *__restrict__ theta, const float *__restrict__ X, long long n,
          const float *__restrict__ d_rgb, const float *__restrict__ d_logit_o, const float *__restrict__ d_log_s,
          const float *__restrict__ d_quat, float *__restrict__ d_theta) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int D = a.D;
    Carve cv{smem};
    const Mat W1 = cv.mat(kW1, kK1), W2 = cv.mat(kW2, kH), W3 = cv.mat(kW3, kH);
    const Mat Xb = cv.mat(kBwdX, 128), Yb = cv.mat(kBwdY, 96);
    const Mat E[2] = {cv.mat(kBwdE, 48), cv.mat(kBwdE, 48)};
    float *bias = reinterpret_cast<float *>(cv.p);
    float *db3 = bias + 2 * kH + 16;
    uint64_t *bar = reinterpret_cast<uint64_t *>(cv.p + kBias);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(cv.p + kBias + 16);
    volatile int *abort = reinterpret_cast<volatile int *>(cv.p + kBias + 32);
    unsigned int *live = reinterpret_cast<unsigned int *>(cv.p + kBias + 64);  // [2][128]: the point has a gradient
    stage_weights(a, theta, W1, W2, W3, bias);
    for (int e = threadIdx.x; e < 16; e += kBwdThreads) db3[e] = 0.f;
    if (threadIdx.x == 0) *abort = 0;
    // constant columns: Y 80 = 1, 81..95 = 0; E 2L..31 = 0, 32 = 1, 33..47 = 0
    for (int e = threadIdx.x; e < kTile * 16; e += kBwdThreads) put(Yb, e / 16, 80 + e % 16, e % 16 == 0 ? 1.f : 0.f);
    for (int e = threadIdx.x; e < 2 * kTile * 48; e += kBwdThreads) {
        const int b = e / (kTile * 48), r = (e / 48) % kTile, c = e % 48;
        if (c >= D) put(E[b], r, c, c == 32 ? 1.f : 0.f);
    }
    Sync s{smem_addr(bar), 0u, *(volatile unsigned long long *)&g_ngp_wait_ns};
    init_bar(s.bar);
    tmem_alloc(tslot, 512u);
    const int warp = (int)(threadIdx.x >> 5);
    const bool consumer = warp < kConsumers / 32;
    const int pt = consumer ? 0 : (int)threadIdx.x - kConsumers;  // producer: its point in the tile
    const long long tiles = (n + kTile - 1) / kTile;
    const long long K = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // tiles of this block
    if (!consumer) produce_encoding(a, theta, X, n, (long long)blockIdx.x * kTile, E[0], pt);
    publish();
    fence_after_sync();
    const uint32_t tm = *tslot;
    const Lane ln = lane_role();  // consumers: row, column half; producers: row = 32 (warp % 4) + lane
    for (long long k = 0; k < K; k++) {
        const long long base = ((long long)blockIdx.x + k * gridDim.x) * kTile;
        const int eb = (int)(k & 1);
        if (consumer) {
            const long long i = base + ln.row;
            const Mat &Ek = E[eb];
            do {
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    mma3(tm + kB_T1, kmajor(Ek, 0), kmajor(W1, 0), kK1 / 16, idesc_bf16(128, 64, 0, 0), false);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                const uint32_t mask1 = epi_relu(tm + kB_T1, ln, bias, Yb, 16);  // H1
                consumer_publish();
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    mma3(tm + kB_T2, kmajor(Yb, 16), kmajor(W2, 0), kH / 16, idesc_bf16(128, 64, 0, 0), false);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                const uint32_t mask2 = epi_relu(tm + kB_T2, ln, bias + kH, Xb, 0);  // H2
                consumer_publish();
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    mma3(tm + kB_T1, kmajor(Xb, 0), kmajor(W3, 0), kH / 16, idesc_bf16(128, 16, 0, 0), false);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                // heads: dO = dL/do (zero beyond the 11 outputs and for points beyond n)
                if (ln.half == 0) {
                    float o[16], g[16];
                    tmem_ld16(tm + kB_T1 + ln.lane_base, o);
#pragma unroll
                    for (int q = 0; q < 16; q++) g[q] = 0.f;
                    if (i < n) {
                        const float *b3 = bias + 2 * kH;
#pragma unroll
                        for (int q = 0; q < 3; q++) {
                            const float sg = sigmoidf(o[q] + b3[q]);
                            g[q] = d_rgb[3 * i + q] * sg * (1.f - sg);
                        }
                        g[3] = d_logit_o[i];
#pragma unroll
                        for (int q = 0; q < 3; q++) g[4 + q] = d_log_s[3 * i + q];
#pragma unroll
                        for (int q = 0; q < 4; q++) g[7 + q] = d_quat[4 * i + q];
                    }
                    put8(Yb, ln.row, 0, g);
                    put8(Yb, ln.row, 8, g + 8);
                    bool any = false;
#pragma unroll
                    for (int q = 0; q < kO; q++) any |= g[q] != 0.f;
                    live[eb * kTile + ln.row] = any ? 1u : 0u;
#pragma unroll
                    for (int q = 0; q < kO; q++) {
                        float v = g[q];
#pragma unroll
                        for (int sft = 16; sft > 0; sft >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sft);
                        if ((threadIdx.x & 31) == 0) atomicAdd(db3 + q, v);
                    }
                }
                consumer_publish();
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    // dH2 = dO W3 (W3 read MN-major as its transpose)
                    mma3(tm + kB_T2, kmajor(Yb, 0), mnmajor(W3, 0), 1, idesc_bf16(128, 64, 0, 1), false);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                epi_mask(tm + kB_T2, ln, mask2, Xb, 64);  // dA2
                consumer_publish();
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    mma3(tm + kB_T1, kmajor(Xb, 64), mnmajor(W2, 0), kH / 16, idesc_bf16(128, 64, 0, 1), false);
                    // [H2 | dA2]^T [dO | H1 | 1]
                    mma3(tm + kB_ACCA, mnmajor(Xb, 0), mnmajor(Yb, 0), kTile / 16, idesc_bf16(128, 96, 1, 1), k > 0);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                epi_mask(tm + kB_T1, ln, mask1, Xb, 0);  // dA1 replaces H2 (the product above is done)
                consumer_publish();
                if (threadIdx.x == 0) {
                    fence_after_sync();
                    mma3(tm + kB_DENC + 32u * (uint32_t)eb, kmajor(Xb, 0), mnmajor(W1, 0), kH / 16,
                         idesc_bf16(128, 32, 0, 1), false);
                    // [dA1 | dA2]^T [ENC | 1]
                    mma3(tm + kB_ACCB, mnmajor(Xb, 0), mnmajor(Ek, 0), kTile / 16, idesc_bf16(128, 48, 1, 1), k > 0);
                    mma_commit(s.bar);
                }
                if (!consumer_wait(s, abort)) break;
                // this tile's coarse levels: even ones by column half 0, odd ones by half 1
                if (kConsumerLevels > 0)
                    produce_table_grad(a, X, i, i < n && live[eb * kTile + ln.row] != 0u,
                                       tm + ln.lane_base + kB_DENC + 32u * (uint32_t)eb, d_theta, ln.half,
                                       kConsumerLevels, 2);
            } while (false);
        } else {
            // the next tile's encoding, then the previous tile's table gradient
            if (k + 1 < K) produce_encoding(a, theta, X, n, base + (long long)gridDim.x * kTile, E[eb ^ 1], pt);
            if (k > 0) {
                fence_after_sync();
                const long long ip = base - (long long)gridDim.x * kTile + pt;
                produce_table_grad(a, X, ip, ip < n && live[(eb ^ 1) * kTile + pt] != 0u,
                                   tm + ln.lane_base + kB_DENC + 32u * (uint32_t)(eb ^ 1), d_theta, kConsumerLevels, kMaxLevels, 1);
            }
        }
        publish();
        fence_after_sync();
        if (*abort) break;
    }
    if (*abort) {
        if (threadIdx.x == 0) {
            atomicOr(&g_ngp_fault, 1u);
            mbar_drain(s.bar, s.phase);  // the MMAs still in flight, bounded
            atomicAdd(d_theta, __int_as_float(0x7fc00000));  // poison: the gradient is incomplete
        }
    } else if (K > 0) {
        if (!consumer) {
            // the last tile's table gradient
            const long long last = ((long long)blockIdx.x + (K - 1) * gridDim.x) * kTile;
            const int eb = (int)((K - 1) & 1);
            const long long ip = last + pt;
            produce_table_grad(a, X, ip, ip < n && live[eb * kTile + pt] != 0u,
                               tm + ln.lane_base + kB_DENC + 32u * (uint32_t)eb, d_theta, kConsumerLevels, kMaxLevels, 1);
        } else {
            // the block's weight gradients: this thread's row of the accumulators
            float *g1 = d_theta + a.w1;
            const int r = ln.row;
            const int c_end = ln.half == 0 ? 64 : 96;
#pragma unroll 1
            for (int c0 = 64 * ln.half; c0 < c_end; c0 += 16) {
                float v[16];
                tmem_ld16(tm + kB_ACCA + ln.lane_base + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int c = c0 + j;
                    if (r < 64) {
                        if (c < kO) atomicAdd(g1 + off_w3(D) + c * kH + r, v[j]);  // dW3[c][r]
                    } else if (c >= 16 && c < 80) {
                        atomicAdd(g1 + off_w2(D) + (r - 64) * kH + (c - 16), v[j]);  // dW2[r - 64][c - 16]
                    } else if (c == 80) {
                        atomicAdd(g1 + off_b2(D) + (r - 64), v[j]);  // db2[r - 64]
                    }
                }
            }
            if (r < 64) {  // uniform per warp (lane quarters 0 and 1)
                float v[16];
                tmem_ld16(tm + kB_ACCB + ln.lane_base + (uint32_t)(16 * ln.half), v);
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int c = 16 * ln.half + j;
                    if (c < D) atomicAdd(g1 + r * D + c, v[j]);  // dW1[r][c]
                }
                if (ln.half == 0) {
                    tmem_ld16(tm + kB_ACCB + ln.lane_base + 32u, v);
                    atomicAdd(g1 + off_b1(D) + r, v[0]);  // db1[r]
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kO; q += kBwdThreads) atomicAdd(d_theta + a.w1 + off_b3(D) + q, db3[q]);
    }
    tmem_free(tm, 512u);
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
    k_ngp_bwd<<<grid, kBwdThreads, bwd_smem(), s>>>(a, theta, X, n, d_rgb, d_logit_o, d_log_s, d_quat, d_theta);
    return cudaGetLastError();
}

cudaError_t ngp_set_wait_limit(unsigned long long ns) { return cudaMemcpyToSymbol(g_ngp_wait_ns, &ns, sizeof(ns)); }

cudaError_t ngp_fault(unsigned int *out) {
    unsigned int v = 0, z = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_ngp_fault, sizeof(v));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ngp_fault, &z, sizeof(z));
    *out = v;
    return e;
}

}  // namespace gs
