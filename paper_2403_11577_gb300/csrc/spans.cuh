// Exact tile binning: the tiles of a record's rectangle that its ellipse can
// meet, shared by the projection (which counts each record's pairs and
// non-empty tile rows) and the pair emission (which lists them), so that
// both compute every span bit for bit alike.
#pragma once

#include "common.cuh"

namespace gs {

// ---------------------------------------------------- exact tile binning
//
// With exact tiles a record is listed only for the tiles of its rectangle
// that its ellipse P(d) <= F - lmin (P = -(A dx^2 + B dx dy + C dy^2), the
// splat's base-2 exponent) can meet: in every tile row the pixel centres
// where a Gaussian reaches alpha_min lie between the x-extremes of the
// ellipse within the row's y-range, a contiguous run of tiles.  The test
// uses the ellipse enlarged by 2^-8 |F - lmin| + 2^-14 M (M bounds P's
// terms over the whole rectangle), four times the margins of the render's
// band culling, and widens each run by 0.02 px + 2^-10 of its offsets, so
// every band the render would keep lies in a listed tile: the image is the
// same, bit for bit, as with whole rectangles.  A degenerate or non-finite
// ellipse keeps whole rows.
struct RowSpanner {
    float mx, my, qb, lim4a, D, ymax, yR, inv2a, full;  // full != 0: whole rows
};

// The span arithmetic is written with explicitly rounded operations (no
// contraction into fused multiply-adds) and hardware approximations whose
// results depend only on their inputs, so that the projection's pair count
// and the emission, separate kernels, compute every span bit for bit alike.
// The approximations (relative error about 2^-22) are far inside the 2^-8
// margin of the test.
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ RowSpanner make_spanner(float4 s0, float4 s1, float lmin, uint2 rc, const gs_frame &fr,
                                                   int T) {
    RowSpanner s;
    s.mx = s0.x;
    s.my = s0.y;
    const float qa = -s0.z, qb = -s0.w, qc = -s1.x;
    s.qb = qb;
    const float lim0 = sub_(s1.y, lmin);
    const float x0 = (float)((rc.x & 0xffffu) * (uint32_t)T), x1 = (float)((rc.y & 0xffffu) * (uint32_t)T + T - 1);
    const float y0 = (float)(fr.row0 + (int)(rc.x >> 16) * T), y1 = (float)(fr.row0 + (int)(rc.y >> 16) * T + T - 1);
    const float Rx = fmaxf(fabsf(sub_(x0, s.mx)), fabsf(sub_(x1, s.mx)));
    const float Ry = fmaxf(fabsf(sub_(y0, s.my)), fabsf(sub_(y1, s.my)));
    const float M = add_(add_(mul_(mul_(qa, Rx), Rx), mul_(mul_(fabsf(qb), Rx), Ry)), mul_(mul_(qc, Ry), Ry));
    const float lim = add_(add_(lim0, mul_(fabsf(lim0), 0x1p-8f)), mul_(M, 0x1p-14f));
    s.D = sub_(mul_(mul_(4.f, qa), qc), mul_(qb, qb));
    const bool ok = qa > 0.f && qc > 0.f && s.D > 0.f && lim > 0.f && isfinite(lim) && isfinite(s.D) &&
                    isfinite(s.mx) && isfinite(s.my) && isfinite(qb);
    s.full = ok ? 0.f : 1.f;
    s.lim4a = mul_(mul_(4.f, qa), lim);
    s.inv2a = rcp_approx(mul_(2.f, qa));
    // largest |y| on the ellipse (widened), and the y of its rightmost point
    // (the leftmost is at -yR)
    s.ymax = ok ? add_(mul_(sqrt_approx(mul_(s.lim4a, rcp_approx(s.D))), 1.f + 0x1p-12f), 1e-3f) : 0.f;
    const float xm = ok ? sqrt_approx(mul_(mul_(mul_(4.f, qc), lim), rcp_approx(s.D))) : 0.f;
    s.yR = ok ? mul_(mul_(-qb, xm), rcp_approx(mul_(2.f, qc))) : 0.f;
    return s;
}

// Tile columns [lo, hi] of tile row ty within the rectangle's columns
// [rx0, rx1] (lo > hi: none).
__device__ __forceinline__ void row_span(const RowSpanner &s, int ty, int rx0, int rx1, const gs_frame &fr, int T,
                                         int &lo, int &hi) {
    lo = rx0;
    hi = rx1;
    if (s.full != 0.f) return;
    const float ylo = (float)(fr.row0 + ty * T), yhi = (float)min(fr.row0 + ty * T + T - 1, fr.height - 1);
    const float a = fmaxf(sub_(ylo, s.my), -s.ymax), b = fminf(sub_(yhi, s.my), s.ymax);
    if (a > b) {
        lo = 1;
        hi = 0;
        return;
    }
    // the x-extremes over y in [a, b]: x+(y) is concave, largest at the
    // clamped y of the rightmost point; x-(y) is its mirror
    const float yr = fminf(fmaxf(s.yR, a), b), yl = fminf(fmaxf(-s.yR, a), b);
    const float rr = sqrt_approx(fmaxf(0.f, sub_(s.lim4a, mul_(mul_(s.D, yr), yr))));
    const float rl = sqrt_approx(fmaxf(0.f, sub_(s.lim4a, mul_(mul_(s.D, yl), yl))));
    const float Xb = mul_(add_(mul_(-s.qb, yr), rr), s.inv2a);
    const float Xa = mul_(sub_(mul_(-s.qb, yl), rl), s.inv2a);
    const float w = add_(add_(0.02f, mul_(0x1p-10f, add_(fabsf(Xa), fabsf(Xb)))), mul_(0x1p-12f, fabsf(s.mx)));
    const float xa = fminf(fmaxf(sub_(add_(s.mx, Xa), w), -1e9f), 1e9f);
    const float xb = fminf(fmaxf(add_(add_(s.mx, Xb), w), -1e9f), 1e9f);
    // T is 8, 16 or 32: x / T and x * (1 / T) are the same real number
    // (a power-of-two scaling), so the rounded product equals the rounded
    // quotient bit for bit
    const float invT = T == 8 ? 0.125f : (T == 16 ? 0.0625f : 0.03125f);
    lo = max(rx0, (int)floorf(mul_(xa, invT)));
    hi = min(rx1, (int)floorf(mul_(xb, invT)));
}


}  // namespace gs
