// Internal definitions shared by the kernels and the C ABI of the wavelet rasterizer (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include <string>

#include "../../include/wipes.h"

namespace wipes {

constexpr int kTile = WIPES_TILE;
constexpr int kTilePixels = kTile * kTile;
constexpr float kExtMargin = 1.0009765625f;  // 1 + 2^-10: footprint half-extent safety factor
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kInvTwoPi = 0.15915494309189535f;
constexpr float kPi = 3.141592653589793f;
constexpr float kDampExp2 = 28.47765864997501f;  // 2 pi^2 log2(e): kappa = exp(-2 pi^2 x) = ex2(-x kDampExp2)

// Projected record (4 x float4 = 64 bytes per primitive), written by the footprint kernels:
//   [0] mx, my, l11, l21    centre (px) and lower Cholesky factor L of Sigma'^-1 = L L^T
//   [1] l22, fx, fy, phc    frequency (cycles/px) and phase (cycles)
//   [2] c_r, c_g, c_b, o    colour and opacity (2D: o = 1)
//   [3] ex, ey, depth, hk   half extents of the cutoff ellipse (px), camera z (3D) and the
//                           oscillation's weight hk = kappa / 2 (3D; 1/2 but under frequency map 2,
//                           where kappa is the damping of the oscillation integrated along the ray)
// The modulation is M = hk cos(2 pi t) + 1/2 (t the phase in cycles).
// The squared Mahalanobis distance at offset (dx, dy) is  q = (l11 dx + l21 dy)^2 + (l22 dy)^2,
// evaluated everywhere by mahalanobis2() so that the cutoff decision is the same in every kernel.
constexpr int kRecF4 = 4;

// Covered pixel range of a primitive (inclusive), u0 > u1 when empty.
struct PixRect {
    int u0, v0, u1, v1;
};

__device__ __forceinline__ float mahalanobis2(float px, float py, float mx, float my, float l11, float l21,
                                              float l22) {
    const float dx = __fsub_rn(px, mx);
    const float dy = __fsub_rn(py, my);
    const float a = __fmaf_rn(l11, dx, __fmul_rn(l21, dy));
    const float b = __fmul_rn(l22, dy);
    return __fmaf_rn(a, a, __fmul_rn(b, b));
}

// Approximate transcendental functions (MUFU): ex2.approx and cos/sin.approx from PTX.
constexpr float kNegHalfLog2e = -0.7213475204444817f;  // -log2(e) / 2: exp(-q/2) = ex2(q * kNegHalfLog2e)

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1 / x to within 1 ulp (MUFU reciprocal)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Phase t given in cycles, reduced to an angle in [-pi, pi]: 2 pi (t - rint(t)).
__device__ __forceinline__ float reduced_angle(float t) { return (t - rintf(t)) * kTwoPi; }

// Packed pairs of binary32 values for sm_100-family f32x2 arithmetic: one instruction performs
// the same correctly rounded operation on both halves, so a lane evaluates two pixels for the
// issue cost of one.  Each result is bit-identical to the scalar operation (fma fused, add, sub
// and mul rounded to nearest even).
struct f2 {
    unsigned long long r;
};
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v.r) : "f"(lo), "f"(hi));
    return v;
}
__device__ __forceinline__ f2 f2_dup(float x) { return f2_pack(x, x); }
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float((unsigned)(v.r & 0xffffffffull)); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((unsigned)(v.r >> 32)); }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
// A staged pair of packed values (16 bytes, one shared-memory vector load).
struct f2x2 {
    f2 x, y;
};
__device__ __forceinline__ f2x2 ld_f2x2(const ulonglong2* p) {
    const ulonglong2 v = *p;
    return f2x2{f2{v.x}, f2{v.y}};
}
// The same load kept in place (not hoisted out of a loop): for values that are cheaper to read
// again from shared memory than to hold in registers.
__device__ __forceinline__ f2x2 ld_f2x2_here(const ulonglong2* p) {
    f2x2 v;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];"
                 : "=l"(v.x.r), "=l"(v.y.r)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}
__device__ __forceinline__ ulonglong2 dup2(float a, float b) { return make_ulonglong2(f2_dup(a).r, f2_dup(b).r); }

// Round to the nearest integer (ties to even) for |t| < 2^22 on the FMA pipe: adding 1.5 2^23
// leaves no fraction bits, and the rounding of that addition is the rounding to an integer.
// Phases are a few hundred cycles at most, far inside that range.
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23
// Packed phase reduction: 2 pi (t - rint(t)) per half.
__device__ __forceinline__ f2 f2_reduced_angle(f2 t) {
    const f2 M = f2_dup(kRoundMagic);
    const f2 r = f2_sub(f2_add(t, M), M);
    return f2_mul(f2_sub(t, r), f2_dup(kTwoPi));
}

// Sum 16 per-lane values over the warp by recursive halving (reduce-scatter): 15 shuffles
// instead of 80.  On return lane l holds the warp total of value (l >> 1).
__device__ __forceinline__ float warp_reduce_scatter16(float v[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16, half = 8; off >= 2; off >>= 1, half >>= 1) {
        const bool hi = lane & off;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = hi ? v[i] : v[half + i];
            const float keep = hi ? v[half + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// View-dependent colour (the spherical-harmonic colour of 3DGS that the paper's 3D primitives carry,
// Sec. 3.1).  Real spherical harmonics of degree <= 3 at the unit vector (x, y, z), Condon-Shortley
// phase, ordered by degree l and order m = -l..l; the constants are the normalisations
// 1/2 sqrt(1/pi), sqrt(3/(4 pi)), 1/2 sqrt(15/pi), 1/4 sqrt(5/pi), 1/4 sqrt(15/pi),
// 1/4 sqrt(35/(2 pi)), 1/2 sqrt(105/pi), 1/4 sqrt(21/(2 pi)), 1/4 sqrt(7/pi), 1/4 sqrt(105/pi).
constexpr int kShMaxCoeffs = 16;
struct ShConst {
    static constexpr float c0 = 0.28209479177387814f, c1 = 0.4886025119029199f;
    static constexpr float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    static constexpr float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    static constexpr float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
};

__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[kShMaxCoeffs]) {
    using K = ShConst;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = K::c0;
    Y[1] = -K::c1 * y;
    Y[2] = K::c1 * z;
    Y[3] = -K::c1 * x;
    Y[4] = K::c2a * x * y;
    Y[5] = -K::c2a * y * z;
    Y[6] = K::c2b * (2.f * zz - xx - yy);
    Y[7] = -K::c2a * x * z;
    Y[8] = K::c2c * (xx - yy);
    Y[9] = -K::c3a * y * (3.f * xx - yy);
    Y[10] = K::c3b * x * y * z;
    Y[11] = -K::c3c * y * (4.f * zz - xx - yy);
    Y[12] = K::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -K::c3c * x * (4.f * zz - xx - yy);
    Y[14] = K::c3e * z * (xx - yy);
    Y[15] = -K::c3a * x * (xx - 3.f * yy);
}

// Partial derivatives dY_k/dx, dY_k/dy, dY_k/dz of the polynomials above.
__device__ __forceinline__ void sh_eval_grad(float x, float y, float z, float gx[kShMaxCoeffs], float gy[kShMaxCoeffs],
                                             float gz[kShMaxCoeffs]) {
    using K = ShConst;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx[0] = 0.f; gy[0] = 0.f; gz[0] = 0.f;
    gx[1] = 0.f; gy[1] = -K::c1; gz[1] = 0.f;
    gx[2] = 0.f; gy[2] = 0.f; gz[2] = K::c1;
    gx[3] = -K::c1; gy[3] = 0.f; gz[3] = 0.f;
    gx[4] = K::c2a * y; gy[4] = K::c2a * x; gz[4] = 0.f;
    gx[5] = 0.f; gy[5] = -K::c2a * z; gz[5] = -K::c2a * y;
    gx[6] = -2.f * K::c2b * x; gy[6] = -2.f * K::c2b * y; gz[6] = 4.f * K::c2b * z;
    gx[7] = -K::c2a * z; gy[7] = 0.f; gz[7] = -K::c2a * x;
    gx[8] = 2.f * K::c2c * x; gy[8] = -2.f * K::c2c * y; gz[8] = 0.f;
    gx[9] = -6.f * K::c3a * x * y; gy[9] = -3.f * K::c3a * (xx - yy); gz[9] = 0.f;
    gx[10] = K::c3b * y * z; gy[10] = K::c3b * x * z; gz[10] = K::c3b * x * y;
    gx[11] = 2.f * K::c3c * x * y; gy[11] = -K::c3c * (4.f * zz - xx - 3.f * yy); gz[11] = -8.f * K::c3c * y * z;
    gx[12] = -6.f * K::c3d * x * z; gy[12] = -6.f * K::c3d * y * z; gz[12] = K::c3d * (6.f * zz - 3.f * xx - 3.f * yy);
    gx[13] = -K::c3c * (4.f * zz - 3.f * xx - yy); gy[13] = 2.f * K::c3c * x * y; gz[13] = -8.f * K::c3c * x * z;
    gx[14] = 2.f * K::c3e * x * z; gy[14] = -2.f * K::c3e * y * z; gz[14] = K::c3e * (xx - yy);
    gx[15] = -3.f * K::c3a * (xx - yy); gy[15] = 6.f * K::c3a * x * y; gz[15] = 0.f;
}

// SH coefficient k (0..15) of channel ch in an [N, WIPES_P3D_SH] record: the record colour for
// k = 0, then three channels per basis function.
// n consecutive floats of a row in 16-byte pieces (VEC: the row is 16-byte aligned) or one by one
template <bool VEC, int n>
__device__ __forceinline__ void load_row(float* dst, const float* __restrict__ src) {
    if (VEC) {
#pragma unroll
        for (int q = 0; q < n / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(src)[q];
            dst[4 * q] = v.x, dst[4 * q + 1] = v.y, dst[4 * q + 2] = v.z, dst[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < n; ++k) dst[k] = src[k];
    }
}
template <bool VEC, int n>
__device__ __forceinline__ void store_row(float* dst, const float* v) {
    if (VEC) {
#pragma unroll
        for (int q = 0; q < n / 4; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < n; ++k) dst[k] = v[k];
    }
}

__device__ __forceinline__ int sh_slot(int k, int ch) { return k == 0 ? 15 + ch : 20 + 3 * (k - 1) + ch; }

// Cutoff test of a rectangle of pixel centres (columns x0..x1, rows y0..y1): does the cutoff
// ellipse q <= lim (lim = cutoff^2 x 1.01) reach it?  With q = A dx^2 + 2 B dx dy + C dy^2
// (A = l11^2, B = l11 l21, C = l21^2 + l22^2) the minimum over the rectangle is 0 when the centre
// lies inside, else the least of the four edge minima: dy = -(B/C) dx clamped on an edge of fixed
// dx, dx = -(B/A) dy clamped on an edge of fixed dy.  Written with explicit single-rounding
// operations so that the tile lists built from it are reproducible operation by operation.  The
// margin exceeds the rounding of the per-pixel test, so a pixel that passes
// mahalanobis2() <= cutoff^2 always lies in a rectangle accepted here.
struct Ellipse {
    float mx, my, l11, l21, l22;
    float rBA, rBC;  // -(B/A), -(B/C)
};

__device__ __forceinline__ Ellipse make_ellipse(float mx, float my, float l11, float l21, float l22) {
    const float A = __fmul_rn(l11, l11), B = __fmul_rn(l11, l21);
    const float C = __fadd_rn(__fmul_rn(l21, l21), __fmul_rn(l22, l22));
    Ellipse e;
    e.mx = mx; e.my = my; e.l11 = l11; e.l21 = l21; e.l22 = l22;
    e.rBA = -__fdiv_rn(B, A);
    e.rBC = -__fdiv_rn(B, C);
    return e;
}

__device__ __forceinline__ bool rect_touched(const Ellipse& k, int x0, int x1, int y0, int y1, float lim) {
    const float dx0 = __fsub_rn(__fadd_rn((float)x0, 0.5f), k.mx), dx1 = __fsub_rn(__fadd_rn((float)x1, 0.5f), k.mx);
    const float dy0 = __fsub_rn(__fadd_rn((float)y0, 0.5f), k.my), dy1 = __fsub_rn(__fadd_rn((float)y1, 0.5f), k.my);
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    float best = 0.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float dx, dy;
        if (e < 2) {
            dx = e == 0 ? dx0 : dx1;
            dy = fminf(fmaxf(__fmul_rn(k.rBC, dx), dy0), dy1);
        } else {
            dy = e == 2 ? dy0 : dy1;
            dx = fminf(fmaxf(__fmul_rn(k.rBA, dy), dx0), dx1);
        }
        const float a = __fadd_rn(__fmul_rn(k.l11, dx), __fmul_rn(k.l21, dy));
        const float b = __fmul_rn(k.l22, dy);
        const float q = __fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b));
        best = e == 0 ? q : fminf(best, q);
    }
    return best <= lim;
}

// Tile (tx, ty) clipped to a covered pixel range, tested with rect_touched().
__device__ __forceinline__ bool tile_touched(const Ellipse& k, const PixRect& r, int tx, int ty, float lim) {
    const int x0 = max(tx * kTile, r.u0), x1 = min(tx * kTile + kTile - 1, r.u1);
    const int y0 = max(ty * kTile, r.v0), y1 = min(ty * kTile + kTile - 1, r.v1);
    return rect_touched(k, x0, x1, y0, y1, lim);
}

// Does the primitive's cutoff ellipse reach the bw x bh pixel box at (bx, by), clipped to its
// covered range?  The same rectangle test as rect_touched() in ordinary (fused) arithmetic; the
// 1 % margin of lim keeps it conservative.  nBA, nBC from ellipse_edge_ratios().
__device__ __forceinline__ bool box_touched_ellipse(const float4& A4, float l22, float nBA, float nBC,
                                                    const PixRect& r, int bx, int by, int bw, int bh, float lim) {
    const float l11 = A4.z, l21 = A4.w;
    const int sx0 = max(bx, r.u0), sx1 = min(bx + bw - 1, r.u1);
    const int sy0 = max(by, r.v0), sy1 = min(by + bh - 1, r.v1);
    if (sx0 > sx1 || sy0 > sy1) return false;
    const float dx0 = ((float)sx0 + 0.5f) - A4.x, dx1 = ((float)sx1 + 0.5f) - A4.x;
    const float dy0 = ((float)sy0 + 0.5f) - A4.y, dy1 = ((float)sy1 + 0.5f) - A4.y;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    float best = 3.4e38f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float dx, dy;
        if (e < 2) {
            dx = e == 0 ? dx0 : dx1;
            dy = fminf(fmaxf(nBC * dx, dy0), dy1);
        } else {
            dy = e == 2 ? dy0 : dy1;
            dx = fminf(fmaxf(nBA * dy, dx0), dx1);
        }
        const float a = fmaf(l11, dx, l21 * dy), b = l22 * dy;
        best = fminf(best, fmaf(a, a, b * b));
    }
    return best <= lim;
}

__device__ __forceinline__ void ellipse_edge_ratios(const float4& A4, float l22, float& nBA, float& nBC) {
    const float l11 = A4.z, l21 = A4.w;
    const float A = l11 * l11, B = l11 * l21, C = fmaf(l21, l21, l22 * l22);
    nBA = -B / A;
    nBC = -B / C;
}

// Which of the eight 8x4 warp sub-tiles of the 16x16 tile at (x0, y0) the primitive's cutoff
// ellipse reaches: bit w for warp w (columns 8 (w & 1) .. +7, rows 4 (w >> 1) .. +3).
__device__ __forceinline__ uint32_t subtile_mask_ellipse(const float4& A4, float l22, const PixRect& r, int x0, int y0,
                                                         float lim) {
    float nBA, nBC;
    ellipse_edge_ratios(A4, l22, nBA, nBC);
    uint32_t m = 0;
#pragma unroll 1
    for (int w = 0; w < 8; ++w)
        if (box_touched_ellipse(A4, l22, nBA, nBC, r, x0 + 8 * (w & 1), y0 + 4 * (w >> 1), 8, 4, lim)) m |= 1u << w;
    return m;
}

// Which of the four 8x8 quadrants of the 16x16 tile at (x0, y0) the primitive's cutoff ellipse
// reaches: bit k for columns 8 (k & 1) .. +7, rows 8 (k >> 1) .. +7.
__device__ __forceinline__ uint32_t quadrant_mask_ellipse(const float4& A4, float l22, const PixRect& r, int x0,
                                                          int y0, float lim) {
    float nBA, nBC;
    ellipse_edge_ratios(A4, l22, nBA, nBC);
    uint32_t m = 0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k)
        if (box_touched_ellipse(A4, l22, nBA, nBC, r, x0 + 8 * (k & 1), y0 + 8 * (k >> 1), 8, 8, lim)) m |= 1u << k;
    return m;
}

// The same test for the two 8x4 sub-tiles of the 8x8 quad at (x0, y0): bit 0 rows 0..3, bit 1
// rows 4..7.  Sub-tile k of quad (qx, qy) is sub-tile 4 qy + 2 k + qx of the 16x16 tile.
__device__ __forceinline__ uint32_t quad_mask_ellipse(const float4& A4, float l22, const PixRect& r, int x0, int y0,
                                                      float lim) {
    float nBA, nBC;
    ellipse_edge_ratios(A4, l22, nBA, nBC);
    uint32_t m = box_touched_ellipse(A4, l22, nBA, nBC, r, x0, y0, 8, 4, lim) ? 1u : 0u;
    if (box_touched_ellipse(A4, l22, nBA, nBC, r, x0, y0 + 4, 8, 4, lim)) m |= 2u;
    return m;
}

// Which of the eight 8x4 warp sub-tiles of the 16x16 tile at (x0, y0) a covered pixel range
// touches: bit w for warp w (columns 8 (w & 1) .. +7, rows 4 (w >> 1) .. +3).
__device__ __forceinline__ uint32_t subtile_mask(const PixRect& r, int x0, int y0) {
    uint32_t xo = 0, yo = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) xo |= (uint32_t)(r.u0 <= x0 + 8 * h + 7 && r.u1 >= x0 + 8 * h) << h;
#pragma unroll
    for (int q = 0; q < 4; ++q) yo |= (uint32_t)(r.v0 <= y0 + 4 * q + 3 && r.v1 >= y0 + 4 * q) << q;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m |= ((xo >> (w & 1)) & (yo >> (w >> 1)) & 1u) << w;
    return m;
}

// Launch helpers ---------------------------------------------------------------------------------

// Programmatic dependent launch.  Every kernel of the library starts with pdl_enter(): it waits
// until the kernel before it on the stream has completed and its writes are visible, then allows
// the kernel after it to be scheduled.  Kernels are launched with launch_pdl(), which lets the
// hardware start that scheduling while the previous kernel drains, so a chain of short dependent
// kernels does not pay a full launch latency at every boundary.  Work on the stream that is not a
// kernel launched this way (copies, memsets, events, other libraries' kernels) keeps the usual
// stream order.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Returns the launch's own result (callers that check errors later may ignore it).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Limit of rect_touched(): cutoff^2 widened by 1 %, in binary32 (host side).
inline float touch_limit(float cutoff) {
    volatile float k2 = cutoff * cutoff;
    return k2 * 1.01f;
}

// Power-of-two scale S with S cutoff^2 in [2^32, 2^33): any binary32 q > cutoff^2 then has
// S (cutoff^2 - q) <= -512, so ex2 of it is 0 (host side; cutoff^2 is a normal binary32 number).
inline float cutoff_scale(float cutoff2) {
    int e = 0;
    std::frexp(cutoff2, &e);
    return std::ldexp(1.0f, std::min(33 - e, 126));
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Camera centre in world coordinates, -R^T t for the view matrix [R | t].
inline void camera_centre(const wipes_camera& cam, float out[3]) {
    for (int j = 0; j < 3; ++j)
        out[j] = -(cam.viewmat[0 * 4 + j] * cam.viewmat[3] + cam.viewmat[1 * 4 + j] * cam.viewmat[7] +
                   cam.viewmat[2 * 4 + j] * cam.viewmat[11]);
}

// Library-wide count of kernel launches (every launcher adds the kernels it enqueues).
void count_launches(int n);

// Launchers implemented in the kernel translation units (all enqueue on `stream`).

// footprint.cu
void launch_footprint2d(const float* params, int64_t N, int W, int H, float cutoff, int cov2d, float4* rec, PixRect* rect,
                        uint32_t* counts, uint32_t* depth_keys, cudaStream_t stream);
void launch_footprint3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float cutoff,
                        float dilation, int fmode, int sh_degree, float4* rec, PixRect* rect, uint32_t* counts,
                        uint32_t* depth_keys, cudaStream_t stream);
void launch_deform6d(const float* params6, int64_t N, float t, float* params3, cudaStream_t stream);
void launch_deform6d_backward(const float* params6, int64_t N, float t, const float* g3, float* g6, int accumulate,
                              cudaStream_t stream);

// binning.cu
// Per-block sums of counts (in the order given by perm, or primitive order if perm is null).
constexpr int kScanBlockElems = 1024;
void launch_block_sums(const uint32_t* counts, const uint32_t* perm, int64_t n, unsigned long long* block_sums,
                       cudaStream_t stream);
// Exclusive scan of nb block sums in place; total written to *total.  With a readback pointer (the
// device address of mapped pinned host memory) the total and *error also go to readback[0..1].
void launch_scan_block_sums(unsigned long long* block_sums, int nb, unsigned long long* total,
                            const unsigned long long* error, unsigned long long* readback, cudaStream_t stream);
// Emit one instance per tile the cutoff ellipse reaches, in scan order: keys[e] = tile id,
// vals[e] = e (the emission index), inst_prim[e] = primitive; offsets[prim] = its first index.
// Also sets the n_tiles tile ranges to empty (for launch_tile_ranges with zeroed = true).  The
// emission writes nothing when the instance total (*total, on the device) exceeds `capacity`, the
// element count of keys, vals and inst_prim.
void launch_emit(const uint32_t* counts, const uint32_t* perm, int64_t n, const float4* rec, const PixRect* rect,
                 const unsigned long long* block_offsets, const unsigned long long* total, int64_t capacity,
                 int tiles_x, float lim, uint32_t* keys, uint32_t* vals, uint32_t* inst_prim, uint32_t* offsets,
                 uint2* ranges, int n_tiles, cudaStream_t stream);
// out[i] = table[idx[i]]
void launch_gather_u32(uint32_t* out, const uint32_t* table, const uint32_t* idx, int64_t n, cudaStream_t stream);
// ranges[t] = [start, end) of tile t in the sorted keys; zeroed: the ranges were set to empty before
// (by launch_emit), else they are cleared here first
void launch_tile_ranges(const uint32_t* sorted_keys, int64_t n, uint2* ranges, int n_tiles, bool zeroed,
                        cudaStream_t stream);
void launch_iota(uint32_t* v, int64_t n, cudaStream_t stream);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).  Uses (keys[0], vals[0]) as
// input and (keys[1], vals[1]) as ping-pong space; returns which buffer index holds the result.
// `hist` must hold radix_hist_words(n) words (8-byte aligned).  With a table, the last pass also
// writes gathered[i] = table[sorted value i].  A look-back wait that runs out sets bit 0 of
// *error (device memory) and leaves the result undefined.
int64_t radix_hist_words(int64_t n);
int radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits, uint32_t* hist, unsigned int* error,
                     cudaStream_t stream, const uint32_t* table = nullptr, uint32_t* gathered = nullptr);
// Diagnostic: one sort pass over sort_timeout_probe_words() words of scratch whose predecessor
// tile never publishes; its look-back runs out and sets bit 0 of *error.
int64_t sort_timeout_probe_words();
void sort_timeout_probe(uint32_t* ws, unsigned int* error, cudaStream_t stream);
// order[0 .. n_tiles) = the tiles, longest list first (see k_tile_order)
// 3D backward: tile lists longer than kBwdChunkFrom entries are walked in chunks of kBwdChunk
// entries at once (a multiple of the 3D blend's batch of 32); shorter ones in one piece
constexpr int kBwdChunk = 256;
constexpr int kBwdChunkFrom = 256;
__host__ __device__ inline uint32_t bwd_chunks(uint32_t len) {
    return len == 0u ? 0u : (len > (uint32_t)kBwdChunkFrom ? (len + kBwdChunk - 1) / kBwdChunk : 1u);
}
// tiles longest list first; and the 3D backward's items (tile, chunk) in that order (items,
// item_base[tile] = the tile's first item, *n_items) when `items` is given
void launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, uint2* items, uint32_t* item_base,
                       uint32_t* n_items, cudaStream_t stream);

// raster2d.cu
// Tile lists: entry i of the sorted list is emission index sorted[i] of primitive prim[i].
struct TileLists {
    const uint32_t* sorted;  // emission indices in tile order
    const uint32_t* prim;    // primitive of each sorted entry
    const uint2* ranges;     // [start, end) of each tile in `sorted`
};
// One frame's forward pass over prepared tile lists (2D summed field or 3D front-to-back blend).
struct BlendOpts3 {
    float cutoff2, lim, alpha_min, alpha_max, T_min;
    float bg[3];
    int damp;  // 3D frequency map 2: the records carry hk = kappa / 2 (else hk = 1/2 everywhere)
    float cut_scale;  // 2D: cutoff_scale(cutoff2), the power-of-two scale of the cutoff in the exponent
};
struct BlendJob {
    const float4* rec;
    const PixRect* rect;
    TileLists tl;
    float* out;
    float* T_final;  // 3D only
    uint32_t* last;  // 3D only
    int dims, W, H, tiles_x;
    BlendOpts3 o;    // 2D uses cutoff2 and lim only
    // 3D one-frame forward, for the chunked backward: every pixel's (T, colour) before list entry
    // k kBwdChunk, k >= 1, at bnd[(item_base[tile] + k) 256 + pixel of the tile], and its final
    // colour without the background at cfin (3 floats per pixel); unused when bnd is null
    const uint32_t* item_base = nullptr;
    float4* bnd = nullptr;
    float* cfin = nullptr;
};
void launch_blend2d(const BlendJob& job, int tiles_y, cudaStream_t stream);
void launch_backward2d(const float4* rec, const PixRect* rect, const TileLists& tl, int W, int H, int tiles_x,
                       int tiles_y, float cutoff, const float* dl_dout, float* partial, cudaStream_t stream);
void launch_reduce_chain2d(const float* params, int64_t N, int cov2d, const uint32_t* offsets, const uint32_t* counts,
                           const float* partial, float* dl_dparams, cudaStream_t stream);
// counters[0] += visited pairs, counters[1] += pairs inside the cutoff ellipse
void launch_count_pairs(const float4* rec, const TileLists& tl, int W, int H, int tiles_x, int tiles_y, float cutoff2,
                        const uint32_t* last, unsigned long long* counters, cudaStream_t stream);

// raster3d.cu: one warp per 8x8 quad, tiles in `order` (launch_tile_order); the backward one warp
// per (quad, chunk of kBwdChunk list entries), items from launch_tile_order, at most max_items
struct BwdChunks {
    const uint2* items;
    const uint32_t* n_items;
    const uint32_t* item_base;
    const float4* bnd;
    const float* cfin;
    unsigned int* counter;  // work counter of the persistent backward (zeroed at its launch)
};
void launch_blend3d(const BlendJob& job, int tiles_y, const uint32_t* order, cudaStream_t stream);
void launch_backward3d(const float4* rec, const PixRect* rect, const TileLists& tl, int W, int H, int tiles_x,
                       const BlendOpts3& o, const float* T_final, const uint32_t* last, const float* dl_dout,
                       float* grad_img, const BwdChunks& ch, int64_t max_items, cudaStream_t stream);
// Floats per primitive of the 3D image-plane gradient (mx my l11 l21 l22 fx fy phc c_r c_g c_b o,
// and under frequency map 2 kappa, in rows of 16 for 16-byte alignment).
inline int image_grad_stride3d(int fmode) { return fmode == 2 ? 16 : 12; }
void launch_chain3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float dilation, int fmode,
                    int sh_degree, const float4* rec, const float* grad_img, float* dl_dparams, cudaStream_t stream);

// batch.cu: one persistent launch over the tiles of up to kMaxBatchJobs frames; blocks take
// (frame, tile) items from counter[0], which the launcher resets.
constexpr int kMaxBatchJobs = 128;
void launch_blend_batch(const BlendJob* jobs, const int* tiles_y, int n_jobs, unsigned int* counter,
                        cudaStream_t stream);

// loss_noalloc.cu: the same loss with its scratch in a file-scope device array (no allocation)
int64_t l2_loss_noalloc_max_elements();
cudaError_t l2_loss_noalloc(const float* img, const float* target, int64_t n, float* loss, float* grad,
                            cudaStream_t stream);

// mlp.cu: the 6D deformation network (tcgen05 kernels, bfloat16 operands, fp32 accumulation)
struct MlpSizes {
    size_t act, scratch, out, theta16;  // bytes of the state buffers for N primitives
};
int64_t mlp_param_count();
MlpSizes mlp_sizes(int64_t N);
// Each returns "" on success, else a description of the failure.  A bounded device wait that runs
// out sets bit 1 of *err (the context's device error word).
std::string mlp_forward(const float* params3, int64_t N, float t, const float* theta, void* theta16, void* act,
                        float* d, float* params_out, unsigned int* err, cudaStream_t stream);
std::string mlp_backward(const float* params3, int64_t N, const void* theta16, const void* act, const float* d,
                         void* scratch, const float* g_out, float* g_theta, float* g_params3, int accumulate,
                         unsigned int* err, cudaStream_t stream);

// loss.cu
// partials: kLossBlocks floats, then one unsigned counter that is zero between calls (the last
// block to finish sums the partials and puts it back to zero)
void launch_l2_loss(const float* img, const float* target, int64_t n, float* loss, float* grad, float* partials,
                    cudaStream_t stream);
constexpr int kLossBlocks = 304;  // 2 x 152 SMs

}  // namespace wipes
