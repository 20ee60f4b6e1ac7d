// Internal definitions shared by the kernels and the C ABI of the wavelet rasterizer (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wipes.h"

namespace wipes {

constexpr int kTile = WIPES_TILE;
constexpr int kTilePixels = kTile * kTile;
constexpr float kExtMargin = 1.0009765625f;  // 1 + 2^-10: footprint half-extent safety factor
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kInvTwoPi = 0.15915494309189535f;
constexpr float kPi = 3.141592653589793f;

// Projected record (4 x float4 = 64 bytes per primitive), written by the footprint kernels:
//   [0] mx, my, l11, l21    centre (px) and lower Cholesky factor L of Sigma'^-1 = L L^T
//   [1] l22, fx, fy, phc    frequency (cycles/px) and phase (cycles)
//   [2] c_r, c_g, c_b, o    colour and opacity (2D: o = 1)
//   [3] ex, ey, depth, 0    half extents of the cutoff ellipse (px) and camera z (3D)
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
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Phase t given in cycles, reduced to an angle in [-pi, pi]: 2 pi (t - rint(t)).
__device__ __forceinline__ float reduced_angle(float t) { return (t - rintf(t)) * kTwoPi; }

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

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Library-wide count of kernel launches (every launcher adds the kernels it enqueues).
void count_launches(int n);

// Launchers implemented in the kernel translation units (all enqueue on `stream`).

// footprint.cu
void launch_footprint2d(const float* params, int64_t N, int W, int H, float cutoff, float4* rec, PixRect* rect,
                        uint32_t* counts, uint32_t* depth_keys, cudaStream_t stream);
void launch_footprint3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float cutoff,
                        float dilation, float4* rec, PixRect* rect, uint32_t* counts, uint32_t* depth_keys,
                        cudaStream_t stream);
void launch_deform6d(const float* params6, int64_t N, float t, float* params3, cudaStream_t stream);
void launch_deform6d_backward(const float* params6, int64_t N, float t, const float* g3, float* g6, int accumulate,
                              cudaStream_t stream);

// binning.cu
// Per-block sums of counts (in the order given by perm, or primitive order if perm is null).
constexpr int kScanBlockElems = 1024;
void launch_block_sums(const uint32_t* counts, const uint32_t* perm, int64_t n, unsigned long long* block_sums,
                       cudaStream_t stream);
// Exclusive scan of nb block sums in place; total written to *total.
void launch_scan_block_sums(unsigned long long* block_sums, int nb, unsigned long long* total, cudaStream_t stream);
// Emit (tile id, primitive) pairs in scan order; offsets[prim] = first instance index of prim.
void launch_emit(const uint32_t* counts, const uint32_t* perm, int64_t n, const PixRect* rect,
                 const unsigned long long* block_offsets, int tiles_x, uint32_t* keys, uint32_t* vals,
                 uint32_t* offsets, cudaStream_t stream);
void launch_tile_ranges(const uint32_t* sorted_keys, int64_t n, uint2* ranges, int n_tiles, cudaStream_t stream);
void launch_iota(uint32_t* v, int64_t n, cudaStream_t stream);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).  Uses (keys[0], vals[0]) as
// input and (keys[1], vals[1]) as ping-pong space; returns which buffer index holds the result.
// `hist` must hold radix_hist_words(n) words.
int64_t radix_hist_words(int64_t n);
int radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits, uint32_t* hist, cudaStream_t stream);

// raster2d.cu
void launch_blend2d(const float4* rec, const PixRect* rect, const uint32_t* sorted_prims, const uint2* ranges, int W,
                    int H, int tiles_x, int tiles_y, float cutoff2, float* out, cudaStream_t stream);
void launch_backward2d(const float4* rec, const PixRect* rect, const uint32_t* offsets, const uint32_t* sorted_prims,
                       const uint2* ranges, int W, int H, int tiles_x, int tiles_y, float cutoff2,
                       const float* dl_dout, float* partial, cudaStream_t stream);
void launch_reduce_chain2d(const float* params, int64_t N, const uint32_t* offsets, const uint32_t* counts,
                           const float* partial, float* dl_dparams, cudaStream_t stream);
// counters[0] += visited pairs, counters[1] += pairs inside the cutoff ellipse
void launch_count_pairs(const float4* rec, const uint32_t* sorted_prims, const uint2* ranges, int W, int H,
                        int tiles_x, int tiles_y, float cutoff2, unsigned long long* counters, cudaStream_t stream);

// raster3d.cu
struct BlendOpts3 {
    float cutoff2, alpha_min, alpha_max, T_min;
    float bg[3];
};
void launch_blend3d(const float4* rec, const PixRect* rect, const uint32_t* sorted_prims, const uint2* ranges, int W,
                    int H, int tiles_x, int tiles_y, const BlendOpts3& o, float* out, float* T_final, uint32_t* last,
                    cudaStream_t stream);
void launch_backward3d(const float4* rec, const PixRect* rect, const uint32_t* sorted_prims, const uint2* ranges,
                       int W, int H, int tiles_x, int tiles_y, const BlendOpts3& o, const float* T_final,
                       const uint32_t* last, const float* dl_dout, float* grad_img, cudaStream_t stream);
void launch_chain3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float dilation,
                    const float4* rec, const float* grad_img, float* dl_dparams, cudaStream_t stream);

// loss.cu
void launch_l2_loss(const float* img, const float* target, int64_t n, float* loss, float* grad, float* partials,
                    cudaStream_t stream);
constexpr int kLossBlocks = 304;  // 2 x 152 SMs

}  // namespace wipes
