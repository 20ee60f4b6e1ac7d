// Per-tile forward rasterization, shared by the one-frame kernels (k_blend2d, k_blend3d) and the
// persistent batch kernel (k_blend_batch) so that a frame renders to the same bits alone or in a
// batch.  Each function is called by a whole 256-thread block for one 16x16 tile.
#pragma once

#include "common.cuh"

namespace wipes {

// Stage one tile-list entry: its record and, in `mask`, the warp sub-tiles its ellipse reaches.
__device__ __forceinline__ uint32_t stage_entry(const float4* __restrict__ rec, const PixRect* __restrict__ rect,
                                                const TileLists& tl, uint32_t i, int x0, int y0, float lim,
                                                float4& A, float4& B, float4& C) {
    const uint32_t prim = tl.inst_prim[tl.sorted[i]];
    A = rec[(size_t)prim * kRecF4 + 0];
    B = rec[(size_t)prim * kRecF4 + 1];
    C = rec[(size_t)prim * kRecF4 + 2];
    return subtile_mask_ellipse(A, B.x, rect[prim], x0, y0, lim);
}

// Forward.  Warp w of the tile's block owns an 8x4 pixel sub-tile (two columns of sub-tiles by
// four rows).  When a batch of the tile list is staged, each thread marks which sub-tiles its
// primitive's cutoff ellipse reaches; a warp then visits only the primitives marked for it.  The
// test is conservative (rect_touched), so skipping is exact.
__device__ __forceinline__ void blend2d_tile(const BlendJob& job, int tile) {
    const float4* __restrict__ rec = job.rec;
    const PixRect* __restrict__ rect = job.rect;
    const TileLists& tl = job.tl;
    const int W = job.W, H = job.H, tiles_x = job.tiles_x;
    const float cutoff2 = job.o.cutoff2, lim = job.o.lim;
    float* __restrict__ out = job.out;
    __shared__ float4 s_a[kTilePixels];  // mx my l11 l21
    __shared__ float4 s_b[kTilePixels];  // l22 fx fy phc
    __shared__ float4 s_c[kTilePixels];  // c_r c_g c_b o
    __shared__ uint8_t s_mask[kTilePixels];
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const int u = x0 + (warp & 1) * 8 + (lane & 7);
    const int v = y0 + (warp >> 1) * 4 + (lane >> 3);
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = tl.ranges[tile];
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            float4 A, B, C;
            s_mask[threadIdx.x] = (uint8_t)stage_entry(rec, rect, tl, b0 + threadIdx.x, x0, y0, lim, A, B, C);
            s_a[threadIdx.x] = A;
            s_b[threadIdx.x] = B;
            s_c[threadIdx.x] = C;
        }
        __syncthreads();
        // two-level summation: a batch-local partial sum per channel, added once per batch
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int c = 0; c < n; c += 32) {
            const uint32_t m = c + lane < n ? s_mask[c + lane] : 0u;
            uint32_t bal = __ballot_sync(0xffffffffu, (m >> warp) & 1u);
            while (bal) {
                const int j = c + __ffs(bal) - 1;
                bal &= bal - 1u;
                const float4 A = s_a[j];
                const float4 B = s_b[j];
                const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
                if (q <= cutoff2) {
                    const float dx = px - A.x, dy = py - A.y;
                    const float G = ex2_approx(q * kNegHalfLog2e);
                    const float t = fmaf(B.y, dx, fmaf(B.z, dy, B.w));
                    const float wv = fmaf(0.5f, cos_approx(reduced_angle(t)), 0.5f) * G;
                    const float4 C = s_c[j];
                    a0 = fmaf(C.x, wv, a0);
                    a1 = fmaf(C.y, wv, a1);
                    a2 = fmaf(C.z, wv, a2);
                }
            }
        }
        c0 += a0;
        c1 += a1;
        c2 += a2;
    }
    if (u < W && v < H) {
        float* o = out + ((size_t)v * W + u) * 3;
        o[0] = c0;
        o[1] = c1;
        o[2] = c2;
    }
}


// Forward.  As in 2D, warp w owns an 8x4 pixel sub-tile and visits only the staged primitives
// whose covered pixel range touches it; positions in the tile list are counted from the list
// start, so the per-pixel last-contributor index does not depend on the culling.
__device__ __forceinline__ void blend3d_tile(const BlendJob& job, int tile) {
    const float4* __restrict__ rec = job.rec;
    const PixRect* __restrict__ rect = job.rect;
    const TileLists& tl = job.tl;
    const int W = job.W, H = job.H, tiles_x = job.tiles_x;
    const BlendOpts3& o = job.o;
    float* __restrict__ out = job.out;
    float* __restrict__ T_final = job.T_final;
    uint32_t* __restrict__ last = job.last;
    __shared__ float4 s_a[kTilePixels];
    __shared__ float4 s_b[kTilePixels];
    __shared__ float4 s_c[kTilePixels];
    __shared__ uint8_t s_mask[kTilePixels];
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const int u = x0 + (warp & 1) * 8 + (lane & 7);
    const int v = y0 + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = u < W && v < H;
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = tl.ranges[tile];
    bool done = !inside;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    uint32_t last_contrib = 0;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        if ((int)threadIdx.x < n) {
            const uint32_t id = tl.inst_prim[tl.sorted[b0 + threadIdx.x]];
            const float4 A = rec[(size_t)id * kRecF4 + 0];
            const float4 B = rec[(size_t)id * kRecF4 + 1];
            s_a[threadIdx.x] = A;
            s_b[threadIdx.x] = B;
            s_c[threadIdx.x] = rec[(size_t)id * kRecF4 + 2];
            s_mask[threadIdx.x] = (uint8_t)subtile_mask_ellipse(A, B.x, rect[id], x0, y0, o.lim);
        }
        __syncthreads();
        for (int c = 0; c < n; c += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const uint32_t m = c + lane < n ? s_mask[c + lane] : 0u;
            uint32_t bal = __ballot_sync(0xffffffffu, (m >> warp) & 1u);
            while (bal) {
                const int j = c + __ffs(bal) - 1;
                bal &= bal - 1u;
                if (done) continue;
                const float4 A = s_a[j];
                const float4 B = s_b[j];
                const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
                if (!(q <= o.cutoff2)) continue;
                const float dx = px - A.x, dy = py - A.y;
                const float G = ex2_approx(q * kNegHalfLog2e);
                const float w = fmaf(0.5f, cos_approx(reduced_angle(fmaf(B.y, dx, fmaf(B.z, dy, B.w)))), 0.5f) * G;
                const float4 C = s_c[j];
                const float alpha = fminf(o.alpha_max, C.w * w);
                if (alpha < o.alpha_min) continue;
                const float test_T = T * (1.f - alpha);
                if (test_T < o.T_min) { done = true; continue; }
                const float wt = alpha * T;
                c0 = fmaf(C.x, wt, c0);
                c1 = fmaf(C.y, wt, c1);
                c2 = fmaf(C.z, wt, c2);
                T = test_T;
                last_contrib = b0 - range.x + (uint32_t)j + 1u;
            }
        }
    }
    if (inside) {
        const size_t pix = (size_t)v * W + u;
        out[pix * 3 + 0] = fmaf(T, o.bg[0], c0);
        out[pix * 3 + 1] = fmaf(T, o.bg[1], c1);
        out[pix * 3 + 2] = fmaf(T, o.bg[2], c2);
        T_final[pix] = T;
        last[pix] = last_contrib;
    }
}


}  // namespace wipes
