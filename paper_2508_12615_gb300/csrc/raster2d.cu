// 2D image task: summed wavelet field C(x) = sum_i c_i W_i(x) (Eq. 4 with the wavelet of Eq. 5,
// Sec. 4.3) over sorted tile lists, and its explicit backward (Sec. 1).
//
// Forward: one 256-thread block per 16x16 tile, one pixel per thread; the tile's primitives are
// staged through shared memory in batches of 256.  Backward: the field is a plain sum, so the
// gradient of each (tile, primitive) pair is independent of every other pair; one warp takes one
// pair, walks the pixels of the primitive's covered range inside the tile, reduces its partial
// gradient in registers and writes it to the pair's emission slot.  A second kernel sums the
// slots of each primitive (contiguous in emission order) and chains them to the record's
// parameters: deterministic, no atomics.
#include "common.cuh"

namespace wipes {
namespace {

constexpr float kNegHalfLog2e = -0.7213475204444817f;  // -log2(e) / 2

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

// phase argument reduced to [-pi, pi]: 2 pi (t - rint(t)) with t in cycles
__device__ __forceinline__ float reduced_angle(float t) { return (t - rintf(t)) * kTwoPi; }

__global__ void __launch_bounds__(kTilePixels) k_blend2d(const float4* __restrict__ rec,
                                                         const uint32_t* __restrict__ sorted_prims,
                                                         const uint2* __restrict__ ranges, int W, int H, int tiles_x,
                                                         float cutoff2, float* __restrict__ out) {
    __shared__ float4 s_a[kTilePixels];  // mx my l11 l21
    __shared__ float4 s_b[kTilePixels];  // l22 fx fy phc
    __shared__ float4 s_c[kTilePixels];  // c_r c_g c_b o
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int u = tx * kTile + (threadIdx.x & (kTile - 1));
    const int v = ty * kTile + (threadIdx.x / kTile);
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = ranges[tile];
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        __syncthreads();
        if ((int)threadIdx.x < n) {
            const uint32_t id = sorted_prims[b0 + threadIdx.x];
            s_a[threadIdx.x] = rec[(size_t)id * kRecF4 + 0];
            s_b[threadIdx.x] = rec[(size_t)id * kRecF4 + 1];
            s_c[threadIdx.x] = rec[(size_t)id * kRecF4 + 2];
        }
        __syncthreads();
        // two-level summation: a batch-local partial sum per channel, added once per batch
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int j = 0; j < n; ++j) {
            const float4 A = s_a[j];
            const float4 B = s_b[j];
            const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
            if (q <= cutoff2) {
                const float dx = px - A.x, dy = py - A.y;
                const float G = ex2_approx(q * kNegHalfLog2e);
                const float t = fmaf(B.y, dx, fmaf(B.z, dy, B.w));
                const float w = fmaf(0.5f, cos_approx(reduced_angle(t)), 0.5f) * G;
                const float4 C = s_c[j];
                a0 = fmaf(C.x, w, a0);
                a1 = fmaf(C.y, w, a1);
                a2 = fmaf(C.z, w, a2);
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

// Partial gradient slot layout (12 floats): mx my l11 l21 l22 fx fy phc c_r c_g c_b 0
constexpr int kSlot = 12;

__global__ void __launch_bounds__(kTilePixels) k_backward2d(const float4* __restrict__ rec,
                                                            const PixRect* __restrict__ rect,
                                                            const uint32_t* __restrict__ offsets,
                                                            const uint32_t* __restrict__ sorted_prims,
                                                            const uint2* __restrict__ ranges, int W, int H, int tiles_x,
                                                            float cutoff2, const float* __restrict__ dl_dout,
                                                            float* __restrict__ partial) {
    __shared__ float s_g[kTilePixels * 3];
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const int u = tx * kTile + (threadIdx.x & (kTile - 1));
        const int v = ty * kTile + (threadIdx.x / kTile);
        const bool in = u < W && v < H;
        const float* g = dl_dout + ((size_t)v * W + u) * 3;
        s_g[threadIdx.x * 3 + 0] = in ? g[0] : 0.f;
        s_g[threadIdx.x * 3 + 1] = in ? g[1] : 0.f;
        s_g[threadIdx.x * 3 + 2] = in ? g[2] : 0.f;
    }
    __syncthreads();
    const uint2 range = ranges[tile];
    for (uint32_t i = range.x + warp; i < range.y; i += kTilePixels / 32) {
        const uint32_t prim = sorted_prims[i];
        const float4 A = rec[(size_t)prim * kRecF4 + 0];  // mx my l11 l21
        const float4 B = rec[(size_t)prim * kRecF4 + 1];  // l22 fx fy phc
        const float4 C = rec[(size_t)prim * kRecF4 + 2];  // colour
        const PixRect r = rect[prim];
        const int ux0 = max(r.u0, tx * kTile), ux1 = min(r.u1, tx * kTile + kTile - 1);
        const int vy0 = max(r.v0, ty * kTile), vy1 = min(r.v1, ty * kTile + kTile - 1);
        const int w = ux1 - ux0 + 1, area = w * (vy1 - vy0 + 1);
        const uint32_t slot = offsets[prim] + (uint32_t)((ty - r.v0 / kTile) * (r.u1 / kTile - r.u0 / kTile + 1) +
                                                         (tx - r.u0 / kTile));
        const uint32_t mdiv = (65536u + (uint32_t)w - 1u) / (uint32_t)w;  // exact k / w for k < 256
        float g_mx = 0.f, g_my = 0.f, g_l11 = 0.f, g_l21 = 0.f, g_l22 = 0.f, g_fx = 0.f, g_fy = 0.f, g_ph = 0.f;
        float g_c0 = 0.f, g_c1 = 0.f, g_c2 = 0.f;
        for (int k = lane; k < area; k += 32) {
            const int lv = (int)(((uint32_t)k * mdiv) >> 16);
            const int u = ux0 + (k - lv * w), v = vy0 + lv;
            const float px = (float)u + 0.5f, py = (float)v + 0.5f;
            const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
            if (q <= cutoff2) {
                const float dx = px - A.x, dy = py - A.y;
                const float a = fmaf(A.z, dx, A.w * dy), b = B.x * dy;
                const float G = ex2_approx(q * kNegHalfLog2e);
                const float ang = reduced_angle(fmaf(B.y, dx, fmaf(B.z, dy, B.w)));
                const float cs = cos_approx(ang), sn = sin_approx(ang);
                const float Wv = fmaf(0.5f, cs, 0.5f) * G;
                const float* g = s_g + ((v - ty * kTile) * kTile + (u - tx * kTile)) * 3;
                const float gW = fmaf(g[0], C.x, fmaf(g[1], C.y, g[2] * C.z));
                const float gq2 = -gW * Wv;       // 2 dL/dq  (dW/dq = -W/2)
                const float gt = -kPi * gW * G * sn;  // dL/dt, t in cycles
                const float ga = gq2 * a, gb = gq2 * b;
                g_l11 = fmaf(ga, dx, g_l11);
                g_l21 = fmaf(ga, dy, g_l21);
                g_l22 = fmaf(gb, dy, g_l22);
                g_mx -= fmaf(ga, A.z, gt * B.y);
                g_my -= fmaf(ga, A.w, fmaf(gb, B.x, gt * B.z));
                g_fx = fmaf(gt, dx, g_fx);
                g_fy = fmaf(gt, dy, g_fy);
                g_ph += gt;
                g_c0 = fmaf(g[0], Wv, g_c0);
                g_c1 = fmaf(g[1], Wv, g_c1);
                g_c2 = fmaf(g[2], Wv, g_c2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            g_mx += __shfl_xor_sync(0xffffffffu, g_mx, o);
            g_my += __shfl_xor_sync(0xffffffffu, g_my, o);
            g_l11 += __shfl_xor_sync(0xffffffffu, g_l11, o);
            g_l21 += __shfl_xor_sync(0xffffffffu, g_l21, o);
            g_l22 += __shfl_xor_sync(0xffffffffu, g_l22, o);
            g_fx += __shfl_xor_sync(0xffffffffu, g_fx, o);
            g_fy += __shfl_xor_sync(0xffffffffu, g_fy, o);
            g_ph += __shfl_xor_sync(0xffffffffu, g_ph, o);
            g_c0 += __shfl_xor_sync(0xffffffffu, g_c0, o);
            g_c1 += __shfl_xor_sync(0xffffffffu, g_c1, o);
            g_c2 += __shfl_xor_sync(0xffffffffu, g_c2, o);
        }
        float val = 0.f;
        val = lane == 0 ? g_mx : val;
        val = lane == 1 ? g_my : val;
        val = lane == 2 ? g_l11 : val;
        val = lane == 3 ? g_l21 : val;
        val = lane == 4 ? g_l22 : val;
        val = lane == 5 ? g_fx : val;
        val = lane == 6 ? g_fy : val;
        val = lane == 7 ? g_ph : val;
        val = lane == 8 ? g_c0 : val;
        val = lane == 9 ? g_c1 : val;
        val = lane == 10 ? g_c2 : val;
        if (lane < kSlot) partial[(size_t)slot * kSlot + lane] = val;
    }
}

// One warp per primitive: sum its slots, then chain (mx, my, L, f, phc, c) to the record
// mu, s, theta, f, phi, c.  L depends on (theta, s_x, s_y) through
// A = c^2/sx^2 + s^2/sy^2, B = c s (1/sx^2 - 1/sy^2), l11 = sqrt(A), l21 = B/l11, l22 = 1/(sx sy l11).
__global__ void __launch_bounds__(256) k_reduce_chain2d(const float* __restrict__ params, int64_t N,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint32_t* __restrict__ counts,
                                                        const float* __restrict__ partial,
                                                        float* __restrict__ dl_dparams) {
    const int64_t prim = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (prim >= N) return;
    const uint32_t off = offsets[prim], cnt = counts[prim];
    float acc[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) acc[k] = 0.f;
    for (uint32_t j = lane; j < cnt; j += 32) {
        const float4* s = reinterpret_cast<const float4*>(partial + (size_t)(off + j) * kSlot);
        const float4 x0 = s[0], x1 = s[1], x2 = s[2];
        acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
        acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
        acc[8] += x2.x; acc[9] += x2.y; acc[10] += x2.z;
    }
#pragma unroll
    for (int k = 0; k < 11; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane != 0) return;
    const float* p = params + prim * WIPES_P2D;
    float* out = dl_dparams + prim * WIPES_P2D;
    const float sx = p[2], sy = p[3];
    float s, c;
    sincosf(p[4], &s, &c);
    const float ix = 1.0f / (sx * sx), iy = 1.0f / (sy * sy);
    const float A = c * c * ix + s * s * iy;
    const float B = c * s * (ix - iy);
    const float l11 = sqrtf(A), l21 = B / l11, l22 = 1.0f / (sx * sy * l11);
    // partial derivatives of A and B
    const float dA_th = -2.0f * B, dA_sx = -2.0f * c * c * ix / sx, dA_sy = -2.0f * s * s * iy / sy;
    const float dB_th = (c * c - s * s) * (ix - iy), dB_sx = -2.0f * c * s * ix / sx, dB_sy = 2.0f * c * s * iy / sy;
    const float h = 0.5f / l11;
    const float d11_th = dA_th * h, d11_sx = dA_sx * h, d11_sy = dA_sy * h;
    const float d21_th = (dB_th - l21 * d11_th) / l11;
    const float d21_sx = (dB_sx - l21 * d11_sx) / l11;
    const float d21_sy = (dB_sy - l21 * d11_sy) / l11;
    const float d22_th = -l22 * d11_th / l11;
    const float d22_sx = -l22 * (1.0f / sx + d11_sx / l11);
    const float d22_sy = -l22 * (1.0f / sy + d11_sy / l11);
    const float g11 = acc[2], g21 = acc[3], g22 = acc[4];
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = g11 * d11_sx + g21 * d21_sx + g22 * d22_sx;
    out[3] = g11 * d11_sy + g21 * d21_sy + g22 * d22_sy;
    out[4] = g11 * d11_th + g21 * d21_th + g22 * d22_th;
    out[5] = acc[5];
    out[6] = acc[6];
    out[7] = acc[7] * kInvTwoPi;
    out[8] = acc[8];
    out[9] = acc[9];
    out[10] = acc[10];
#pragma unroll
    for (int k = 11; k < WIPES_P2D; ++k) out[k] = 0.f;
}

// Visited and inside-cutoff (pixel, primitive) pairs over the sorted tile lists.
__global__ void __launch_bounds__(kTilePixels) k_count_pairs(const float4* __restrict__ rec,
                                                             const uint32_t* __restrict__ sorted_prims,
                                                             const uint2* __restrict__ ranges, int W, int H,
                                                             int tiles_x, float cutoff2,
                                                             unsigned long long* __restrict__ counters) {
    __shared__ unsigned long long s_sum[2];
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int u = tx * kTile + (threadIdx.x & (kTile - 1));
    const int v = ty * kTile + (threadIdx.x / kTile);
    const bool in = u < W && v < H;
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = ranges[tile];
    unsigned long long inside = 0;
    if (threadIdx.x < 2) s_sum[threadIdx.x] = 0ull;
    __syncthreads();
    if (in) {
        for (uint32_t i = range.x; i < range.y; ++i) {
            const uint32_t id = sorted_prims[i];
            const float4 A = rec[(size_t)id * kRecF4 + 0];
            const float l22 = rec[(size_t)id * kRecF4 + 1].x;
            inside += mahalanobis2(px, py, A.x, A.y, A.z, A.w, l22) <= cutoff2;
        }
        atomicAdd(&s_sum[0], (unsigned long long)(range.y - range.x));
        atomicAdd(&s_sum[1], inside);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&counters[0], s_sum[0]);
        atomicAdd(&counters[1], s_sum[1]);
    }
}

}  // namespace

void launch_blend2d(const float4* rec, const uint32_t* sorted_prims, const uint2* ranges, int W, int H, int tiles_x,
                    int tiles_y, float cutoff2, float* out, cudaStream_t stream) {
    k_blend2d<<<tiles_x * tiles_y, kTilePixels, 0, stream>>>(rec, sorted_prims, ranges, W, H, tiles_x, cutoff2, out); count_launches(1);
}

void launch_backward2d(const float4* rec, const PixRect* rect, const uint32_t* offsets, const uint32_t* sorted_prims,
                       const uint2* ranges, int W, int H, int tiles_x, int tiles_y, float cutoff2,
                       const float* dl_dout, float* partial, cudaStream_t stream) {
    k_backward2d<<<tiles_x * tiles_y, kTilePixels, 0, stream>>>(rec, rect, offsets, sorted_prims, ranges, W, H,
                                                                 tiles_x, cutoff2, dl_dout, partial); count_launches(1);
}

void launch_count_pairs(const float4* rec, const uint32_t* sorted_prims, const uint2* ranges, int W, int H,
                        int tiles_x, int tiles_y, float cutoff2, unsigned long long* counters, cudaStream_t stream) {
    k_count_pairs<<<tiles_x * tiles_y, kTilePixels, 0, stream>>>(rec, sorted_prims, ranges, W, H, tiles_x, cutoff2,
                                                                  counters); count_launches(1);
}

void launch_reduce_chain2d(const float* params, int64_t N, const uint32_t* offsets, const uint32_t* counts,
                           const float* partial, float* dl_dparams, cudaStream_t stream) {
    if (N == 0) return;
    k_reduce_chain2d<<<ceil_div(N * 32, 256), 256, 0, stream>>>(params, N, offsets, counts, partial, dl_dparams); count_launches(1);
}

}  // namespace wipes
