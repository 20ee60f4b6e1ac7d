// 2D image task: summed wavelet field C(x) = sum_i c_i W_i(x) (Eq. 4 with the wavelet of Eq. 5,
// Sec. 4.3) over sorted tile lists, and its explicit backward (Sec. 1).
//
// Forward: one 256-thread block per 16x16 tile, one pixel per thread; the tile's primitives are
// staged through shared memory in batches of 256.  Backward: the field is a plain sum, so the
// gradient of each (tile, primitive) pair is independent of every other pair; one warp takes one
// pair, walks the pixels of the cutoff ellipse inside the tile, reduces its partial gradient in
// registers and writes it to the pair's emission slot.  A second kernel sums the slots of each
// primitive (contiguous in emission order) and chains them to the record's parameters:
// deterministic, no atomics.
#include "blend_tile.cuh"

namespace wipes {
namespace {

__global__ void __launch_bounds__(kTilePixels) k_blend2d(BlendJob job) { pdl_enter(); blend2d_tile(job, blockIdx.x); }

// Partial gradient slot layout (12 floats): mx my l11 l21 l22 fx fy phc c_r c_g c_b 0
constexpr int kSlot = 12;

// Reduce-scatter within each half-warp: 16 values over its 16 lanes; lane h of a half ends with the
// half's total of value h.
__device__ __forceinline__ float half_reduce_scatter16(float v[16]) {
    const int hl = threadIdx.x & 15;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        const bool hi = hl & off;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = hi ? v[i] : v[off + i];
            const float keep = hi ? v[off + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

// Reduce-scatter within each group of 4 lanes: 16 values over its 4 lanes; lane q of a group ends
// with the group's totals of values 4q .. 4q + 3 in v[0 .. 3].
__device__ __forceinline__ void group4_reduce_scatter16(float v[16]) {
    const int q = threadIdx.x & 3;
#pragma unroll
    for (int off = 2, half = 8; off >= 1; off >>= 1, half >>= 1) {
        const bool hi = q & off;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = hi ? v[i] : v[half + i];
            const float keep = hi ? v[half + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
}

// The 2D backward's pairs are independent of one another, so a tile's staged batches of 256 list
// entries are shared out over kBwdSplit blocks: more, smaller blocks leave a shorter tail.
constexpr int kBwdSplit = 2;

// Backward.  The tile's dL/dimage sits in shared memory by pixel pairs: pair (k, r, c) holds the
// pixels (c, r) and (c, r + 4) of the 8x8 quadrant k.  Batches of the tile list
// are staged with the mask of the quadrants that each pair's cutoff ellipse reaches, and ordered
// by the number of those quadrants.  Each group of 4 lanes takes one (tile, primitive) pair, so a
// warp works on eight pairs that reach equally many quadrants.  In a quadrant, lane r of a group
// walks the row pair (r, r + 4) across the eight columns (from column 0 or from column 7, by the
// parity of the pair's staged position) in packed f32x2 arithmetic:
//  - dy and b = l22 dy are constant along the walk, so the Mahalanobis distance costs two FMAs
//    per pixel pair (the same operations as mahalanobis2(), so the cutoff decision is the same);
//  - the oscillation's phasor (cos, sin)(2 pi t) is evaluated once at the first column and
//    advanced column by column by the rotation through +-2 pi fx (sincospif of 2 fx: accurate to
//    an ulp or so, so that seven steps stay within the MUFU cos/sin error);
//  - the cutoff enters the exponent: outside, the argument is S (cutoff^2 - q) <= -256 and ex2
//    returns 0, inside it is -q log2(e) / 2 (S a power of two that makes the scaled gap of any
//    binary32 q > cutoff^2 at least 256).
// Per pixel inside the cutoff a lane accumulates the factored sums
//   sum ga, sum gb, sum gt, sum ga dx, sum ga dy, sum gb dy, sum gt dx, sum gt dy, sum g W
// (ga = 2 dL/dq a, gb = 2 dL/dq b, gt = dL/dt, with q = a^2 + b^2, a = l11 dx + l21 dy,
// b = l22 dy, t the phase in cycles), those with a factor constant along a walk (b, dy) once per
// walk.  The pair's gradient follows from them after one reduction over the group's 4 lanes, since
// L, f and the centre are constant over the pair.  The colours are staged halved and the
// modulation taken as G (1 + cos), which saves the 1/2 of W per pixel; the sums are taken of
// -ga, -gb and -gt / (2 pi) and scaled once per pair.
__global__ void __launch_bounds__(kTilePixels, 3) k_backward2d(const float4* __restrict__ rec,
                                                            const PixRect* __restrict__ rect, TileLists tl, int W,
                                                            int H, int tiles_x, float cutoff2, float lim,
                                                            float cut_scale, const float* __restrict__ dl_dout,
                                                            float* __restrict__ partial) {
    pdl_enter();
    // (g_r, g_g) and g_b pairs by pixel pair, column-swizzled: pair (k, r, c) at slot
    // 32 k + 8 r + ((c + 2 r) & 7), so that the four rows of a walk read four different bank groups
    __shared__ ulonglong2 s_g[kTilePixels / 2];
    __shared__ unsigned long long s_gb[kTilePixels / 2];
    // staged entry k: (mx, my) (l11, l21) (l22, fx) (fy, phc) (c_r, c_g) / 2, each value twice, then
    // (c_b / 2, c_b / 2) and the column rotation (cos 2 pi fx, sin 2 pi fx)
    __shared__ ulonglong2 s_e[6][kTilePixels];
    __shared__ uint32_t s_slot[kTilePixels];
    __shared__ uint8_t s_mask[kTilePixels];
    __shared__ uint16_t s_order[kTilePixels];  // staged entries, most quadrants first
    __shared__ uint32_t s_nq[5];               // staged entries that reach 0 .. 4 quadrants
    // block (part, tile): the tile's staged batches part, part + kBwdSplit, ...; the first parts of
    // all tiles come first
    const int n_tiles = (int)(gridDim.x / kBwdSplit);
    const int tile = (int)blockIdx.x % n_tiles, part = (int)blockIdx.x / n_tiles;
    const uint2 range = tl.ranges[tile];
    if (range.x + (uint32_t)part * kTilePixels >= range.y) return;  // the whole block: no batch of its own
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ql = lane & 3, grp = lane >> 2;
    __shared__ __align__(16) float s_red[kTilePixels / 32][8][16];  // per warp and group: the pair's 16 sums
    if (threadIdx.x < kTilePixels / 2) {
        // pixel pair p = threadIdx.x: quadrant k = p >> 5, column p & 7, rows (p >> 3) & 3 and + 4
        const int k = threadIdx.x >> 5;
        const int u = x0 + (k & 1) * 8 + (lane & 7);
        const int v = y0 + (k >> 1) * 8 + (lane >> 3);
        float g0[3] = {0.f, 0.f, 0.f}, g1[3] = {0.f, 0.f, 0.f};
        if (u < W && v < H) {
            const float* g = dl_dout + ((size_t)v * W + u) * 3;
            g0[0] = g[0], g0[1] = g[1], g0[2] = g[2];
        }
        if (u < W && v + 4 < H) {
            const float* g = dl_dout + ((size_t)(v + 4) * W + u) * 3;
            g1[0] = g[0], g1[1] = g[1], g1[2] = g[2];
        }
        const int r = (threadIdx.x >> 3) & 3, slot = (threadIdx.x & ~7) | (((threadIdx.x & 7) + 2 * r) & 7);
        s_g[slot] = make_ulonglong2(f2_pack(g0[0], g1[0]).r, f2_pack(g0[1], g1[1]).r);
        s_gb[slot] = f2_pack(g0[2], g1[2]).r;
    }
    if (threadIdx.x < 5) s_nq[threadIdx.x] = 0u;
    const f2 K = f2_dup(kNegHalfLog2e);
    const f2 NEG_S = f2_dup(-cut_scale), CUT_S = f2_dup(cutoff2 * cut_scale);  // exact: a power-of-two scale
    for (uint32_t b0 = range.x + (uint32_t)part * kTilePixels; b0 < range.y; b0 += kBwdSplit * kTilePixels) {
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        __syncthreads();
        int my_q = 0;
        uint32_t my_rank = 0u;
        if ((int)threadIdx.x < n) {
            const uint32_t e = tl.sorted[b0 + threadIdx.x];
            const uint32_t prim = tl.prim[b0 + threadIdx.x];
            const float4 A = rec[(size_t)prim * kRecF4 + 0];
            const float4 B = rec[(size_t)prim * kRecF4 + 1];
            const float4 C = rec[(size_t)prim * kRecF4 + 2];
            s_e[0][threadIdx.x] = dup2(A.x, A.y);
            s_e[1][threadIdx.x] = dup2(A.z, A.w);
            s_e[2][threadIdx.x] = dup2(B.x, B.y);
            s_e[3][threadIdx.x] = dup2(B.z, B.w);
            s_e[4][threadIdx.x] = dup2(0.5f * C.x, 0.5f * C.y);
            float srot, crot;
            sincospif(2.0f * B.y, &srot, &crot);  // once per staged entry, for every lane that walks it
            s_e[5][threadIdx.x] = make_ulonglong2(f2_dup(0.5f * C.z).r, f2_pack(crot, srot).r);
            const uint32_t m = quadrant_mask_ellipse(A, B.x, rect[prim], x0, y0, lim);
            s_mask[threadIdx.x] = (uint8_t)m;
            s_slot[threadIdx.x] = e;
            my_q = __popc(m);
            my_rank = atomicAdd(&s_nq[my_q], 1u);
        }
        __syncthreads();
        if ((int)threadIdx.x < n) {
            uint32_t pos = my_rank;
            for (int q = 4; q > my_q; --q) pos += s_nq[q];
            s_order[pos] = (uint16_t)threadIdx.x;
        }
        __syncthreads();
        if (threadIdx.x < 5) s_nq[threadIdx.x] = 0u;  // read by no one until the next batch's counts
        const int ngroups = (n + 7) >> 3;
        for (int pi = warp; pi < ngroups; pi += kTilePixels / 32) {
            const int idx = 8 * pi + grp;
            const bool has = idx < n;
            const int j = has ? (int)s_order[idx] : 0;
            uint32_t mask = has ? (uint32_t)s_mask[j] : 0u;
            // pairs at even staged positions walk the columns 0 -> 7, odd ones 7 -> 0: the walk (and
            // so the summation order) is a property of the pair, and the groups of a warp, about
            // half each way, spread their dL/dimage reads over all eight bank groups
            const int c0 = (j & 1) ? 7 : 0, cstep = (j & 1) ? -1 : 1;
            const float dir = (float)cstep;
            const f2 STEP = f2_dup(dir);
            // per pixel pair (packed): 3 -ga dx, 6 -gt' dx, 8..10 2 g W; per walk (scalar, both
            // pixels summed): 0 -ga, 1 -gb, 2 -gt', 4 -ga dy, 5 -gb dy, 7 -gt' dy
            f2 acc3 = f2_dup(0.f), acc6 = acc3, acc8 = acc3, acc9 = acc3, acc10 = acc3;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s4 = 0.f, s5 = 0.f, s7 = 0.f;
            // the rotation of the phasor from one column to the next: 2 pi fx
            f2 CX, SX, NSX;
            {
                const f2 rot = ld_f2x2(&s_e[5][j]).y;  // (cos, sin)(2 pi fx), staged
                const float cx = f2_lo(rot), sx = f2_hi(rot);
                CX = f2_dup(cx), SX = f2_dup(dir * sx), NSX = f2_dup(-dir * sx);
            }
            while (__any_sync(0xffffffffu, mask != 0u)) {
                if (mask) {
                    const int k = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const f2x2 e0 = ld_f2x2_here(&s_e[0][j]), e1 = ld_f2x2_here(&s_e[1][j]);
                    const f2x2 e2 = ld_f2x2_here(&s_e[2][j]), e3 = ld_f2x2_here(&s_e[3][j]);
                    // integers below 2^24 are exact in binary32, so these equal (float)u + 0.5f
                    const float px0 = (float)(x0 + (k & 1) * 8 + c0) + 0.5f;
                    const float py = (float)(y0 + (k >> 1) * 8 + ql) + 0.5f;
                    const f2 DY = f2_sub(f2_pack(py, py + 4.0f), e0.y);
                    const f2 L21DY = f2_mul(e1.y, DY);
                    const f2 B = f2_mul(e2.x, DY);
                    const f2 BB = f2_mul(B, B);
                    f2 PX = f2_dup(px0);
                    f2 cs, sn;
                    {
                        const f2 ang = f2_reduced_angle(f2_fma(e2.y, f2_sub(PX, e0.x), f2_fma(e3.x, DY, e3.y)));
                        const float alo = f2_lo(ang), ahi = f2_hi(ang);
                        cs = f2_pack(cos_approx(alo), cos_approx(ahi));
                        sn = f2_pack(sin_approx(alo), sin_approx(ahi));
                    }
                    const f2x2 e4 = ld_f2x2_here(&s_e[4][j]);
                    const f2 CB = ld_f2x2_here(&s_e[5][j]).x;
                    f2 sa = f2_dup(0.f), sq = sa, st = sa;  // this walk's sums of ha, hq, ht
                    const int gbase = 32 * k + 8 * ql;
                    int gofs = c0 + 2 * ql;  // the column's slot in the swizzled row, before & 7
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        // the cutoff test in the operation order of mahalanobis2()
                        const f2 dx = f2_sub(PX, e0.x);
                        const f2 a = f2_fma(e1.x, dx, L21DY);
                        const f2 q = f2_fma(a, a, BB);
                        const f2 ex = f2_mul(q, K), cut = f2_fma(q, NEG_S, CUT_S);
                        const f2 G = f2_pack(ex2_approx(fminf(f2_lo(ex), f2_lo(cut))),
                                             ex2_approx(fminf(f2_hi(ex), f2_hi(cut))));
                        const f2 Wv = f2_fma(cs, G, G);  // 2 W
                        const f2x2 g01 = ld_f2x2(&s_g[gbase + (gofs & 7)]);
                        const f2 gb_{s_gb[gbase + (gofs & 7)]};
                        const f2 gW = f2_fma(g01.x, e4.x, f2_fma(g01.y, e4.y, f2_mul(gb_, CB)));  // g.c / 2
                        const f2 hq = f2_mul(gW, Wv);                  // -2 dL/dq
                        const f2 ht = f2_mul(G, f2_mul(gW, sn));      // -dL/dt / (2 pi), t in cycles
                        const f2 ha = f2_mul(hq, a);
                        sa = f2_add(sa, ha);
                        sq = f2_add(sq, hq);
                        st = f2_add(st, ht);
                        acc3 = f2_fma(ha, dx, acc3);
                        acc6 = f2_fma(ht, dx, acc6);
                        acc8 = f2_fma(g01.x, Wv, acc8);
                        acc9 = f2_fma(g01.y, Wv, acc9);
                        acc10 = f2_fma(gb_, Wv, acc10);
                        if (c < 7) {
                            PX = f2_add(PX, STEP);
                            gofs += cstep;
                            const f2 cs_next = f2_fma(sn, NSX, f2_mul(cs, CX));
                            sn = f2_fma(cs, SX, f2_mul(sn, CX));
                            cs = cs_next;
                        }
                    }
                    // b and dy are constant along the walk (recomputed: cheaper than holding them)
                    const f2 DY2 = f2_sub(f2_pack(py, py + 4.0f), ld_f2x2_here(&s_e[0][j]).y);
                    const f2 B2 = f2_mul(ld_f2x2_here(&s_e[2][j]).x, DY2);
                    const f2 hb = f2_mul(sq, B2), ady = f2_mul(sa, DY2), bdy = f2_mul(hb, DY2), tdy = f2_mul(st, DY2);
                    s0 += f2_lo(sa) + f2_hi(sa);
                    s1 += f2_lo(hb) + f2_hi(hb);
                    s2 += f2_lo(st) + f2_hi(st);
                    s4 += f2_lo(ady) + f2_hi(ady);
                    s5 += f2_lo(bdy) + f2_hi(bdy);
                    s7 += f2_lo(tdy) + f2_hi(tdy);
                }
            }
            // the lane's pixels, then the sums of ga, gb, gt from the scaled ones
            float sums[16] = {s0, s1, s2, f2_lo(acc3) + f2_hi(acc3), s4, s5, f2_lo(acc6) + f2_hi(acc6), s7,
                              f2_lo(acc8) + f2_hi(acc8), f2_lo(acc9) + f2_hi(acc9), f2_lo(acc10) + f2_hi(acc10),
                              0.f, 0.f, 0.f, 0.f, 0.f};
            sums[0] = -sums[0], sums[1] = -sums[1], sums[3] = -sums[3], sums[4] = -sums[4], sums[5] = -sums[5];
            sums[2] *= -kTwoPi, sums[6] *= -kTwoPi, sums[7] *= -kTwoPi;
            sums[8] *= 0.5f, sums[9] *= 0.5f, sums[10] *= 0.5f;
            // lane q of the group ends with the totals of sums 4q .. 4q + 3, which the group shares
            // through shared memory; lanes 0 .. 2 write slots 4q .. 4q + 3 of the pair
            group4_reduce_scatter16(sums);
            const int q4 = ql;
            float* red = s_red[warp][grp];
            *reinterpret_cast<float4*>(red + 4 * q4) = make_float4(sums[0], sums[1], sums[2], sums[3]);
            __syncwarp();
            if (has && q4 < 3) {
                const float sga = red[0], sgb = red[1], sgt = red[2];
                const f2x2 e1 = ld_f2x2(&s_e[1][j]), e2 = ld_f2x2(&s_e[2][j]);
                const float l11 = f2_lo(e1.x), l21 = f2_lo(e1.y), l22 = f2_lo(e2.x), fx = f2_lo(e2.y);
                const float fy = f2_lo(ld_f2x2(&s_e[3][j]).x);
                float val[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // slots 4 q4 + e: l11 <- ga dx (3), l21 <- ga dy (4), l22 <- gb dy (5), fx <- gt dx (6),
                    // fy <- gt dy (7), phc <- gt (2), colour 8..10
                    const int slot = 4 * q4 + e;
                    const int m = slot == 7 ? 2 : (slot >= 2 && slot <= 6 ? slot + 1 : slot);
                    val[e] = red[m];
                }
                if (q4 == 0) {
                    val[0] = -fmaf(l11, sga, fx * sgt);
                    val[1] = -fmaf(l21, sga, fmaf(l22, sgb, fy * sgt));
                }
                if (q4 == 2) val[3] = 0.f;  // slot 11 is padding
                *reinterpret_cast<float4*>(partial + (size_t)s_slot[j] * kSlot + 4 * q4) =
                    make_float4(val[0], val[1], val[2], val[3]);
            }
            __syncwarp();  // the group's sums are read before the next pass overwrites them
        }
    }
}

// The RS part of the 2D chain: (g11, g21, g22) on L to (s_x, s_y, theta).
__device__ __forceinline__ void chain_rs(const float* p, float g11, float g21, float g22, float* out) {
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
    out[2] = g11 * d11_sx + g21 * d21_sx + g22 * d22_sx;
    out[3] = g11 * d11_sy + g21 * d21_sy + g22 * d22_sy;
    out[4] = g11 * d11_th + g21 * d21_th + g22 * d22_th;
}

constexpr int kChainPrims = 8;  // primitives per warp in k_reduce_chain2d

// One warp per kChainPrims primitives: sum each one's slots, then chain (mx, my, L, f, phc, c) to the record
// mu, s, theta, f, phi, c.  L depends on (theta, s_x, s_y) through
// A = c^2/sx^2 + s^2/sy^2, B = c s (1/sx^2 - 1/sy^2), l11 = sqrt(A), l21 = B/l11, l22 = 1/(sx sy l11);
// for the Cholesky record (cov2d = 1) on (l1, l2, l3) through, with u = l2^2 + l3^2, s = sqrt(u):
// l11 = s / |l1 l3|, l21 = -sgn(l1) l2 / (|l3| s), l22 = 1 / s, so that
//   dl11/dl1 = -l11/l1, dl11/dl2 = l11 l2/u, dl11/dl3 = l11 (l3/u - 1/l3),
//   dl21/dl2 = -sgn(l1) l3^2 / (|l3| s u), dl21/dl3 = -l21 (1/l3 + l3/u),
//   dl22/dl2 = -l2 / (s u), dl22/dl3 = -l3 / (s u).
// VEC: the output rows are 16-byte aligned and go out as four 16-byte stores.
template <bool VEC>
__global__ void __launch_bounds__(256) k_reduce_chain2d(const float* __restrict__ params, int64_t N, int cov2d,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint32_t* __restrict__ counts,
                                                        const float* __restrict__ partial,
                                                        float* __restrict__ dl_dparams) {
    pdl_enter();
    // a warp takes kChainPrims consecutive primitives: its half-warps sum the slots of two of them
    // at a time (lanes over the slots, coalesced), keeping the 11 totals of primitive k in
    // s_tot[warp][k]; then lane k chains primitive k.  The slot loads are the kernel's latency, so
    // a few primitives per warp and many warps hide it best.
    __shared__ float s_tot[8][kChainPrims][12];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hl = lane & 15, half = lane >> 4;
    const int64_t prim0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * kChainPrims;
    // the offsets and counts of the warp's primitives, loaded once (lane k: primitive k)
    uint32_t my_off = 0u, my_cnt = 0u;
    if (lane < kChainPrims && prim0 + lane < N) {
        my_off = offsets[prim0 + lane];
        my_cnt = counts[prim0 + lane];
    }
#pragma unroll
    for (int k2 = 0; k2 < kChainPrims; k2 += 2) {
        if (prim0 + k2 >= N) break;  // uniform across the warp
        const int64_t pk = prim0 + k2 + half;
        const uint32_t off = __shfl_sync(0xffffffffu, my_off, k2 + half), cnt = __shfl_sync(0xffffffffu, my_cnt, k2 + half);
        float acc[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) acc[m] = 0.f;
        for (uint32_t j = hl; j < cnt; j += 16) {
            const float4* src = reinterpret_cast<const float4*>(partial + (size_t)(off + j) * kSlot);
            const float4 x0 = src[0], x1 = src[1], x2 = src[2];
            acc[0] += x0.x; acc[1] += x0.y; acc[2] += x0.z; acc[3] += x0.w;
            acc[4] += x1.x; acc[5] += x1.y; acc[6] += x1.z; acc[7] += x1.w;
            acc[8] += x2.x; acc[9] += x2.y; acc[10] += x2.z;
        }
        // lane h of each half holds the half's total of slot h
        const float tot = half_reduce_scatter16(acc);
        if (hl < 11 && pk < N) s_tot[warp][k2 + half][hl] = tot;
    }
    __syncwarp();
    const int64_t prim = prim0 + lane;
    if (lane >= kChainPrims || prim >= N) return;
    const float* t = s_tot[warp][lane];
    const uint32_t cnt = counts[prim];
    const float* p = params + prim * WIPES_P2D;
    float* out_row = dl_dparams + prim * WIPES_P2D;
    float out[WIPES_P2D];
#pragma unroll
    for (int k = 0; k < WIPES_P2D; ++k) out[k] = 0.f;
    const float g11 = t[2], g21 = t[3], g22 = t[4];
    if (cnt == 0) {
        // off-screen or degenerate: the record's parameters get no gradient
    } else if (cov2d) {
        const float a = p[2], b = p[3], c = p[4];
        const float u = b * b + c * c, sq = sqrtf(u), aac = fabsf(a * c);
        const float l11 = sq / aac, l21 = -(a * b) / (aac * sq);
        const float isu = 1.0f / (sq * u);
        const float sgn_a = a < 0.0f ? -1.0f : 1.0f;
        out[2] = g11 * (-l11 / a);
        out[3] = g11 * (l11 * b / u) + g21 * (-sgn_a * c * c * isu / fabsf(c)) + g22 * (-b * isu);
        out[4] = g11 * (l11 * (c / u - 1.0f / c)) + g21 * (-l21 * (1.0f / c + c / u)) + g22 * (-c * isu);
    } else {
        chain_rs(p, g11, g21, g22, out);
    }
    if (cnt != 0) {
        out[0] = t[0];
        out[1] = t[1];
        out[5] = t[5];
        out[6] = t[6];
        out[7] = t[7] * kInvTwoPi;
        out[8] = t[8];
        out[9] = t[9];
        out[10] = t[10];
    }
    if (VEC) {
#pragma unroll
        for (int q = 0; q < WIPES_P2D / 4; ++q)
            reinterpret_cast<float4*>(out_row)[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < WIPES_P2D; ++k) out_row[k] = out[k];
    }
}


// Visited and inside-cutoff (pixel, primitive) pairs over the sorted tile lists; with `last`
// (3D), only list entries up to each pixel's last contributor count.
__global__ void __launch_bounds__(kTilePixels) k_count_pairs(const float4* __restrict__ rec, TileLists tl, int W,
                                                             int H, int tiles_x, float cutoff2,
                                                             const uint32_t* __restrict__ last,
                                                             unsigned long long* __restrict__ counters) {
    pdl_enter();
    __shared__ unsigned long long s_sum[2];
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int u = tx * kTile + (threadIdx.x & (kTile - 1));
    const int v = ty * kTile + (threadIdx.x / kTile);
    const bool in = u < W && v < H;
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = tl.ranges[tile];
    unsigned long long inside = 0;
    if (threadIdx.x < 2) s_sum[threadIdx.x] = 0ull;
    __syncthreads();
    if (in) {
        const uint32_t end = last ? range.x + last[(size_t)v * W + u] : range.y;
        for (uint32_t i = range.x; i < end; ++i) {
            const uint32_t id = tl.prim[i];
            const float4 A = rec[(size_t)id * kRecF4 + 0];
            const float l22 = rec[(size_t)id * kRecF4 + 1].x;
            inside += mahalanobis2(px, py, A.x, A.y, A.z, A.w, l22) <= cutoff2;
        }
        atomicAdd(&s_sum[0], (unsigned long long)(end - range.x));
        atomicAdd(&s_sum[1], inside);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&counters[0], s_sum[0]);
        atomicAdd(&counters[1], s_sum[1]);
    }
}

}  // namespace

void launch_blend2d(const BlendJob& job, int tiles_y, cudaStream_t stream) {
    launch_pdl(k_blend2d, job.tiles_x * tiles_y, kTilePixels, 0, stream, job);
    count_launches(1);
}

void launch_backward2d(const float4* rec, const PixRect* rect, const TileLists& tl, int W, int H, int tiles_x,
                       int tiles_y, float cutoff, const float* dl_dout, float* partial, cudaStream_t stream) {
    const float cutoff2 = cutoff * cutoff;
    launch_pdl(k_backward2d, kBwdSplit * tiles_x * tiles_y, kTilePixels, 0, stream, rec, rect, tl, W, H, tiles_x, cutoff2,
               touch_limit(cutoff), cutoff_scale(cutoff2), dl_dout, partial);
    count_launches(1);
}

void launch_count_pairs(const float4* rec, const TileLists& tl, int W, int H, int tiles_x, int tiles_y, float cutoff2,
                        const uint32_t* last, unsigned long long* counters, cudaStream_t stream) {
    launch_pdl(k_count_pairs, tiles_x * tiles_y, kTilePixels, 0, stream, rec, tl, W, H, tiles_x, cutoff2, last, counters);
    count_launches(1);
}

void launch_reduce_chain2d(const float* params, int64_t N, int cov2d, const uint32_t* offsets, const uint32_t* counts,
                           const float* partial, float* dl_dparams, cudaStream_t stream) {
    if (N == 0) return;
    const int64_t blocks = ceil_div(N, 8 * kChainPrims);  // 8 warps per block
    if ((reinterpret_cast<uintptr_t>(dl_dparams) & 15u) == 0)
        launch_pdl(k_reduce_chain2d<true>, blocks, 256, 0, stream, params, N, cov2d, offsets, counts, partial,
                   dl_dparams);
    else
        launch_pdl(k_reduce_chain2d<false>, blocks, 256, 0, stream, params, N, cov2d, offsets, counts, partial,
                   dl_dparams);
    count_launches(1);
}

}  // namespace wipes
