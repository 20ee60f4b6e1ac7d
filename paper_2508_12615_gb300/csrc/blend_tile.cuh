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
    const uint32_t prim = tl.prim[i];
    A = rec[(size_t)prim * kRecF4 + 0];
    B = rec[(size_t)prim * kRecF4 + 1];
    C = rec[(size_t)prim * kRecF4 + 2];
    return subtile_mask_ellipse(A, B.x, rect[prim], x0, y0, lim);
}

// Forward.  The 16x16 tile is four 8x8 quadrants.  Warp w serves quadrant w & 3 and, of each
// staged batch, every second entry (from w >> 2) of the entries whose cutoff ellipse reaches that
// quadrant; lane l owns the two pixels (l & 7, l >> 3) and (l & 7, (l >> 3) + 4) of its quadrant
// and evaluates both at once in packed f32x2 arithmetic.  When a batch is staged, each thread
// stores its record with every value duplicated (so that a warp reads ready-made pairs by
// broadcast) and the colour halved (the modulation is then taken as G (1 + cos)), and marks which
// quadrants its primitive's cutoff ellipse reaches (exact in binary32, conservative); the marks
// become one list of staged entries per quadrant, in tile-list order.  The cutoff enters the
// exponent: outside it the argument is S (cutoff^2 - q) <= -512 and ex2 returns 0 (S the
// power-of-two scale of cutoff_scale()), inside it is -q log2(e) / 2.  Per pixel, the sum runs
// over the batch (a batch-local partial, added once per batch), and at the end the two warps of a
// quadrant add their totals in a fixed order.
__device__ __forceinline__ void blend2d_tile(const BlendJob& job, int tile) {
    const float4* __restrict__ rec = job.rec;
    const PixRect* __restrict__ rect = job.rect;
    const TileLists& tl = job.tl;
    const int W = job.W, H = job.H, tiles_x = job.tiles_x;
    const float lim = job.o.lim;
    float* __restrict__ out = job.out;
    // staged entry k: (mx, my) (l11, l21) (l22, fx) (fy, phc) (c_r, c_g) / 2 (c_b / 2, 0), each value twice
    __shared__ ulonglong2 s_e[6][kTilePixels];
    __shared__ uint8_t s_list[4][kTilePixels];        // per quadrant: the staged entries that reach it
    __shared__ uint32_t s_cnt[kTilePixels / 32][4];   // per warp and quadrant: its staged entries that reach it
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int quad = warp & 3, half = warp >> 2;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const int u = x0 + (quad & 1) * 8 + (lane & 7);
    const int v = y0 + (quad >> 1) * 8 + (lane >> 3);  // and v + 4
    const f2 PX = f2_dup((float)u + 0.5f);
    const f2 PY = f2_pack((float)v + 0.5f, (float)(v + 4) + 0.5f);
    const f2 K = f2_dup(kNegHalfLog2e);
    const f2 NEG_S = f2_dup(-job.o.cut_scale), CUT_S = f2_dup(job.o.cutoff2 * job.o.cut_scale);
    const uint2 range = tl.ranges[tile];
    f2 c0 = f2_dup(0.f), c1 = c0, c2 = c0;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        __syncthreads();
        uint32_t m = 0u;
        if ((int)threadIdx.x < n) {
            const uint32_t prim = tl.prim[b0 + threadIdx.x];
            const float4 A = rec[(size_t)prim * kRecF4 + 0];
            const float4 B = rec[(size_t)prim * kRecF4 + 1];
            const float4 C = rec[(size_t)prim * kRecF4 + 2];
            m = quadrant_mask_ellipse(A, B.x, rect[prim], x0, y0, lim);
            s_e[0][threadIdx.x] = dup2(A.x, A.y);
            s_e[1][threadIdx.x] = dup2(A.z, A.w);
            s_e[2][threadIdx.x] = dup2(B.x, B.y);
            s_e[3][threadIdx.x] = dup2(B.z, B.w);
            s_e[4][threadIdx.x] = dup2(0.5f * C.x, 0.5f * C.y);
            s_e[5][threadIdx.x] = dup2(0.5f * C.z, 0.f);
        }
        uint32_t bal[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) bal[k] = __ballot_sync(0xffffffffu, (m >> k) & 1u);
        if (lane < 4) s_cnt[warp][lane] = __popc(lane == 0 ? bal[0] : lane == 1 ? bal[1] : lane == 2 ? bal[2] : bal[3]);
        __syncthreads();
        // each entry's place in the list of every quadrant it reaches: the entries of earlier
        // warps, then those of earlier lanes
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((m >> k) & 1u) {
                uint32_t pos = __popc(bal[k] & ((1u << lane) - 1u));
                for (int w = 0; w < warp; ++w) pos += s_cnt[w][k];
                s_list[k][pos] = (uint8_t)threadIdx.x;
            }
        }
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < kTilePixels / 32; ++w) cnt += s_cnt[w][quad];
        __syncthreads();
        f2 a0 = f2_dup(0.f), a1 = a0, a2 = a0;
        for (uint32_t i = half; i < cnt; i += 2) {
            const int j = s_list[quad][i];
            const f2x2 e0 = ld_f2x2(&s_e[0][j]), e1 = ld_f2x2(&s_e[1][j]);
            const f2x2 e2 = ld_f2x2(&s_e[2][j]), e3 = ld_f2x2(&s_e[3][j]);
            // the cutoff test in the operation order of mahalanobis2()
            const f2 dx = f2_sub(PX, e0.x), dy = f2_sub(PY, e0.y);
            const f2 a = f2_fma(e1.x, dx, f2_mul(e1.y, dy));
            const f2 b = f2_mul(e2.x, dy);
            const f2 q = f2_fma(a, a, f2_mul(b, b));
            const f2 ex = f2_mul(q, K), cut = f2_fma(q, NEG_S, CUT_S);
            const f2 G = f2_pack(ex2_approx(fminf(f2_lo(ex), f2_lo(cut))), ex2_approx(fminf(f2_hi(ex), f2_hi(cut))));
            const f2 ang = f2_reduced_angle(f2_fma(e2.y, dx, f2_fma(e3.x, dy, e3.y)));
            const f2 cs = f2_pack(cos_approx(f2_lo(ang)), cos_approx(f2_hi(ang)));
            const f2 wv = f2_fma(cs, G, G);  // 2 W
            const f2x2 e4 = ld_f2x2(&s_e[4][j]), e5 = ld_f2x2(&s_e[5][j]);
            a0 = f2_fma(e4.x, wv, a0);
            a1 = f2_fma(e4.y, wv, a1);
            a2 = f2_fma(e5.x, wv, a2);
        }
        c0 = f2_add(c0, a0);
        c1 = f2_add(c1, a1);
        c2 = f2_add(c2, a2);
    }
    // the second warp of each quadrant hands its sums to the first
    __syncthreads();
    f2* s_sum = reinterpret_cast<f2*>(&s_e[0][0]);
    const int slot = (quad * 32 + lane) * 3;
    if (half == 1) {
        s_sum[slot + 0] = c0;
        s_sum[slot + 1] = c1;
        s_sum[slot + 2] = c2;
    }
    __syncthreads();
    if (half == 0) {
        c0 = f2_add(c0, s_sum[slot + 0]);
        c1 = f2_add(c1, s_sum[slot + 1]);
        c2 = f2_add(c2, s_sum[slot + 2]);
        if (u < W && v < H) {
            float* o = out + ((size_t)v * W + u) * 3;
            o[0] = f2_lo(c0);
            o[1] = f2_lo(c1);
            o[2] = f2_lo(c2);
        }
        if (u < W && v + 4 < H) {
            float* o = out + ((size_t)(v + 4) * W + u) * 3;
            o[0] = f2_hi(c0);
            o[1] = f2_hi(c1);
            o[2] = f2_hi(c2);
        }
    }
}


// One pixel's state in the 3D front-to-back blend.
struct Px3 {
    float T, c0, c1, c2;
    uint32_t last;  // 1-based tile-list position of the last entry that contributed (0: none)
    bool done;      // the next contribution would have taken T below T_min
};

// One tile-list entry at one pixel (Eq. 3 with W'): nothing outside the cutoff ellipse or below
// alpha_min; stop before an entry that would take T below T_min; else add c alpha T and update T.
// `pos` is the entry's 1-based position in the tile list; hk the record's oscillation weight
// (1/2, or kappa / 2 under frequency map 2).  Every 3D forward kernel blends in these operations,
// so a pixel gets the same bits whatever the block shape.
__device__ __forceinline__ void blend3d_pair(Px3& s, float px, float py, const float4& A, const float4& B,
                                             const float4& C, float hk, const BlendOpts3& o, uint32_t pos) {
    const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
    if (!(q <= o.cutoff2)) return;
    const float dx = px - A.x, dy = py - A.y;
    const float G = ex2_approx(q * kNegHalfLog2e);
    const float w = fmaf(hk, cos_approx(reduced_angle(fmaf(B.y, dx, fmaf(B.z, dy, B.w)))), 0.5f) * G;
    const float alpha = fminf(o.alpha_max, C.w * w);
    if (alpha < o.alpha_min) return;
    const float test_T = s.T * (1.f - alpha);
    if (test_T < o.T_min) {
        s.done = true;
        return;
    }
    const float wt = alpha * s.T;
    s.c0 = fmaf(C.x, wt, s.c0);
    s.c1 = fmaf(C.y, wt, s.c1);
    s.c2 = fmaf(C.z, wt, s.c2);
    s.T = test_T;
    s.last = pos;
}

__device__ __forceinline__ void store_px3(const BlendJob& job, int u, int v, const Px3& s) {
    const size_t pix = (size_t)v * job.W + u;
    job.out[pix * 3 + 0] = fmaf(s.T, job.o.bg[0], s.c0);
    job.out[pix * 3 + 1] = fmaf(s.T, job.o.bg[1], s.c1);
    job.out[pix * 3 + 2] = fmaf(s.T, job.o.bg[2], s.c2);
    if (job.cfin) {  // the colour without the background, for the chunked backward
        job.cfin[pix * 3 + 0] = s.c0;
        job.cfin[pix * 3 + 1] = s.c1;
        job.cfin[pix * 3 + 2] = s.c2;
    }
    job.T_final[pix] = s.T;
    job.last[pix] = s.last;
}

// Forward over a whole 16x16 tile (256 threads; used by the batch kernel).  As in 2D, warp w owns
// an 8x4 pixel sub-tile and visits only the staged primitives whose cutoff ellipse reaches it;
// positions in the tile list are counted from the list start, so the per-pixel last-contributor
// index does not depend on the culling.
__device__ __forceinline__ void blend3d_tile(const BlendJob& job, int tile) {
    const float4* __restrict__ rec = job.rec;
    const PixRect* __restrict__ rect = job.rect;
    const TileLists& tl = job.tl;
    const int W = job.W, H = job.H, tiles_x = job.tiles_x;
    const BlendOpts3& o = job.o;
    __shared__ float4 s_a[kTilePixels];
    __shared__ float4 s_b[kTilePixels];
    __shared__ float4 s_c[kTilePixels];
    __shared__ float s_k[kTilePixels];
    __shared__ uint8_t s_mask[kTilePixels];
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = tx * kTile, y0 = ty * kTile;
    const int u = x0 + (warp & 1) * 8 + (lane & 7);
    const int v = y0 + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = u < W && v < H;
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = tl.ranges[tile];
    Px3 s{1.f, 0.f, 0.f, 0.f, 0u, !inside};
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        if (__syncthreads_count(s.done) == kTilePixels) break;
        const int n = (int)min((uint32_t)kTilePixels, range.y - b0);
        if ((int)threadIdx.x < n) {
            const uint32_t id = tl.prim[b0 + threadIdx.x];
            const float4 A = rec[(size_t)id * kRecF4 + 0];
            const float4 B = rec[(size_t)id * kRecF4 + 1];
            s_a[threadIdx.x] = A;
            s_b[threadIdx.x] = B;
            s_c[threadIdx.x] = rec[(size_t)id * kRecF4 + 2];
            s_k[threadIdx.x] = o.damp ? rec[(size_t)id * kRecF4 + 3].w : 0.5f;
            s_mask[threadIdx.x] = (uint8_t)subtile_mask_ellipse(A, B.x, rect[id], x0, y0, o.lim);
        }
        __syncthreads();
        for (int c = 0; c < n; c += 32) {
            if (__all_sync(0xffffffffu, s.done)) break;
            const uint32_t m = c + lane < n ? s_mask[c + lane] : 0u;
            uint32_t bal = __ballot_sync(0xffffffffu, (m >> warp) & 1u);
            while (bal) {
                const int j = c + __ffs(bal) - 1;
                bal &= bal - 1u;
                if (s.done) continue;
                blend3d_pair(s, px, py, s_a[j], s_b[j], s_c[j], s_k[j], o, b0 - range.x + (uint32_t)j + 1u);
            }
        }
    }
    if (inside) store_px3(job, u, v, s);
}

// Forward over one 8x8 quad of a 16x16 tile, for a block of one warp: lane l owns the pixels
// (l & 7, l >> 3) and (l & 7, (l >> 3) + 4) of the quad and blends both at once in packed f32x2
// arithmetic, each pixel with exactly the operations of blend3d_pair (so a pixel gets the same
// bits here and in blend3d_tile).  Long tile lists spread over four blocks, which the scheduler
// can place on four SMs.  Batches of 32 entries are staged in shared memory with every value
// twice, marked by whether the entry's cutoff ellipse reaches the quad; the records of the next
// batch are loaded into registers (from primitive ids fetched one batch earlier still) while the
// current batch is blended, so the gathers overlap the arithmetic.
constexpr int kQuadThreads = 32;

// One entry at a lane's two pixels, before the transmittance: cutoff, alpha (packed as in
// blend3d_pair: q, envelope, phase, modulation, alpha = min(alpha_max, o W')).
struct Eval3 {
    f2 q, alpha;
};
// DAMP: frequency map 2, the entry's oscillation weight hk = kappa / 2 is staged in s_e[6][j].x
// (else the constant 1/2, the same bits as hk = 1/2).
template <bool DAMP>
__device__ __forceinline__ void eval3_entry(Eval3& r, const ulonglong2 (*s_e)[kQuadThreads], int j, f2 PX, f2 PY,
                                            const BlendOpts3& o) {
    const f2x2 e0 = ld_f2x2(&s_e[0][j]), e1 = ld_f2x2(&s_e[1][j]), e2 = ld_f2x2(&s_e[2][j]);
    const f2x2 e3 = ld_f2x2(&s_e[3][j]), e5 = ld_f2x2(&s_e[5][j]);
    // the cutoff test in the operation order of mahalanobis2()
    const f2 dx = f2_sub(PX, e0.x), dy = f2_sub(PY, e0.y);
    const f2 a = f2_fma(e1.x, dx, f2_mul(e1.y, dy));
    const f2 b = f2_mul(e2.x, dy);
    r.q = f2_fma(a, a, f2_mul(b, b));
    const f2 e = f2_mul(r.q, f2_dup(kNegHalfLog2e));
    const f2 G = f2_pack(ex2_approx(f2_lo(e)), ex2_approx(f2_hi(e)));
    const f2 ang = f2_reduced_angle(f2_fma(e2.y, dx, f2_fma(e3.x, dy, e3.y)));
    const f2 HALF = f2_dup(0.5f);
    f2 hk = HALF;
    if constexpr (DAMP) hk = ld_f2x2(&s_e[6][j]).x;
    const f2 w = f2_mul(f2_fma(hk, f2_pack(cos_approx(f2_lo(ang)), cos_approx(f2_hi(ang))), HALF), G);
    const f2 raw = f2_mul(e5.y, w);
    r.alpha = f2_pack(fminf(o.alpha_max, f2_lo(raw)), fminf(o.alpha_max, f2_hi(raw)));
}
// The entry's effect on the pixels' state, in list order (blend3d_pair's skip, stop and update).
__device__ __forceinline__ void apply3_entry(const Eval3& r, const ulonglong2 (*s_e)[kQuadThreads], int j,
                                             const BlendOpts3& o, f2& T, f2& c0, f2& c1, f2& c2, uint32_t& last0,
                                             uint32_t& last1, bool& done0, bool& done1, uint32_t pos) {
    const float al0 = f2_lo(r.alpha), al1 = f2_hi(r.alpha);
    const bool k0 = !done0 && f2_lo(r.q) <= o.cutoff2 && al0 >= o.alpha_min;
    const bool k1 = !done1 && f2_hi(r.q) <= o.cutoff2 && al1 >= o.alpha_min;
    if (!__any_sync(0xffffffffu, k0 || k1)) return;
    const f2 test_T = f2_mul(T, f2_sub(f2_dup(1.f), r.alpha));
    // stop before an entry that would take T below T_min
    const bool s0 = k0 && f2_lo(test_T) < o.T_min, s1 = k1 && f2_hi(test_T) < o.T_min;
    done0 |= s0;
    done1 |= s1;
    const bool p0 = k0 && !s0, p1 = k1 && !s1;
    const f2 wt = f2_pack(p0 ? al0 * f2_lo(T) : 0.f, p1 ? al1 * f2_hi(T) : 0.f);
    const f2x2 e4 = ld_f2x2(&s_e[4][j]), e5 = ld_f2x2(&s_e[5][j]);
    c0 = f2_fma(e4.x, wt, c0);
    c1 = f2_fma(e4.y, wt, c1);
    c2 = f2_fma(e5.x, wt, c2);
    T = f2_pack(p0 ? f2_lo(test_T) : f2_lo(T), p1 ? f2_hi(test_T) : f2_hi(T));
    if (p0) last0 = pos;
    if (p1) last1 = pos;
}


template <bool DAMP>
__device__ __forceinline__ void blend3d_quad(const BlendJob& job, int tile, int quad) {
    const float4* __restrict__ rec = job.rec;
    const PixRect* __restrict__ rect = job.rect;
    const TileLists& tl = job.tl;
    const BlendOpts3& o = job.o;
    // staged entry: (mx, my) (l11, l21) (l22, fx) (fy, phc) (c_r, c_g) (c_b, o), each value twice,
    // and with DAMP (hk, 0)
    __shared__ ulonglong2 s_e[DAMP ? 7 : 6][kQuadThreads];
    const int tx = tile % job.tiles_x, ty = tile / job.tiles_x;
    const int lane = threadIdx.x & 31;
    const int x0 = tx * kTile + (quad & 1) * 8, y0 = ty * kTile + (quad >> 1) * 8;
    const int u = x0 + (lane & 7), v = y0 + (lane >> 3);  // and v + 4
    const bool in0 = u < job.W && v < job.H, in1 = u < job.W && v + 4 < job.H;
    const f2 PX = f2_dup((float)u + 0.5f), PY = f2_pack((float)v + 0.5f, (float)(v + 4) + 0.5f);
    const uint2 range = tl.ranges[tile];
    f2 T = f2_dup(1.f), c0 = f2_dup(0.f), c1 = c0, c2 = c0;
    uint32_t last0 = 0u, last1 = 0u;
    bool done0 = !in0, done1 = !in1;
    // registers of the software pipeline: records of the batch to stage next, primitive id of the
    // batch after it
    float4 nA = make_float4(0.f, 0.f, 0.f, 0.f), nB = nA, nC = nA;
    float nK = 0.5f;
    PixRect nR{0, 0, -1, -1};
    uint32_t np = 0u;
    if (range.x + lane < range.y) {
        const uint32_t p = tl.prim[range.x + lane];
        nA = rec[(size_t)p * kRecF4 + 0];
        nB = rec[(size_t)p * kRecF4 + 1];
        nC = rec[(size_t)p * kRecF4 + 2];
        if (DAMP) nK = rec[(size_t)p * kRecF4 + 3].w;
        nR = rect[p];
    }
    if (range.x + kQuadThreads + lane < range.y) np = tl.prim[range.x + kQuadThreads + lane];
    // the chunked backward's boundaries: the pixels' state before list entries kBwdChunk, 2 kBwdChunk,
    // ... of a list of more than one chunk, recorded when the walk reaches them
    const uint32_t n_bnd = job.bnd ? bwd_chunks(range.y - range.x) : 0u;
    uint32_t next_bnd = n_bnd > 1u ? range.x + kBwdChunk : 0xFFFFFFFFu;
    float4* rowb = n_bnd > 1u ? job.bnd + (size_t)job.item_base[tile] * kTilePixels : nullptr;
    const int px_in_tile = (quad & 1) * 8 + (lane & 7) + ((quad >> 1) * 8 + (lane >> 3)) * kTile;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kQuadThreads) {
        if (__all_sync(0xffffffffu, done0 && done1)) break;
        if (b0 == next_bnd) {
            rowb += kTilePixels;
            rowb[px_in_tile] = make_float4(f2_lo(T), f2_lo(c0), f2_lo(c1), f2_lo(c2));
            rowb[px_in_tile + 4 * kTile] = make_float4(f2_hi(T), f2_hi(c0), f2_hi(c1), f2_hi(c2));
            next_bnd += kBwdChunk;
        }
        const int n = (int)min((uint32_t)kQuadThreads, range.y - b0);
        __syncwarp();
        bool hit = false;
        if (lane < n) {
            s_e[0][lane] = dup2(nA.x, nA.y);
            s_e[1][lane] = dup2(nA.z, nA.w);
            s_e[2][lane] = dup2(nB.x, nB.y);
            s_e[3][lane] = dup2(nB.z, nB.w);
            s_e[4][lane] = dup2(nC.x, nC.y);
            s_e[5][lane] = dup2(nC.z, nC.w);
            if constexpr (DAMP) s_e[6][lane] = dup2(nK, 0.f);
            float nBA, nBC;
            ellipse_edge_ratios(nA, nB.x, nBA, nBC);
            hit = box_touched_ellipse(nA, nB.x, nBA, nBC, nR, x0, y0, 8, 8, o.lim);
        }
        uint32_t bal = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        if (b0 + kQuadThreads + lane < range.y) {
            nA = rec[(size_t)np * kRecF4 + 0];
            nB = rec[(size_t)np * kRecF4 + 1];
            nC = rec[(size_t)np * kRecF4 + 2];
            if (DAMP) nK = rec[(size_t)np * kRecF4 + 3].w;
            nR = rect[np];
        }
        if (b0 + 2 * kQuadThreads + lane < range.y) np = tl.prim[b0 + 2 * kQuadThreads + lane];
        // two entries per step: their envelope, phase and alpha do not depend on each other, only
        // the transmittance update does, so evaluating them together doubles the independent work
        // in flight; the updates then follow in list order
        while (bal) {
            const int j1 = __ffs(bal) - 1;
            bal &= bal - 1u;
            const int j2 = bal ? __ffs(bal) - 1 : -1;
            if (bal) bal &= bal - 1u;
            Eval3 ea, eb;
            eval3_entry<DAMP>(ea, s_e, j1, PX, PY, o);
            if (j2 >= 0) eval3_entry<DAMP>(eb, s_e, j2, PX, PY, o);
            apply3_entry(ea, s_e, j1, o, T, c0, c1, c2, last0, last1, done0, done1, b0 - range.x + (uint32_t)j1 + 1u);
            if (j2 >= 0)
                apply3_entry(eb, s_e, j2, o, T, c0, c1, c2, last0, last1, done0, done1, b0 - range.x + (uint32_t)j2 + 1u);
        }
    }
    if (in0) store_px3(job, u, v, Px3{f2_lo(T), f2_lo(c0), f2_lo(c1), f2_lo(c2), last0, done0});
    if (in1) store_px3(job, u, v + 4, Px3{f2_hi(T), f2_hi(c0), f2_hi(c1), f2_hi(c2), last1, done1});
}


}  // namespace wipes
