// 3D view synthesis: front-to-back alpha blending of projected wavelets over depth-sorted tile
// lists (Eq. 3 with G' replaced by W', Sec. 4.1), its backward with the transmittance recomputed
// from the stored final value, and the chain through the EWA projection (Sec. 3.1) and the
// frequency projection (Sec. 4.1) to the 3D record.
//
// Blend rule per pixel, over the tile list in order: skip a primitive outside its cutoff ellipse;
// alpha = min(alpha_max, o W'); skip alpha < alpha_min; stop before a primitive that would take
// T (1 - alpha) below T_min; otherwise C += c alpha T, T *= 1 - alpha.  Finally C += T bg.
#include "blend_tile.cuh"

namespace wipes {
namespace {

// One block per 8x8 quad, tiles taken in the given order (longest list first).  DAMP: frequency
// map 2 (the records carry the oscillation weight hk = kappa / 2).
template <bool DAMP>
__global__ void __launch_bounds__(kQuadThreads) k_blend3d(BlendJob job, const uint32_t* __restrict__ order) {
    pdl_enter();
    blend3d_quad<DAMP>(job, (int)order[blockIdx.x >> 2], (int)(blockIdx.x & 3u));
}

// Entries whose terms come from at most this many lanes of a warp are added by those lanes
// directly instead of through the warp's reduce-scatter.
constexpr int kBwdDirectLanes = 4;

// Image-plane gradient per primitive: mx my l11 l21 l22 fx fy phc c_r c_g c_b o (12 floats a row),
// and with DAMP kappa (13 components in rows of 16).
template <bool DAMP>
__host__ __device__ constexpr int grad_components() { return DAMP ? 13 : 12; }
template <bool DAMP>
__host__ __device__ constexpr int grad_stride() { return DAMP ? 16 : 12; }

// Record of one staged entry with every value twice, for packed arithmetic over a lane's two
// pixels: (mx, my) (l11, l21) (l22, fx) (fy, phc) (c_r, c_g) (c_b, o), and with DAMP (hk, 0).
template <bool DAMP>
__device__ __forceinline__ void stage_dup(ulonglong2 (*s_e)[32], int i, const float4& A, const float4& B,
                                          const float4& C, float hk) {
    s_e[0][i] = dup2(A.x, A.y);
    s_e[1][i] = dup2(A.z, A.w);
    s_e[2][i] = dup2(B.x, B.y);
    s_e[3][i] = dup2(B.z, B.w);
    s_e[4][i] = dup2(C.x, C.y);
    s_e[5][i] = dup2(C.z, C.w);
    if constexpr (DAMP) s_e[6][i] = dup2(hk, 0.f);
}

// One entry at a lane's two pixels, before the transmittance: the offsets, the cutoff form, the
// envelope, the modulation, alpha and whether the entry contributes to each pixel (with DAMP also
// the cosine and the entry's hk).
struct BwdEval {
    f2 dx, dy, a, b, G, w, raw, sn, cs, hk;
    float alpha0, alpha1;
    bool k0, k1;
};
template <bool DAMP>
__device__ __forceinline__ void bwd_eval(BwdEval& r, const ulonglong2 (*s_e)[32], int j, f2 PX, f2 PY,
                                         const BlendOpts3& o, bool live0, bool live1) {
    const f2x2 e0 = ld_f2x2(&s_e[0][j]), e1 = ld_f2x2(&s_e[1][j]), e2 = ld_f2x2(&s_e[2][j]);
    const f2x2 e3 = ld_f2x2(&s_e[3][j]), e5 = ld_f2x2(&s_e[5][j]);
    // the cutoff test in the operation order of mahalanobis2()
    r.dx = f2_sub(PX, e0.x);
    r.dy = f2_sub(PY, e0.y);
    r.a = f2_fma(e1.x, r.dx, f2_mul(e1.y, r.dy));
    r.b = f2_mul(e2.x, r.dy);
    const f2 q = f2_fma(r.a, r.a, f2_mul(r.b, r.b));
    const f2 e = f2_mul(q, f2_dup(kNegHalfLog2e));
    const bool c0 = live0 && f2_lo(q) <= o.cutoff2, c1 = live1 && f2_hi(q) <= o.cutoff2;
    r.G = f2_pack(ex2_approx(c0 ? f2_lo(e) : -INFINITY), ex2_approx(c1 ? f2_hi(e) : -INFINITY));
    const f2 ang = f2_reduced_angle(f2_fma(e2.y, r.dx, f2_fma(e3.x, r.dy, e3.y)));
    const float al = f2_lo(ang), ah = f2_hi(ang);
    const f2 HALF = f2_dup(0.5f);
    if constexpr (DAMP) {
        r.hk = ld_f2x2(&s_e[6][j]).x;
        r.cs = f2_pack(cos_approx(al), cos_approx(ah));
        r.w = f2_mul(f2_fma(r.hk, r.cs, HALF), r.G);
    } else {
        r.w = f2_mul(f2_fma(HALF, f2_pack(cos_approx(al), cos_approx(ah)), HALF), r.G);
    }
    r.sn = f2_pack(sin_approx(al), sin_approx(ah));
    r.raw = f2_mul(e5.y, r.w);
    r.alpha0 = fminf(o.alpha_max, f2_lo(r.raw));
    r.alpha1 = fminf(o.alpha_max, f2_hi(r.raw));
    r.k0 = c0 && r.alpha0 >= o.alpha_min;
    r.k1 = c1 && r.alpha1 >= o.alpha_min;
}
// The entry's gradient at the lane's pixels, with the transmittance recovered in front of it and
// the colour behind it advanced; the warp's sum is added to the primitive's image-plane gradient.
template <bool DAMP>
__device__ __forceinline__ void bwd_apply(const BwdEval& r, const ulonglong2 (*s_e)[32], int j, const BlendOpts3& o,
                                          f2& T, f2& S0, f2& S1, f2& S2, f2 g0, f2 g1, f2 g2, float* grad) {
    constexpr int kG = grad_components<DAMP>();
    if (!__any_sync(0xffffffffu, r.k0 || r.k1)) return;
    const int lane = threadIdx.x & 31;
    const f2x2 e1 = ld_f2x2(&s_e[1][j]), e2 = ld_f2x2(&s_e[2][j]), e3 = ld_f2x2(&s_e[3][j]);
    const f2x2 e4 = ld_f2x2(&s_e[4][j]), e5 = ld_f2x2(&s_e[5][j]);
    const f2 ONE = f2_dup(1.f), NEG1 = f2_dup(-1.f);
    // a pixel for which the entry is no contributor gets alpha 0: T, S unchanged, no terms
    const f2 alpha = f2_pack(r.k0 ? r.alpha0 : 0.f, r.k1 ? r.alpha1 : 0.f);
    const f2 om = f2_sub(ONE, alpha);
    const f2 inv = f2_pack(r.k0 ? rcp_approx(f2_lo(om)) : 1.f, r.k1 ? rcp_approx(f2_hi(om)) : 1.f);
    T = f2_mul(T, inv);  // transmittance in front of the entry
    const f2 wt = f2_mul(alpha, T);
    f2 acc[kG];
    acc[8] = f2_mul(g0, wt);
    acc[9] = f2_mul(g1, wt);
    acc[10] = f2_mul(g2, wt);
    const f2 x0c = f2_fma(e4.x, T, f2_mul(NEG1, f2_mul(S0, inv)));
    const f2 x1c = f2_fma(e4.y, T, f2_mul(NEG1, f2_mul(S1, inv)));
    const f2 x2c = f2_fma(e5.x, T, f2_mul(NEG1, f2_mul(S2, inv)));
    const f2 galpha = f2_fma(g0, x0c, f2_fma(g1, x1c, f2_mul(g2, x2c)));
    S0 = f2_fma(e4.x, wt, S0);
    S1 = f2_fma(e4.y, wt, S1);
    S2 = f2_fma(e5.x, wt, S2);
    // through alpha = o W' (zero where alpha was clamped to alpha_max)
    const f2 gal = f2_pack(r.k0 && f2_lo(r.raw) < o.alpha_max ? f2_lo(galpha) : 0.f,
                           r.k1 && f2_hi(r.raw) < o.alpha_max ? f2_hi(galpha) : 0.f);
    acc[11] = f2_mul(gal, r.w);
    const f2 gW = f2_mul(gal, e5.y);
    const f2 gq2 = f2_mul(NEG1, f2_mul(gW, r.w));  // 2 dL/dq  (dW/dq = -W/2)
    // dL/dt, t in cycles: dW/dt = -2 pi hk sin(2 pi t) G (hk = 1/2 without DAMP)
    f2 gt;
    if constexpr (DAMP) {
        gt = f2_mul(f2_mul(f2_mul(f2_dup(-2.f * kPi), r.hk), r.G), f2_mul(gW, r.sn));
        acc[12] = f2_mul(f2_mul(gW, f2_dup(0.5f)), f2_mul(r.cs, r.G));  // dW/dkappa = cos G / 2
    } else {
        gt = f2_mul(f2_mul(f2_dup(-kPi), r.G), f2_mul(gW, r.sn));
    }
    const f2 ga = f2_mul(gq2, r.a), gb = f2_mul(gq2, r.b);
    acc[2] = f2_mul(ga, r.dx);
    acc[3] = f2_mul(ga, r.dy);
    acc[4] = f2_mul(gb, r.dy);
    acc[0] = f2_mul(NEG1, f2_fma(ga, e1.x, f2_mul(gt, e2.y)));
    acc[1] = f2_mul(NEG1, f2_fma(ga, e1.y, f2_fma(gb, e2.x, f2_mul(gt, e3.x))));
    acc[5] = f2_mul(gt, r.dx);
    acc[6] = f2_mul(gt, r.dy);
    acc[7] = gt;
    float tot16[16];
#pragma unroll
    for (int i = 0; i < kG; ++i) tot16[i] = f2_lo(acc[i]) + f2_hi(acc[i]);
    // an entry that reaches the pixels of only a few lanes (a small footprint, or the edge of a
    // larger one): those lanes add their terms directly, which costs fewer instructions than the
    // warp's reduction (a lane whose pixels the entry does not reach holds only zero terms)
    const bool mine = r.k0 || r.k1;
    if (__popc(__ballot_sync(0xffffffffu, mine)) <= kBwdDirectLanes) {
        if (mine) {
#pragma unroll
            for (int i = 0; i < kG; ++i) atomicAdd(grad + i, tot16[i]);
        }
        return;
    }
#pragma unroll
    for (int i = kG; i < 16; ++i) tot16[i] = 0.f;
    const float tot = warp_reduce_scatter16(tot16);
    if ((lane & 1) == 0 && (lane >> 1) < kG) atomicAdd(grad + (lane >> 1), tot);
}

// Backward.  One warp per 8x8 quad of a tile (quads of the tiles in the given order, longest list
// first); lane l owns the pixels (l & 7, l >> 3) and (l & 7, (l >> 3) + 4) of the quad and works
// on both at once in packed f32x2 arithmetic.  Each pixel walks its tile list back to front from
// its last contributor, recovering the transmittance in front of each contributor as
// T_i = T_{i+1} / (1 - alpha_i) from the stored final value.  The warp's 64 per-pixel gradients of
// one primitive are summed by a reduce-scatter and added to the primitive's image-plane gradient
// with one atomic per component.  Batches of 32 entries are staged in shared memory with the bit
// "the cutoff ellipse reaches the quad"; the records of the next batch are loaded while the
// current one is processed.
template <bool DAMP>
__device__ __forceinline__ void bwd3d_unit(const float4* __restrict__ rec, const PixRect* __restrict__ rect,
                                           const TileLists& tl, int W, int H, int tiles_x, const BlendOpts3& o,
                                           const float* __restrict__ T_final, const uint32_t* __restrict__ last,
                                           const float* __restrict__ dl_dout, float* __restrict__ grad_img,
                                           const BwdChunks& ch, ulonglong2 (*s_e)[32], uint32_t* s_id,
                                           uint32_t item, int quad) {
    const uint2 it = ch.items[item];  // (tile, chunk)
    const int tile = (int)it.x;
    const uint32_t chunk = it.y;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lane = threadIdx.x & 31;
    const int x0 = tx * kTile + (quad & 1) * 8, y0 = ty * kTile + (quad >> 1) * 8;
    const int u = x0 + (lane & 7), v = y0 + (lane >> 3);  // and v + 4
    const bool in0 = u < W && v < H, in1 = u < W && v + 4 < H;
    const size_t pix0 = (size_t)v * W + u, pix1 = pix0 + (size_t)4 * W;
    const f2 PX = f2_dup((float)u + 0.5f), PY = f2_pack((float)v + 0.5f, (float)(v + 4) + 0.5f);
    const uint2 range = tl.ranges[tile];
    const uint32_t last0 = in0 ? last[pix0] : 0u, last1 = in1 ? last[pix1] : 0u;
    // entries past every pixel's last contributor are skipped; this item walks [c_lo, min(c_hi,
    // max last)) of the tile list (chunk kBwdChunk .. its end, the list's end for the last chunk),
    // back to front
    const uint32_t max_last = __reduce_max_sync(0xffffffffu, max(last0, last1));
    const uint32_t n_chunks = bwd_chunks(range.y - range.x);
    const uint32_t c_lo = chunk * kBwdChunk, c_hi = chunk + 1 == n_chunks ? range.y - range.x : c_lo + kBwdChunk;
    if (c_lo >= max_last) return;  // uniform across the warp
    // a pixel whose last contributor lies past this chunk starts from its state after the chunk,
    // recorded by the forward pass; the others from the final transmittance
    const float Tf0 = in0 ? T_final[pix0] : 1.f, Tf1 = in1 ? T_final[pix1] : 1.f;
    const bool rec0 = last0 > c_hi, rec1 = last1 > c_hi;
    float4 B0 = make_float4(Tf0, 0.f, 0.f, 0.f), B1 = make_float4(Tf1, 0.f, 0.f, 0.f);
    float Cf0[3] = {0.f, 0.f, 0.f}, Cf1[3] = {0.f, 0.f, 0.f};
    if (rec0 || rec1) {
        const float4* rowb = ch.bnd + (size_t)(ch.item_base[tile] + chunk + 1) * kTilePixels;
        const int px_in_tile = (quad & 1) * 8 + (lane & 7) + ((quad >> 1) * 8 + (lane >> 3)) * kTile;
        if (rec0) {
            B0 = rowb[px_in_tile];
            for (int k = 0; k < 3; ++k) Cf0[k] = ch.cfin[pix0 * 3 + k];
        }
        if (rec1) {
            B1 = rowb[px_in_tile + 4 * kTile];
            for (int k = 0; k < 3; ++k) Cf1[k] = ch.cfin[pix1 * 3 + k];
        }
    }
    f2 T = f2_pack(B0.x, B1.x);
    f2 g0 = f2_dup(0.f), g1 = g0, g2 = g0;
    if (in0 || in1) {
        const float* a0 = dl_dout + pix0 * 3;
        const float* a1 = dl_dout + pix1 * 3;
        g0 = f2_pack(in0 ? a0[0] : 0.f, in1 ? a1[0] : 0.f);
        g1 = f2_pack(in0 ? a0[1] : 0.f, in1 ? a1[1] : 0.f);
        g2 = f2_pack(in0 ? a0[2] : 0.f, in1 ? a1[2] : 0.f);
    }
    // colour accumulated behind the current primitive: the background term, plus (for a pixel
    // starting after the chunk) the colour of the entries after the chunk
    const f2 TF = f2_pack(Tf0, Tf1);
    f2 S0 = f2_fma(TF, f2_dup(o.bg[0]), f2_pack(rec0 ? Cf0[0] - B0.y : 0.f, rec1 ? Cf1[0] - B1.y : 0.f));
    f2 S1 = f2_fma(TF, f2_dup(o.bg[1]), f2_pack(rec0 ? Cf0[1] - B0.z : 0.f, rec1 ? Cf1[1] - B1.z : 0.f));
    f2 S2 = f2_fma(TF, f2_dup(o.bg[2]), f2_pack(rec0 ? Cf0[2] - B0.w : 0.f, rec1 ? Cf1[2] - B1.w : 0.f));
    // batches run [b0, b_end) downwards over the chunk's part below max last
    const uint32_t lo = range.x + c_lo;
    const uint32_t end = range.x + min(c_hi, max_last);
    uint32_t b_end = end;
    uint32_t b0 = end - min(end - lo, 32u);
    // software pipeline: records (and id) of the batch to stage next, id of the batch after it
    float4 nA = make_float4(0.f, 0.f, 0.f, 0.f), nB = nA, nC = nA;
    float nK = 0.5f;
    PixRect nR{0, 0, -1, -1};
    uint32_t nid = 0u, np = 0u;
    if (b0 + lane < b_end) {
        nid = tl.prim[b0 + lane];
        nA = rec[(size_t)nid * kRecF4 + 0];
        nB = rec[(size_t)nid * kRecF4 + 1];
        nC = rec[(size_t)nid * kRecF4 + 2];
        if (DAMP) nK = rec[(size_t)nid * kRecF4 + 3].w;
        nR = rect[nid];
    }
    uint32_t nb0 = b0 - min(b0 - lo, 32u);  // start of the next batch
    if (nb0 + lane < b0) np = tl.prim[nb0 + lane];
    while (b_end > lo) {
        const int n = (int)(b_end - b0);
        __syncwarp();
        bool hit = false;
        if (lane < n) {
            s_id[lane] = nid;
            stage_dup<DAMP>(s_e, lane, nA, nB, nC, nK);
            float nBA, nBC;
            ellipse_edge_ratios(nA, nB.x, nBA, nBC);
            hit = box_touched_ellipse(nA, nB.x, nBA, nBC, nR, x0, y0, 8, 8, o.lim);
        }
        uint32_t bal = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        // loads for the next two batches: [nb0, b0) and [nnb0, nb0)
        const uint32_t nnb0 = nb0 - min(nb0 - lo, 32u);
        if (nb0 + lane < b0) {
            nid = np;
            nA = rec[(size_t)nid * kRecF4 + 0];
            nB = rec[(size_t)nid * kRecF4 + 1];
            nC = rec[(size_t)nid * kRecF4 + 2];
            if (DAMP) nK = rec[(size_t)nid * kRecF4 + 3].w;
            nR = rect[nid];
        }
        if (nnb0 + lane < nb0) np = tl.prim[nnb0 + lane];
        // two entries per step (back to front): their envelope, phase and alpha do not depend on
        // each other, so they are evaluated together; the transmittance recovery, the colour behind
        // and the gradient terms then follow in list order
        while (bal) {
            const int j1 = 31 - __clz(bal);
            bal &= ~(1u << j1);
            const int j2 = bal ? 31 - __clz(bal) : -1;
            if (bal) bal &= ~(1u << j2);
            const uint32_t pos1 = b0 - range.x + (uint32_t)j1 + 1u;  // 1-based positions in the tile list
            const uint32_t pos2 = b0 - range.x + (uint32_t)j2 + 1u;
            BwdEval ea, eb;
            bwd_eval<DAMP>(ea, s_e, j1, PX, PY, o, in0 && pos1 <= last0, in1 && pos1 <= last1);
            if (j2 >= 0) bwd_eval<DAMP>(eb, s_e, j2, PX, PY, o, in0 && pos2 <= last0, in1 && pos2 <= last1);
            constexpr int kGS = grad_stride<DAMP>();
            bwd_apply<DAMP>(ea, s_e, j1, o, T, S0, S1, S2, g0, g1, g2, grad_img + (size_t)s_id[j1] * kGS);
            if (j2 >= 0)
                bwd_apply<DAMP>(eb, s_e, j2, o, T, S0, S1, S2, g0, g1, g2, grad_img + (size_t)s_id[j2] * kGS);
        }
        b_end = b0;
        b0 = nb0;
        nb0 = nnb0;
    }
}

// Persistent: each warp takes (item, quad) units in order from a counter until they run out, so no
// block is spent on an item past the last one.
template <bool DAMP>
__global__ void __launch_bounds__(32) k_backward3d(const float4* __restrict__ rec, const PixRect* __restrict__ rect,
                                                   TileLists tl, int W, int H, int tiles_x, BlendOpts3 o,
                                                   const float* __restrict__ T_final,
                                                   const uint32_t* __restrict__ last,
                                                   const float* __restrict__ dl_dout,
                                                   float* __restrict__ grad_img, BwdChunks ch) {
    pdl_enter();
    __shared__ ulonglong2 s_e[DAMP ? 7 : 6][32];
    __shared__ uint32_t s_id[32];
    const uint32_t n_units = 4u * *ch.n_items;
    for (;;) {
        uint32_t unit = 0u;
        if ((threadIdx.x & 31) == 0) unit = atomicAdd(ch.counter, 1u);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= n_units) break;
        __syncwarp();
        bwd3d_unit<DAMP>(rec, rect, tl, W, H, tiles_x, o, T_final, last, dl_dout, grad_img, ch, s_e, s_id,
                         unit >> 2, (int)(unit & 3u));
    }
}

struct Cam3 {
    float V[12];
    float fx, fy, cx, cy, near_z;
    float cpos[3];  // camera centre in world coordinates
};

// d R(q)_e / d q_m for a unit quaternion q = (w, x, y, z)
__device__ __forceinline__ void quat_rot_grad(const float q[4], const float gR[9], float gq[4]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    // row e of R, derivative with respect to (w, x, y, z)
    const float J[9][4] = {{0.f, 0.f, -4.f * y, -4.f * z},
                           {-2.f * z, 2.f * y, 2.f * x, -2.f * w},
                           {2.f * y, 2.f * z, 2.f * w, 2.f * x},
                           {2.f * z, 2.f * y, 2.f * x, 2.f * w},
                           {0.f, -4.f * x, 0.f, -4.f * z},
                           {-2.f * x, -2.f * w, 2.f * z, 2.f * y},
                           {-2.f * y, 2.f * z, -2.f * w, 2.f * x},
                           {2.f * x, 2.f * w, 2.f * z, 2.f * y},
                           {0.f, -4.f * x, -4.f * y, 0.f}};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < 9; ++e) s = fmaf(gR[e], J[e][m], s);
        gq[m] = s;
    }
}

// Chain the image-plane gradient (mx, my, L, f', phc, c, o) to the record mu, s, q, f, phi, o, c.
// With sh_degree > 0 the records and gradients hold WIPES_P3D_SH floats: dL/dsh_k = dL/dc Y_k(dir)
// where the colour was not clamped, and mu gains dL/ddir (I - dir dir^T) / |mu - camera centre|.
// One thread per primitive.  Its record, image-plane gradient and output row move in 16-byte
// pieces when the caller's parameter and gradient rows are 16-byte aligned (VEC), so that each
// load or store instruction covers whole sectors of the rows.
template <bool VEC>
__global__ void __launch_bounds__(128) k_chain3d(const float* __restrict__ params, int64_t N, Cam3 cam, int W, int H,
                                                 float dil, int fmode, int sh_degree, const float4* __restrict__ rec,
                                                 const float* __restrict__ grad_img, float* __restrict__ dl_dparams) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int stride = sh_degree ? WIPES_P3D_SH : WIPES_P3D;
    float* out_row = dl_dparams + i * stride;
    const float4 r0 = rec[(size_t)i * kRecF4 + 0];
    if (!(r0.z > 0.f)) {  // culled or degenerate: no gradient
        for (int k = 0; k < stride; ++k) out_row[k] = 0.f;
        return;
    }
    float p[WIPES_P3D];  // the record's geometry, frequency, phase, opacity and base colour
    load_row<VEC, WIPES_P3D>(p, params + i * stride);
    const float* p_sh = params + i * stride;  // the SH coefficients are read where they are used
    float g[16];
    if (fmode == 2) {
        load_row<true, 16>(g, grad_img + (size_t)i * 16);
    } else {
        load_row<true, 12>(g, grad_img + (size_t)i * 12);
        g[12] = 0.f;
    }
    float out[WIPES_P3D];
    const float g_mx = g[0], g_my = g[1], g11 = g[2], g21 = g[3], g22 = g[4], g_fx = g[5], g_fy = g[6];
    const float* V = cam.V;
    const float tx = V[0] * p[0] + V[1] * p[1] + V[2] * p[2] + V[3];
    const float ty = V[4] * p[0] + V[5] * p[1] + V[6] * p[2] + V[7];
    const float tz = V[8] * p[0] + V[9] * p[1] + V[10] * p[2] + V[11];
    const float qn2 = p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9];
    const float qinv = rsqrtf(qn2);
    const float qn[4] = {p[6] * qinv, p[7] * qinv, p[8] * qinv, p[9] * qinv};
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    const float s[3] = {p[3], p[4], p[5]};
    float M[9], Q[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[a * 3 + b] = R[a * 3 + b] * s[b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Q[a * 3 + b] = V[a * 4 + 0] * M[0 * 3 + b] + V[a * 4 + 1] * M[1 * 3 + b] + V[a * 4 + 2] * M[2 * 3 + b];
    const float limx = 1.3f * (0.5f * (float)W / cam.fx), limy = 1.3f * (0.5f * (float)H / cam.fy);
    const float rx = tx / tz, ry = ty / tz;
    const bool free_x = rx > -limx && rx < limx, free_y = ry > -limy && ry < limy;
    const float txz = fminf(limx, fmaxf(-limx, rx)), tyz = fminf(limy, fmaxf(-limy, ry));
    const float j00 = cam.fx / tz, j02 = -cam.fx * txz / tz, j11 = cam.fy / tz, j12 = -cam.fy * tyz / tz;
    float P0[3], P1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        P0[b] = j00 * Q[b] + j02 * Q[6 + b];
        P1[b] = j11 * Q[3 + b] + j12 * Q[6 + b];
    }
    const float n0 = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2];
    const float n1 = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2];
    const float S01 = P0[0] * P1[0] + P0[1] * P1[1] + P0[2] * P1[2];
    const float c0 = P0[1] * P1[2] - P0[2] * P1[1], c1 = P0[2] * P1[0] - P0[0] * P1[2],
                c2 = P0[0] * P1[1] - P0[1] * P1[0];
    const float S00 = n0 + dil, S11 = n1 + dil;
    const float D = c0 * c0 + c1 * c1 + c2 * c2 + dil * (n0 + n1) + dil * dil;
    const float l22 = rsqrtf(S11), l11 = sqrtf(S11 / D);
    const float u = rsqrtf(S11 * D), u3 = u * u * u;
    // L as a function of (S00, S01, S11), D = S00 S11 - S01^2
    const float d11_00 = -0.5f * l11 * S11 / D;
    const float d11_11 = 0.5f * l11 * (1.f / S11 - S00 / D);
    const float d11_01 = l11 * S01 / D;
    const float d21_00 = 0.5f * S01 * u3 * S11 * S11;
    const float d21_11 = 0.5f * S01 * u3 * (D + S11 * S00);
    const float d21_01 = -u - S01 * S01 * S11 * u3;
    const float d22_11 = -0.5f * l22 * l22 * l22;
    const float gS00 = g11 * d11_00 + g21 * d21_00;
    const float gS11 = g11 * d11_11 + g21 * d21_11 + g22 * d22_11;
    const float gS01 = g11 * d11_01 + g21 * d21_01;
    // S00 = |P0|^2 + dil, S11 = |P1|^2 + dil, S01 = P0.P1
    float gP0[3], gP1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        gP0[b] = 2.f * gS00 * P0[b] + gS01 * P1[b];
        gP1[b] = 2.f * gS11 * P1[b] + gS01 * P0[b];
    }
    float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f, gQ[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        gj00 += gP0[b] * Q[b];
        gj02 += gP0[b] * Q[6 + b];
        gj11 += gP1[b] * Q[3 + b];
        gj12 += gP1[b] * Q[6 + b];
        gQ[b] = gP0[b] * j00;
        gQ[3 + b] = gP1[b] * j11;
        gQ[6 + b] = gP0[b] * j02 + gP1[b] * j12;
    }
    // Q = V M, M = R diag(s)
    float gR[9], gs[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float gM = V[0 * 4 + a] * gQ[0 * 3 + b] + V[1 * 4 + a] * gQ[1 * 3 + b] + V[2 * 4 + a] * gQ[2 * 3 + b];
            gR[a * 3 + b] = gM * s[b];
            gs[b] += gM * R[a * 3 + b];
        }
    // camera-frame frequency; with f' = J fc (fmode 1) dL/dJ gains dL/df' fc^T
    const float fcx = V[0] * p[10] + V[1] * p[11] + V[2] * p[12];
    const float fcy = V[4] * p[10] + V[5] * p[11] + V[6] * p[12];
    const float fcz = V[8] * p[10] + V[9] * p[11] + V[10] * p[12];
    // frequency map 2 (integrated along the ray, as in the footprint kernel): reverse mode through
    // m = A^T n, w = S^-2 m, c = m . w, b = A w, fn = fc . n, r = fn / c, f' = P0^T (fc - r b) and
    // kappa = exp(-2 pi^2 fn r), with A = V R and n = (txz, tyz, 1); the pieces for the centre
    // (through n and P0) and the frequency are kept for below
    float gn0 = 0.f, gn1 = 0.f, gtz_map = 0.f, gfc_map[3] = {0.f, 0.f, 0.f};
    if (fmode == 2) {
        const float g_kap = g[12];
        float A[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                A[a * 3 + b] = V[a * 4 + 0] * R[0 * 3 + b] + V[a * 4 + 1] * R[1 * 3 + b] + V[a * 4 + 2] * R[2 * 3 + b];
        const float nv[3] = {txz, tyz, 1.f};
        float m[3], wv[3], is2[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            m[b] = A[b] * txz + A[3 + b] * tyz + A[6 + b];
            is2[b] = 1.f / (s[b] * s[b]);
            wv[b] = m[b] * is2[b];
        }
        const float c = m[0] * wv[0] + m[1] * wv[1] + m[2] * wv[2];
        const float bx = A[0] * wv[0] + A[1] * wv[1] + A[2] * wv[2];
        const float by = A[3] * wv[0] + A[4] * wv[1] + A[5] * wv[2];
        const float fn = fcx * txz + fcy * tyz + fcz;
        const float ic = 1.f / c, r = fn * ic;
        const float k2pi2 = 2.f * kPi * kPi;
        const float kap = __expf(-k2pi2 * fn * r);
        // f'x = (fcx - r bx) tz / fx, f'y = (fcy - r by) tz / fy, x = 2 pi^2 fn r, kappa = exp(-x)
        const float gx = g_fx * tz / cam.fx, gy = g_fy * tz / cam.fy;
        gtz_map = g_fx * (fcx - r * bx) / cam.fx + g_fy * (fcy - r * by) / cam.fy;
        const float gxx = -kap * g_kap;
        const float gr = -(gx * bx + gy * by) + k2pi2 * fn * gxx;
        const float gbx = -r * gx, gby = -r * gy;
        const float gfn = k2pi2 * r * gxx + gr * ic;
        const float gc = -gr * r * ic;
        gfc_map[0] = gx + gfn * txz;
        gfc_map[1] = gy + gfn * tyz;
        gfc_map[2] = gfn;
        gn0 = gfn * fcx;
        gn1 = gfn * fcy;
        float gA[9];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float gw = A[b] * gbx + A[3 + b] * gby + gc * m[b];
            const float gm = gc * wv[b] + gw * is2[b];
            gs[b] += -2.f * gw * wv[b] / s[b];
            gA[b] = gbx * wv[b] + nv[0] * gm;
            gA[3 + b] = gby * wv[b] + nv[1] * gm;
            gA[6 + b] = nv[2] * gm;
            gn0 += A[b] * gm;
            gn1 += A[3 + b] * gm;
        }
        // A = V R: dL/dR = V^T dL/dA (V's rows are the first three entries of cam.V's rows)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                gR[k * 3 + b] += V[0 * 4 + k] * gA[b] + V[1 * 4 + k] * gA[3 + b] + V[2 * 4 + k] * gA[6 + b];
    }
    float gqn[4];
    quat_rot_grad(qn, gR, gqn);
    const float dot = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
    if (fmode == 1) {
        gj00 += g_fx * fcx;
        gj02 += g_fx * fcz;
        gj11 += g_fy * fcy;
        gj12 += g_fy * fcz;
    }
    // camera-frame centre
    const float iz = 1.f / tz, iz2 = iz * iz;
    float gtx = g_mx * cam.fx * iz;
    float gty = g_my * cam.fy * iz;
    float gtz = -g_mx * cam.fx * tx * iz2 - g_my * cam.fy * ty * iz2;
    if (fmode == 0) gtz += g_fx * fcx / cam.fx + g_fy * fcy / cam.fy;
    if (fmode == 2) gtz += gtz_map;
    gtz += -gj00 * cam.fx * iz2 - gj11 * cam.fy * iz2 + gj02 * cam.fx * txz * iz2 + gj12 * cam.fy * tyz * iz2;
    if (free_x) {
        gtx += -gj02 * cam.fx * iz2;
        gtz += gj02 * cam.fx * tx * iz2 * iz;
        // map 2: txz = tx / tz
        gtx += gn0 * iz;
        gtz += -gn0 * tx * iz2;
    }
    if (free_y) {
        gty += -gj12 * cam.fy * iz2;
        gtz += gj12 * cam.fy * ty * iz2 * iz;
        gty += gn1 * iz;
        gtz += -gn1 * ty * iz2;
    }
    const float gfc0 = fmode == 2 ? gfc_map[0] : fmode ? g_fx * j00 : g_fx * tz / cam.fx;
    const float gfc1 = fmode == 2 ? gfc_map[1] : fmode ? g_fy * j11 : g_fy * tz / cam.fy;
    const float gfc2 = fmode == 2 ? gfc_map[2] : fmode ? g_fx * j02 + g_fy * j12 : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[a] = V[0 * 4 + a] * gtx + V[1 * 4 + a] * gty + V[2 * 4 + a] * gtz;
        out[3 + a] = gs[a];
        out[10 + a] = V[0 * 4 + a] * gfc0 + V[1 * 4 + a] * gfc1 + V[2 * 4 + a] * gfc2;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) out[6 + m] = (gqn[m] - qn[m] * dot) * qinv;
    out[13] = g[7] * kInvTwoPi;
    out[14] = g[11];
    out[15] = g[8];
    out[16] = g[9];
    out[17] = g[10];
    out[18] = 0.f;
    out[19] = 0.f;
    if (sh_degree) {
        const float vx = p[0] - cam.cpos[0], vy = p[1] - cam.cpos[1], vz = p[2] - cam.cpos[2];
        const float dist = sqrtf(vx * vx + vy * vy + vz * vz);
        const float dx = vx / dist, dy = vy / dist, dz = vz / dist;
        float Y[kShMaxCoeffs], Yx[kShMaxCoeffs], Yy[kShMaxCoeffs], Yz[kShMaxCoeffs];
        sh_eval(dx, dy, dz, Y);
        sh_eval_grad(dx, dy, dz, Yx, Yy, Yz);
        const int nk = (sh_degree + 1) * (sh_degree + 1);
        float gdx = 0.f, gdy = 0.f, gdz = 0.f, gc[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float raw = 0.5f;
#pragma unroll
            for (int k = 0; k < kShMaxCoeffs; ++k)
                if (k < nk) raw += Y[k] * p_sh[sh_slot(k, ch)];
            gc[ch] = raw > 0.f ? g[8 + ch] : 0.f;
#pragma unroll
            for (int k = 0; k < kShMaxCoeffs; ++k) {
                if (k >= nk) continue;
                const float c = p_sh[sh_slot(k, ch)];
                gdx += gc[ch] * c * Yx[k];
                gdy += gc[ch] * c * Yy[k];
                gdz += gc[ch] * c * Yz[k];
            }
            out[15 + ch] = gc[ch] * Y[0];
        }
        const float dd = gdx * dx + gdy * dy + gdz * dz;
        out[0] += (gdx - dd * dx) / dist;
        out[1] += (gdy - dd * dy) / dist;
        out[2] += (gdz - dd * dz) / dist;
        // the coefficients of degree >= 1: slot 20 + 3 (k - 1) + ch, zero past the record's degree
        constexpr int kShSlots = WIPES_P3D_SH - WIPES_P3D;
        float osh[kShSlots];
#pragma unroll
        for (int sl = 0; sl < kShSlots; ++sl) {
            const int k = sl / 3 + 1, ch = sl % 3;
            osh[sl] = (k < kShMaxCoeffs && k < nk) ? gc[ch] * Y[k] : 0.f;
        }
        store_row<VEC, kShSlots>(out_row + WIPES_P3D, osh);
    }
    store_row<VEC, WIPES_P3D>(out_row, out);
}

}  // namespace

void launch_blend3d(const BlendJob& job, int tiles_y, const uint32_t* order, cudaStream_t stream) {
    if (job.o.damp) launch_pdl(k_blend3d<true>, 4 * job.tiles_x * tiles_y, kQuadThreads, 0, stream, job, order);
    else launch_pdl(k_blend3d<false>, 4 * job.tiles_x * tiles_y, kQuadThreads, 0, stream, job, order);
    count_launches(1);
}

void launch_backward3d(const float4* rec, const PixRect* rect, const TileLists& tl, int W, int H, int tiles_x,
                       const BlendOpts3& o, const float* T_final, const uint32_t* last, const float* dl_dout,
                       float* grad_img, const BwdChunks& ch, int64_t max_items, cudaStream_t stream) {
    if (max_items <= 0) return;
    cudaMemsetAsync(ch.counter, 0, sizeof(unsigned int), stream);
    int per_sm = 0, dev = 0, sms = 0;
    if (o.damp) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward3d<true>, 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward3d<false>, 32, 0);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>((int64_t)std::max(1, per_sm) * std::max(1, sms), 4 * max_items);
    if (o.damp)
        launch_pdl(k_backward3d<true>, (unsigned)grid, 32, 0, stream, rec, rect, tl, W, H, tiles_x, o, T_final, last,
                   dl_dout, grad_img, ch);
    else
        launch_pdl(k_backward3d<false>, (unsigned)grid, 32, 0, stream, rec, rect, tl, W, H, tiles_x, o, T_final, last,
                   dl_dout, grad_img, ch);
    count_launches(1);
}

void launch_chain3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float dilation, int fmode,
                    int sh_degree, const float4* rec, const float* grad_img, float* dl_dparams, cudaStream_t stream) {
    if (N == 0) return;
    Cam3 c;
    for (int k = 0; k < 12; ++k) c.V[k] = cam.viewmat[k];
    c.fx = cam.fx; c.fy = cam.fy; c.cx = cam.cx; c.cy = cam.cy; c.near_z = cam.near_z;
    camera_centre(cam, c.cpos);
    const bool vec = ((reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(dl_dparams)) & 15u) == 0;
    if (vec)
        launch_pdl(k_chain3d<true>, ceil_div(N, 128), 128, 0, stream, params, N, c, W, H, dilation, fmode, sh_degree,
                   rec, grad_img, dl_dparams);
    else
        launch_pdl(k_chain3d<false>, ceil_div(N, 128), 128, 0, stream, params, N, c, W, H, dilation, fmode, sh_degree,
                   rec, grad_img, dl_dparams);
    count_launches(1);
}

}  // namespace wipes
