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

// One block per 8x8 quad, tiles taken in the given order (longest list first).
__global__ void __launch_bounds__(kQuadThreads) k_blend3d(BlendJob job, const uint32_t* __restrict__ order) {
    pdl_enter();
    blend3d_quad(job, (int)order[blockIdx.x >> 2], (int)(blockIdx.x & 3u));
}

// Image-plane gradient per primitive (12 floats): mx my l11 l21 l22 fx fy phc c_r c_g c_b o
constexpr int kG = 12;

// Backward.  Each pixel walks its tile list back to front from its last contributor, recovering
// the transmittance in front of each contributor as T_i = T_{i+1} / (1 - alpha_i) from the stored
// final value.  Blocks of kQuadThreads take one 8x8 quad of a tile (tiles in the given order,
// longest list first); warps visit only the entries marked for their 8x4 sub-tile, and a warp's
// per-pixel gradients of one primitive are summed by a reduce-scatter and added to the
// primitive's image-plane gradient with one atomic per component.  As in the forward pass, the
// records of the next batch are loaded while the current one is processed.
__global__ void __launch_bounds__(kQuadThreads) k_backward3d(const float4* __restrict__ rec,
                                                             const PixRect* __restrict__ rect, TileLists tl, int W,
                                                             int H, int tiles_x, BlendOpts3 o,
                                                             const float* __restrict__ T_final,
                                                             const uint32_t* __restrict__ last,
                                                             const float* __restrict__ dl_dout,
                                                             float* __restrict__ grad_img,
                                                             const uint32_t* __restrict__ order) {
    pdl_enter();
    __shared__ float4 s_a[kQuadThreads];
    __shared__ float4 s_b[kQuadThreads];
    __shared__ float4 s_c[kQuadThreads];
    __shared__ uint32_t s_id[kQuadThreads];
    __shared__ uint8_t s_mask[kQuadThreads];
    __shared__ uint32_t s_max_last;
    const int tile = (int)order[blockIdx.x >> 2], quad = (int)(blockIdx.x & 3u);
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int x0 = tx * kTile + (quad & 1) * 8, y0 = ty * kTile + (quad >> 1) * 8;
    const int u = x0 + (lane & 7), v = y0 + warp * 4 + (lane >> 3);
    const bool inside = u < W && v < H;
    const float px = (float)u + 0.5f, py = (float)v + 0.5f;
    const uint2 range = tl.ranges[tile];
    const size_t pix = (size_t)v * W + u;
    float T = inside ? T_final[pix] : 1.f;
    const uint32_t my_last = inside ? last[pix] : 0u;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) { g0 = dl_dout[pix * 3 + 0]; g1 = dl_dout[pix * 3 + 1]; g2 = dl_dout[pix * 3 + 2]; }
    // colour accumulated behind the current primitive, starting with the background term
    float S0 = T * o.bg[0], S1 = T * o.bg[1], S2 = T * o.bg[2];
    if (t == 0) s_max_last = 0u;
    __syncthreads();
    atomicMax(&s_max_last, my_last);
    __syncthreads();
    // entries past every pixel's last contributor are skipped; batches run [b0, b_end) downwards
    const uint32_t end = range.x + s_max_last;
    uint32_t b_end = end;
    uint32_t b0 = end - min(end - range.x, (uint32_t)kQuadThreads);
    // software pipeline: records (and id) of the batch to stage next, id of the batch after it
    float4 nA = make_float4(0.f, 0.f, 0.f, 0.f), nB = nA, nC = nA;
    PixRect nR{0, 0, -1, -1};
    uint32_t nid = 0u, np = 0u;
    if (b0 + t < b_end) {
        nid = tl.prim[b0 + t];
        nA = rec[(size_t)nid * kRecF4 + 0];
        nB = rec[(size_t)nid * kRecF4 + 1];
        nC = rec[(size_t)nid * kRecF4 + 2];
        nR = rect[nid];
    }
    uint32_t nb0 = b0 - min(b0 - range.x, (uint32_t)kQuadThreads);  // start of the next batch
    if (nb0 + t < b0) np = tl.prim[nb0 + t];
    while (b_end > range.x) {
        const int n = (int)(b_end - b0);
        __syncthreads();
        if (t < n) {
            s_id[t] = nid;
            s_a[t] = nA;
            s_b[t] = nB;
            s_c[t] = nC;
            s_mask[t] = (uint8_t)quad_mask_ellipse(nA, nB.x, nR, x0, y0, o.lim);
        }
        __syncthreads();
        // loads for the next two batches: [nb0, b0) and [nnb0, nb0)
        const uint32_t nnb0 = nb0 - min(nb0 - range.x, (uint32_t)kQuadThreads);
        if (nb0 + t < b0) {
            nid = np;
            nA = rec[(size_t)nid * kRecF4 + 0];
            nB = rec[(size_t)nid * kRecF4 + 1];
            nC = rec[(size_t)nid * kRecF4 + 2];
            nR = rect[nid];
        }
        if (nnb0 + t < nb0) np = tl.prim[nnb0 + t];
        for (int c = (n - 1) & ~31; c >= 0; c -= 32) {
            const uint32_t m = c + lane < n ? s_mask[c + lane] : 0u;
            uint32_t bal = __ballot_sync(0xffffffffu, (m >> warp) & 1u);
            while (bal) {
                const int hb = 31 - __clz(bal);
                bal &= ~(1u << hb);
                const int j = c + hb;
                const uint32_t pos = b0 - range.x + (uint32_t)j + 1u;  // 1-based position in the tile list
                bool contrib = false;
                float acc[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = 0.f;
                const float4 A = s_a[j];
                const float4 B = s_b[j];
                if (pos <= my_last) {
                    const float q = mahalanobis2(px, py, A.x, A.y, A.z, A.w, B.x);
                    if (q <= o.cutoff2) {
                        const float dx = px - A.x, dy = py - A.y;
                        const float G = ex2_approx(q * kNegHalfLog2e);
                        const float ang = reduced_angle(fmaf(B.y, dx, fmaf(B.z, dy, B.w)));
                        const float cs = cos_approx(ang);
                        const float w = fmaf(0.5f, cs, 0.5f) * G;
                        const float4 C = s_c[j];
                        const float raw = C.w * w;
                        const float alpha = fminf(o.alpha_max, raw);
                        if (alpha >= o.alpha_min) {
                            contrib = true;
                            const float om = 1.f - alpha;
                            T = T / om;
                            const float wt = alpha * T;
                            acc[8] = g0 * wt;
                            acc[9] = g1 * wt;
                            acc[10] = g2 * wt;
                            const float inv = 1.f / om;
                            const float galpha = g0 * (C.x * T - S0 * inv) + g1 * (C.y * T - S1 * inv) +
                                                 g2 * (C.z * T - S2 * inv);
                            S0 = fmaf(C.x, wt, S0);
                            S1 = fmaf(C.y, wt, S1);
                            S2 = fmaf(C.z, wt, S2);
                            if (raw < o.alpha_max) {
                                acc[11] = galpha * w;
                                const float gW = galpha * C.w;
                                const float sn = sin_approx(ang);
                                const float a = fmaf(A.z, dx, A.w * dy), b = B.x * dy;
                                const float gq2 = -gW * w;
                                const float gt = (-kPi * G) * (gW * sn);
                                const float ga = gq2 * a, gb = gq2 * b;
                                acc[2] = ga * dx;
                                acc[3] = ga * dy;
                                acc[4] = gb * dy;
                                acc[0] = -fmaf(ga, A.z, gt * B.y);
                                acc[1] = -fmaf(ga, A.w, fmaf(gb, B.x, gt * B.z));
                                acc[5] = gt * dx;
                                acc[6] = gt * dy;
                                acc[7] = gt;
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    const float tot = warp_reduce_scatter16(acc);
                    if ((lane & 1) == 0 && (lane >> 1) < kG) atomicAdd(grad_img + (size_t)s_id[j] * kG + (lane >> 1), tot);
                }
            }
        }
        b_end = b0;
        b0 = nb0;
        nb0 = nnb0;
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
__global__ void __launch_bounds__(128) k_chain3d(const float* __restrict__ params, int64_t N, Cam3 cam, int W, int H,
                                                 float dil, int fmode, int sh_degree, const float4* __restrict__ rec,
                                                 const float* __restrict__ grad_img, float* __restrict__ dl_dparams) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int stride = sh_degree ? WIPES_P3D_SH : WIPES_P3D;
    float* out = dl_dparams + i * stride;
    const float4 r0 = rec[(size_t)i * kRecF4 + 0];
    if (!(r0.z > 0.f)) {  // culled or degenerate: no gradient
        for (int k = 0; k < stride; ++k) out[k] = 0.f;
        return;
    }
    const float* p = params + i * stride;
    const float* g = grad_img + (size_t)i * kG;
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
    float gqn[4];
    quat_rot_grad(qn, gR, gqn);
    const float dot = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
    // camera-frame frequency; with f' = J fc (fmode 1) dL/dJ gains dL/df' fc^T
    const float fcx = V[0] * p[10] + V[1] * p[11] + V[2] * p[12];
    const float fcy = V[4] * p[10] + V[5] * p[11] + V[6] * p[12];
    const float fcz = V[8] * p[10] + V[9] * p[11] + V[10] * p[12];
    if (fmode) {
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
    if (!fmode) gtz += g_fx * fcx / cam.fx + g_fy * fcy / cam.fy;
    gtz += -gj00 * cam.fx * iz2 - gj11 * cam.fy * iz2 + gj02 * cam.fx * txz * iz2 + gj12 * cam.fy * tyz * iz2;
    if (free_x) {
        gtx += -gj02 * cam.fx * iz2;
        gtz += gj02 * cam.fx * tx * iz2 * iz;
    }
    if (free_y) {
        gty += -gj12 * cam.fy * iz2;
        gtz += gj12 * cam.fy * ty * iz2 * iz;
    }
    const float gfc0 = fmode ? g_fx * j00 : g_fx * tz / cam.fx;
    const float gfc1 = fmode ? g_fy * j11 : g_fy * tz / cam.fy;
    const float gfc2 = fmode ? g_fx * j02 + g_fy * j12 : 0.f;
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
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float raw = 0.5f;
#pragma unroll
            for (int k = 0; k < kShMaxCoeffs; ++k)
                if (k < nk) raw += Y[k] * p[sh_slot(k, ch)];
            const float gc = raw > 0.f ? g[8 + ch] : 0.f;
#pragma unroll
            for (int k = 0; k < kShMaxCoeffs; ++k) {
                if (k >= nk) continue;
                const float c = p[sh_slot(k, ch)];
                out[sh_slot(k, ch)] = gc * Y[k];
                gdx += gc * c * Yx[k];
                gdy += gc * c * Yy[k];
                gdz += gc * c * Yz[k];
            }
        }
        for (int k = 20 + 3 * (nk - 1); k < WIPES_P3D_SH; ++k) out[k] = 0.f;
        const float dd = gdx * dx + gdy * dy + gdz * dz;
        out[0] += (gdx - dd * dx) / dist;
        out[1] += (gdy - dd * dy) / dist;
        out[2] += (gdz - dd * dz) / dist;
    }
}

}  // namespace

void launch_blend3d(const BlendJob& job, int tiles_y, const uint32_t* order, cudaStream_t stream) {
    launch_pdl(k_blend3d, 4 * job.tiles_x * tiles_y, kQuadThreads, 0, stream, job, order);
    count_launches(1);
}

void launch_backward3d(const float4* rec, const PixRect* rect, const TileLists& tl, int W, int H, int tiles_x,
                       int tiles_y, const BlendOpts3& o, const float* T_final, const uint32_t* last,
                       const float* dl_dout, float* grad_img, const uint32_t* order, cudaStream_t stream) {
    launch_pdl(k_backward3d, 4 * tiles_x * tiles_y, kQuadThreads, 0, stream, rec, rect, tl, W, H, tiles_x, o, T_final,
                                                                      last, dl_dout, grad_img, order);
    count_launches(1);
}

void launch_chain3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float dilation, int fmode,
                    int sh_degree, const float4* rec, const float* grad_img, float* dl_dparams, cudaStream_t stream) {
    if (N == 0) return;
    Cam3 c;
    for (int k = 0; k < 12; ++k) c.V[k] = cam.viewmat[k];
    c.fx = cam.fx; c.fy = cam.fy; c.cx = cam.cx; c.cy = cam.cy; c.near_z = cam.near_z;
    camera_centre(cam, c.cpos);
    launch_pdl(k_chain3d, ceil_div(N, 128), 128, 0, stream, params, N, c, W, H, dilation, fmode, sh_degree, rec,
               grad_img, dl_dparams); count_launches(1);
}

}  // namespace wipes
