// Footprint kernels: per-primitive projection to the image plane, the cutoff ellipse, the covered
// pixel range and the number of covered tiles (the binning front end of the 3DGS-style pipeline
// the paper follows, Sec. 4.1), plus the 6D time model.
//
// This translation unit is compiled with -fmad=false: every float expression below is a sequence
// of single IEEE binary32 operations in source order, so the centre, the Cholesky factor of the
// inverse covariance, the extents and the depth are bit-for-bit reproducible.  The tile lists and
// the per-pixel cutoff decision depend only on these values.
#include "common.cuh"

namespace wipes {
namespace {

__device__ __forceinline__ bool finite4(float a, float b, float c, float d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

__device__ __forceinline__ PixRect covered_pixels(float mx, float my, float ex, float ey, int W, int H) {
    float xlo = (mx - ex) - 0.5f;
    float xhi = (mx + ex) - 0.5f;
    float ylo = (my - ey) - 0.5f;
    float yhi = (my + ey) - 0.5f;
    xlo = fminf(fmaxf(xlo, -1.0f), (float)W);
    xhi = fminf(fmaxf(xhi, -1.0f), (float)W);
    ylo = fminf(fmaxf(ylo, -1.0f), (float)H);
    yhi = fminf(fmaxf(yhi, -1.0f), (float)H);
    PixRect r;
    r.u0 = max(0, (int)ceilf(xlo));
    r.u1 = min(W - 1, (int)floorf(xhi));
    r.v0 = max(0, (int)ceilf(ylo));
    r.v1 = min(H - 1, (int)floorf(yhi));
    if (r.u0 > r.u1 || r.v0 > r.v1) { r.u0 = 1; r.u1 = 0; r.v0 = 1; r.v1 = 0; }
    return r;
}

// Number of tiles of each lane's covered pixel range that its cutoff ellipse reaches
// (tile_touched()).  The warp's ranges are laid end to end (an exclusive prefix of their tile
// counts over the lanes) and tested 32 tiles a round: the tile in slot s belongs to the lane whose
// prefix range holds s (a binary search over the lanes' inclusive prefixes), and each lane counts
// the hits in its own slots of the round's ballot.  Every lane of the warp must call it; an empty
// range counts 0.
__device__ __forceinline__ uint32_t warp_tile_counts(float mx, float my, float l11, float l21, float l22,
                                                     const PixRect& r, float lim) {
    const int lane = threadIdx.x & 31;
    Ellipse mine = make_ellipse(0.f, 0.f, 1.f, 0.f, 1.f);
    int tx0 = 0, ty0 = 0, nx = 1, nt = 0;
    if (r.u0 <= r.u1) {
        mine = make_ellipse(mx, my, l11, l21, l22);
        tx0 = r.u0 / kTile, ty0 = r.v0 / kTile;
        nx = r.u1 / kTile - tx0 + 1;
        nt = nx * (r.v1 / kTile - ty0 + 1);
    }
    int incl = nt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - nt;
    uint32_t result = 0;
    for (int s0 = 0; s0 < total; s0 += 32) {
        const int s = s0 + lane;
        int k = 0;  // the number of lanes whose inclusive prefix is at most s: the slot's owner
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
            if (__shfl_sync(0xffffffffu, incl, k + step - 1) <= s) k += step;
        PixRect rk;
        rk.u0 = __shfl_sync(0xffffffffu, r.u0, k);
        rk.u1 = __shfl_sync(0xffffffffu, r.u1, k);
        rk.v0 = __shfl_sync(0xffffffffu, r.v0, k);
        rk.v1 = __shfl_sync(0xffffffffu, r.v1, k);
        Ellipse e;
        e.mx = __shfl_sync(0xffffffffu, mine.mx, k);
        e.my = __shfl_sync(0xffffffffu, mine.my, k);
        e.l11 = __shfl_sync(0xffffffffu, mine.l11, k);
        e.l21 = __shfl_sync(0xffffffffu, mine.l21, k);
        e.l22 = __shfl_sync(0xffffffffu, mine.l22, k);
        e.rBA = __shfl_sync(0xffffffffu, mine.rBA, k);
        e.rBC = __shfl_sync(0xffffffffu, mine.rBC, k);
        const int t = s - __shfl_sync(0xffffffffu, excl, k);
        const int nxk = __shfl_sync(0xffffffffu, nx, k);
        const int txk = __shfl_sync(0xffffffffu, tx0, k), tyk = __shfl_sync(0xffffffffu, ty0, k);
        const int row = t / nxk, col = t - row * nxk;
        const bool hit = s < total && tile_touched(e, rk, txk + col, tyk + row, lim);
        const uint32_t hits = __ballot_sync(0xffffffffu, hit);
        // this lane's slots of the round: [excl, incl) within [s0, s0 + 32)
        const int lo = max(excl - s0, 0), hi = min(incl - s0, 32);
        if (lo < hi) result += (uint32_t)__popc((hits >> lo) & (0xffffffffu >> (32 - (hi - lo))));
    }
    return result;
}

__device__ __forceinline__ void write_empty(int64_t i, float4* rec, PixRect* rect, uint32_t* counts,
                                            uint32_t* depth_keys) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    rec[i * kRecF4 + 0] = z; rec[i * kRecF4 + 1] = z; rec[i * kRecF4 + 2] = z; rec[i * kRecF4 + 3] = z;
    PixRect e; e.u0 = 1; e.u1 = 0; e.v0 = 1; e.v1 = 0;
    rect[i] = e;
    counts[i] = 0u;
    if (depth_keys) depth_keys[i] = 0xFFFFFFFFu;
}

// cos and sin of a 2D rotation angle for the footprint rule: a fixed sequence of IEEE operations
// (each written as its correctly rounded intrinsic, so no contraction or reassociation can change
// a bit), with no library transcendental.  Any IEEE evaluation of the sequence gives the same
// bits, which keeps the tile lists bit-exact without relying on two math libraries agreeing.
// |th| <= 2^16 (the common case, rule_cos_sin): binary32 arithmetic with fused multiply-adds.
// Reduction by Cody and Waite: k = rint(th * 2/pi), r = th - k pi/2 with pi/2 in three binary32
// pieces; the first product is exact (th and k P1 are multiples of 2^-23, or of 2^-24 when
// |th| < 1, and differ by less than 1).  Then the Taylor series of sin r to r^11 and cos r to r^10
// (|r| <= pi/4 + 0.01, truncation below 2e-10) in Horner form in z = r^2; k mod 4 selects the
// quadrant.  Each result is within one binary32 ulp of the correctly rounded value.
// 2^16 < |th| <= 1e15 (rule_cos_sin_wide): the same steps in binary64 (pi/2 in three pieces of 33,
// 33 and 53 significant bits, k times the first two exact for |k| < 2^20; Taylor series to r^17
// and r^18), rounded once to binary32.  A larger or non-finite th gives NaN (the primitive becomes
// invalid).
__device__ __noinline__ void rule_cos_sin_wide(double th, float& c, float& s) {
    if (!(fabs(th) <= 1e15)) {
        c = s = __int_as_float(0x7fc00000);
        return;
    }
    const double k = rint(__dmul_rn(th, 0x1.45f306dc9c883p-1));
    double r = __dsub_rn(th, __dmul_rn(k, 0x1.921fb544p+0));
    r = __dsub_rn(r, __dmul_rn(k, 0x1.0b4611a6p-34));
    r = __dsub_rn(r, __dmul_rn(k, 0x1.3198a2e037073p-69));
    const double z = __dmul_rn(r, r);
    // sin: coefficients 1/17!, -1/15!, ..., -1/3!
    double ps = 0x1.952c77030ad4ap-49;
    ps = __dsub_rn(__dmul_rn(ps, z), 0x1.ae7f3e733b81fp-41);
    ps = __dadd_rn(__dmul_rn(ps, z), 0x1.6124613a86d09p-33);
    ps = __dsub_rn(__dmul_rn(ps, z), 0x1.ae64567f544e4p-26);
    ps = __dadd_rn(__dmul_rn(ps, z), 0x1.71de3a556c734p-19);
    ps = __dsub_rn(__dmul_rn(ps, z), 0x1.a01a01a01a01ap-13);
    ps = __dadd_rn(__dmul_rn(ps, z), 0x1.1111111111111p-7);
    ps = __dsub_rn(__dmul_rn(ps, z), 0x1.5555555555555p-3);
    const double sr = __dadd_rn(r, __dmul_rn(__dmul_rn(r, z), ps));
    // cos: coefficients -1/18!, 1/16!, ..., -1/2!
    double pc = -0x1.6827863b97d97p-53;
    pc = __dadd_rn(__dmul_rn(pc, z), 0x1.ae7f3e733b81fp-45);
    pc = __dsub_rn(__dmul_rn(pc, z), 0x1.93974a8c07c9dp-37);
    pc = __dadd_rn(__dmul_rn(pc, z), 0x1.1eed8eff8d898p-29);
    pc = __dsub_rn(__dmul_rn(pc, z), 0x1.27e4fb7789f5cp-22);
    pc = __dadd_rn(__dmul_rn(pc, z), 0x1.a01a01a01a01ap-16);
    pc = __dsub_rn(__dmul_rn(pc, z), 0x1.6c16c16c16c17p-10);
    pc = __dadd_rn(__dmul_rn(pc, z), 0x1.5555555555555p-5);
    pc = __dsub_rn(__dmul_rn(pc, z), 0.5);
    const double cr = __dadd_rn(1.0, __dmul_rn(z, pc));
    switch ((int)((long long)k & 3)) {
        case 0: c = __double2float_rn(cr); s = __double2float_rn(sr); break;
        case 1: c = __double2float_rn(-sr); s = __double2float_rn(cr); break;
        case 2: c = __double2float_rn(-cr); s = __double2float_rn(-sr); break;
        default: c = __double2float_rn(sr); s = __double2float_rn(-cr); break;
    }
}

__device__ __forceinline__ void rule_cos_sin(float th, float& c, float& s) {
    if (!(fabsf(th) <= 0x1p16f)) {
        rule_cos_sin_wide((double)th, c, s);
        return;
    }
    const float k = rintf(__fmul_rn(th, 0x1.45f306p-1f));  // th 2/pi
    float r = __fmaf_rn(-k, 0x1.921fb6p+0f, th);           // - k P1, exact
    r = __fmaf_rn(-k, -0x1.777a5cp-25f, r);                // - k P2
    r = __fmaf_rn(-k, -0x1.ee59dap-50f, r);                // - k P3
    const float z = __fmul_rn(r, r);
    // sin: coefficients -1/11!, 1/9!, ..., -1/3! (binary32)
    float ps = -0x1.ae6456p-26f;
    ps = __fmaf_rn(ps, z, 0x1.71de3ap-19f);
    ps = __fmaf_rn(ps, z, -0x1.a01a02p-13f);
    ps = __fmaf_rn(ps, z, 0x1.111112p-7f);
    ps = __fmaf_rn(ps, z, -0x1.555556p-3f);
    const float sr = __fmaf_rn(__fmul_rn(r, z), ps, r);
    // cos: coefficients -1/10!, 1/8!, ..., -1/2!
    float pc = -0x1.27e4fcp-22f;
    pc = __fmaf_rn(pc, z, 0x1.a01a02p-16f);
    pc = __fmaf_rn(pc, z, -0x1.6c16c2p-10f);
    pc = __fmaf_rn(pc, z, 0x1.555556p-5f);
    pc = __fmaf_rn(pc, z, -0.5f);
    const float cr = __fmaf_rn(z, pc, 1.0f);
    switch ((int)k & 3) {
        case 0: c = cr; s = sr; break;
        case 1: c = -sr; s = cr; break;
        case 2: c = -cr; s = -sr; break;
        default: c = sr; s = -cr; break;
    }
}

// 2D, RS record (cov2d = 0): Sigma = R(theta) diag(sx^2, sy^2) R(theta)^T;
// Sigma^-1 = R diag(1/sx^2, 1/sy^2) R^T, whose Cholesky factor is l11 = sqrt(A), l21 = B / l11,
// l22 = sqrt(det)/l11 = 1 / (sx sy l11).
// 2D, Cholesky record (cov2d = 1, Sec. 5.1): Sigma = L L^T, L = [[l1, 0], [l2, l3]]; with
// u = l2^2 + l3^2 = Sigma_yy: l11 = sqrt(u) / |l1 l3|, l21 = -l1 l2 / (|l1 l3| sqrt(u)), l22 = 1/sqrt(u).
__global__ void __launch_bounds__(256) k_footprint2d(const float4* __restrict__ params, int64_t N, int W, int H,
                                                     float cutoff, int cov2d, float lim, float4* __restrict__ rec,
                                                     PixRect* __restrict__ rect, uint32_t* __restrict__ counts) {
    pdl_enter();
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < N;
    const int64_t i = live ? i0 : N - 1;  // lanes past the end repeat the last primitive, write nothing
    const float4 p0 = params[i * 4 + 0];  // mu_x mu_y s_x s_y   | mu_x mu_y l1 l2
    const float4 p1 = params[i * 4 + 1];  // theta f_x f_y phi   | l3 f_x f_y phi
    const float4 p2 = params[i * 4 + 2];  // c_r c_g c_b -
    float l11, l21, l22, ex, ey;
    bool shape_ok;
    if (cov2d) {
        const float a = p0.z, b = p0.w, c = p1.x;
        const float u = b * b + c * c;
        const float su = sqrtf(u);
        const float aac = fabsf(a * c);
        l11 = su / aac;
        l21 = -(a * b) / (aac * su);
        l22 = 1.0f / su;
        const float vxx = a * a;
        ex = (cutoff * sqrtf(vxx)) * kExtMargin;
        ey = (cutoff * su) * kExtMargin;
        shape_ok = aac > 0.0f;
    } else {
        const float sx = p0.z, sy = p0.w;
        float c, s;
        rule_cos_sin(p1.x, c, s);
        const float sx2 = sx * sx, sy2 = sy * sy;
        const float ix = 1.0f / sx2, iy = 1.0f / sy2;
        const float cc = c * c, ss = s * s, cs = c * s;
        const float A = cc * ix + ss * iy;
        const float B = cs * (ix - iy);
        l11 = sqrtf(A);
        l21 = B / l11;
        l22 = 1.0f / ((sx * sy) * l11);
        const float vxx = cc * sx2 + ss * sy2;
        const float vyy = ss * sx2 + cc * sy2;
        ex = (cutoff * sqrtf(vxx)) * kExtMargin;
        ey = (cutoff * sqrtf(vyy)) * kExtMargin;
        shape_ok = sx > 0.0f && sy > 0.0f;
    }
    const float mx = p0.x, my = p0.y;
    const bool valid = finite4(mx, my, l11, l21) && finite4(l22, ex, ey, 1.0f) && shape_ok && l11 > 0.0f && l22 > 0.0f;
    PixRect r;
    r.u0 = 1; r.u1 = 0; r.v0 = 1; r.v1 = 0;
    if (valid && live) r = covered_pixels(mx, my, ex, ey, W, H);
    const uint32_t cnt = warp_tile_counts(mx, my, l11, l21, l22, r, lim);
    if (!live) return;
    if (!valid) { write_empty(i, rec, rect, counts, nullptr); return; }
    rec[i * kRecF4 + 0] = make_float4(mx, my, l11, l21);
    rec[i * kRecF4 + 1] = make_float4(l22, p1.y, p1.z, p1.w * kInvTwoPi);
    rec[i * kRecF4 + 2] = make_float4(p2.x, p2.y, p2.z, 1.0f);
    rec[i * kRecF4 + 3] = make_float4(ex, ey, 0.0f, 0.0f);
    rect[i] = r;
    counts[i] = cnt;
}

struct Cam {
    float V[12];
    float fx, fy, cx, cy, near_z;
    float cpos[3];  // camera centre in world coordinates (spherical-harmonic colour)
};

// 3D: camera-frame centre t = V mu + t0; P = J V R(q) S (2x3), Sigma' = P P^T + dil I with the
// local affine Jacobian J of the perspective map (Sec. 3.1).  det Sigma' is evaluated as
// |P0 x P1|^2 + dil (|P0|^2 + |P1|^2) + dil^2, a sum of non-negative terms.
// Cholesky of Sigma'^-1: l22 = 1/sqrt(S11), l11 = sqrt(S11/D), l21 = -S01/sqrt(S11 D).
// Frequency: fc = V f; fmode 0: f' = (fc_x tz / fx, fc_y tz / fy) (phase gradient on the
// fronto-parallel plane through the centre; the viewing-axis component is dropped, Sec. 4.1);
// fmode 1: f' = J fc (the same W and J as the covariance, read literally, Sec. 4.1).
// Colour: the record's c, or with sh_degree > 0 (records of WIPES_P3D_SH floats)
// max(0, 1/2 + sum_k Y_k(dir) sh_k) per channel, dir the unit vector from the camera centre to mu.
__global__ void __launch_bounds__(256) k_footprint3d(const float* __restrict__ params, int64_t N, Cam cam, int W,
                                                     int H, float cutoff, float lim, float dil, int fmode,
                                                     int sh_degree, float4* __restrict__ rec,
                                                     PixRect* __restrict__ rect, uint32_t* __restrict__ counts,
                                                     uint32_t* __restrict__ depth_keys) {
    pdl_enter();
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < N;
    const int64_t i = live ? i0 : N - 1;  // lanes past the end repeat the last primitive, write nothing
    const int stride = sh_degree ? WIPES_P3D_SH : WIPES_P3D;
    const float4* pp = reinterpret_cast<const float4*>(params + i * stride);
    const float4 a0 = pp[0], a1 = pp[1], a2 = pp[2], a3 = pp[3], a4 = pp[4];
    float p[20] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y,
                   a2.z, a2.w, a3.x, a3.y, a3.z, a3.w, a4.x, a4.y, a4.z, a4.w};
    const float* V = cam.V;
    const float tx = ((V[0] * p[0] + V[1] * p[1]) + V[2] * p[2]) + V[3];
    const float ty = ((V[4] * p[0] + V[5] * p[1]) + V[6] * p[2]) + V[7];
    const float tz = ((V[8] * p[0] + V[9] * p[1]) + V[10] * p[2]) + V[11];
    const bool in_front = tz > cam.near_z && isfinite(tz) && isfinite(tx) && isfinite(ty);
    float qw = p[6], qx = p[7], qy = p[8], qz = p[9];
    const float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    const float r = sqrtf(n2);
    qw = qw / r; qx = qx / r; qy = qy / r; qz = qz / r;
    const float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    const float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    const float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[a * 3 + b] = R[a * 3 + b] * p[3 + b];
    float Q[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Q[a * 3 + b] = (V[a * 4 + 0] * M[0 * 3 + b] + V[a * 4 + 1] * M[1 * 3 + b]) + V[a * 4 + 2] * M[2 * 3 + b];
    const float limx = 1.3f * ((0.5f * (float)W) / cam.fx);
    const float limy = 1.3f * ((0.5f * (float)H) / cam.fy);
    const float txz = fminf(limx, fmaxf(-limx, tx / tz));
    const float tyz = fminf(limy, fmaxf(-limy, ty / tz));
    const float j00 = cam.fx / tz, j02 = -((cam.fx * txz) / tz);
    const float j11 = cam.fy / tz, j12 = -((cam.fy * tyz) / tz);
    float P0[3], P1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        P0[b] = j00 * Q[0 * 3 + b] + j02 * Q[2 * 3 + b];
        P1[b] = j11 * Q[1 * 3 + b] + j12 * Q[2 * 3 + b];
    }
    const float n0 = (P0[0] * P0[0] + P0[1] * P0[1]) + P0[2] * P0[2];
    const float n1 = (P1[0] * P1[0] + P1[1] * P1[1]) + P1[2] * P1[2];
    const float s01 = (P0[0] * P1[0] + P0[1] * P1[1]) + P0[2] * P1[2];
    const float c0 = P0[1] * P1[2] - P0[2] * P1[1];
    const float c1 = P0[2] * P1[0] - P0[0] * P1[2];
    const float c2 = P0[0] * P1[1] - P0[1] * P1[0];
    const float S00 = n0 + dil, S11 = n1 + dil;
    const float D = (((c0 * c0 + c1 * c1) + c2 * c2) + dil * (n0 + n1)) + dil * dil;
    const float l22 = 1.0f / sqrtf(S11);
    const float l11 = sqrtf(S11 / D);
    const float l21 = -(s01 / sqrtf(S11 * D));
    const float mx = ((cam.fx * tx) / tz) + cam.cx;
    const float my = ((cam.fy * ty) / tz) + cam.cy;
    const float ex = (cutoff * sqrtf(S00)) * kExtMargin;
    const float ey = (cutoff * sqrtf(S11)) * kExtMargin;
    const bool valid = in_front && finite4(mx, my, l11, l21) && finite4(l22, ex, ey, D) && D > 0.0f && S11 > 0.0f &&
                       l11 > 0.0f && l22 > 0.0f;
    PixRect rr;
    rr.u0 = 1; rr.u1 = 0; rr.v0 = 1; rr.v1 = 0;
    if (valid && live) rr = covered_pixels(mx, my, ex, ey, W, H);
    const uint32_t cnt = warp_tile_counts(mx, my, l11, l21, l22, rr, lim);
    if (!live) return;
    if (!valid) { write_empty(i, rec, rect, counts, depth_keys); return; }
    // projected frequency (not part of any integer decision)
    const float fcx = (V[0] * p[10] + V[1] * p[11]) + V[2] * p[12];
    const float fcy = (V[4] * p[10] + V[5] * p[11]) + V[6] * p[12];
    float fpx, fpy, hk = 0.5f;
    if (fmode == 2) {
        // the oscillation integrated along the viewing ray (Sec. 4.1's integral over z) in the EWA
        // ray space: n = (txz, tyz, 1) the ray direction (J n = 0), A = V R the camera-frame
        // principal axes; m = A^T n, w = S^-2 m, c = n^T Sigma_c^-1 n = m . w, b = Sigma_c^-1 n = A w,
        // fn = fc . n;  f' = P0^T (fc - (fn / c) b) with P0^T v = (v_x tz / fx, v_y tz / fy), and the
        // damping kappa = exp(-2 pi^2 fn^2 / c) = ex2(kx)
        const float fcz = (V[8] * p[10] + V[9] * p[11]) + V[10] * p[12];
        float A[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                A[a * 3 + b] = (V[a * 4 + 0] * R[0 * 3 + b] + V[a * 4 + 1] * R[1 * 3 + b]) + V[a * 4 + 2] * R[2 * 3 + b];
        float m[3], w[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            m[b] = (A[0 * 3 + b] * txz + A[1 * 3 + b] * tyz) + A[2 * 3 + b];
            w[b] = m[b] / (p[3 + b] * p[3 + b]);
        }
        const float cq = (m[0] * w[0] + m[1] * w[1]) + m[2] * w[2];
        const float bx = (A[0] * w[0] + A[1] * w[1]) + A[2] * w[2];
        const float by = (A[3] * w[0] + A[4] * w[1]) + A[5] * w[2];
        const float fn = (fcx * txz + fcy * tyz) + fcz;
        const float rr = fn / cq;
        fpx = ((fcx - rr * bx) * tz) / cam.fx;
        fpy = ((fcy - rr * by) * tz) / cam.fy;
        hk = 0.5f * ex2_approx(-((kDampExp2 * fn) * rr));
    } else if (fmode) {
        const float fcz = (V[8] * p[10] + V[9] * p[11]) + V[10] * p[12];
        fpx = j00 * fcx + j02 * fcz;
        fpy = j11 * fcy + j12 * fcz;
    } else {
        fpx = fcx * tz / cam.fx;
        fpy = fcy * tz / cam.fy;
    }
    float col[3] = {p[15], p[16], p[17]};
    if (sh_degree) {
        const float vx = p[0] - cam.cpos[0], vy = p[1] - cam.cpos[1], vz = p[2] - cam.cpos[2];
        const float dist = sqrtf(vx * vx + vy * vy + vz * vz);
        float Y[kShMaxCoeffs];
        sh_eval(vx / dist, vy / dist, vz / dist, Y);
        const int nk = (sh_degree + 1) * (sh_degree + 1);
        // the coefficients of degree >= 1 (slots 20 .. 67, the row 16-byte aligned) in 16-byte pieces
        float q[WIPES_P3D_SH];
#pragma unroll
        for (int k = 15; k < 18; ++k) q[k] = p[k];
        load_row<true, WIPES_P3D_SH - WIPES_P3D>(q + WIPES_P3D, params + i * stride + WIPES_P3D);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float r = 0.5f;
#pragma unroll
            for (int k = 0; k < kShMaxCoeffs; ++k)
                if (k < nk) r += Y[k] * q[sh_slot(k, ch)];
            col[ch] = fmaxf(r, 0.f);
        }
    }
    rec[i * kRecF4 + 0] = make_float4(mx, my, l11, l21);
    rec[i * kRecF4 + 1] = make_float4(l22, fpx, fpy, p[13] * kInvTwoPi);
    rec[i * kRecF4 + 2] = make_float4(col[0], col[1], col[2], p[14]);
    rec[i * kRecF4 + 3] = make_float4(ex, ey, tz, hk);
    rect[i] = rr;
    counts[i] = cnt;
    depth_keys[i] = __float_as_uint(tz);
}

// VEC (both kernels): the caller's rows are 16-byte aligned and move in 16-byte pieces.
template <bool VEC>
__global__ void __launch_bounds__(256) k_deform6d(const float* __restrict__ p6, int64_t N, float t,
                                                  float* __restrict__ p3) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float a[WIPES_P6D], o[WIPES_P3D];
    load_row<VEC, WIPES_P6D>(a, p6 + i * WIPES_P6D);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // single rounding of mu0 + v t (and of f, phi below): the correctly rounded linear model
        o[j] = __fmaf_rn(a[20 + j], t, a[j]);
        o[3 + j] = a[3 + j] * expf(a[27 + j] * t);
        o[10 + j] = __fmaf_rn(a[23 + j], t, a[10 + j]);
    }
#pragma unroll
    for (int j = 6; j < 10; ++j) o[j] = a[j];
    o[13] = __fmaf_rn(a[26], t, a[13]);
#pragma unroll
    for (int j = 14; j < 20; ++j) o[j] = a[j];
    store_row<VEC, WIPES_P3D>(p3 + i * WIPES_P3D, o);
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_deform6d_backward(const float* __restrict__ p6, int64_t N, float t,
                                                           const float* __restrict__ g3, float* __restrict__ g6,
                                                           int accumulate) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float a[WIPES_P6D], g[WIPES_P3D], o[WIPES_P6D];
    load_row<VEC, WIPES_P6D>(a, p6 + i * WIPES_P6D);
    load_row<VEC, WIPES_P3D>(g, g3 + i * WIPES_P3D);
#pragma unroll
    for (int j = 0; j < WIPES_P6D; ++j) o[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < 20; ++j) o[j] = g[j];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float e = expf(a[27 + j] * t);
        o[3 + j] = g[3 + j] * e;
        o[20 + j] = g[j] * t;
        o[23 + j] = g[10 + j] * t;
        o[27 + j] = g[3 + j] * a[3 + j] * e * t;
    }
    o[26] = g[13] * t;
    float* out = g6 + i * WIPES_P6D;
    if (accumulate) {
        float prev[WIPES_P6D];
        load_row<VEC, WIPES_P6D>(prev, out);
#pragma unroll
        for (int j = 0; j < WIPES_P6D; ++j) o[j] = prev[j] + o[j];
    }
    store_row<VEC, WIPES_P6D>(out, o);
}

}  // namespace

void launch_footprint2d(const float* params, int64_t N, int W, int H, float cutoff, int cov2d, float4* rec, PixRect* rect,
                        uint32_t* counts, uint32_t* /*depth_keys*/, cudaStream_t stream) {
    if (N == 0) return;
    launch_pdl(k_footprint2d, ceil_div(N, 256), 256, 0, stream, reinterpret_cast<const float4*>(params), N, W, H, cutoff,
               cov2d, touch_limit(cutoff), rec, rect, counts);
    count_launches(1);
}

void launch_footprint3d(const float* params, int64_t N, const wipes_camera& cam, int W, int H, float cutoff,
                        float dilation, int fmode, int sh_degree, float4* rec, PixRect* rect, uint32_t* counts,
                        uint32_t* depth_keys, cudaStream_t stream) {
    if (N == 0) return;
    Cam c;
    for (int k = 0; k < 12; ++k) c.V[k] = cam.viewmat[k];
    c.fx = cam.fx; c.fy = cam.fy; c.cx = cam.cx; c.cy = cam.cy; c.near_z = cam.near_z;
    camera_centre(cam, c.cpos);
    launch_pdl(k_footprint3d, ceil_div(N, 256), 256, 0, stream, params, N, c, W, H, cutoff, touch_limit(cutoff), dilation,
               fmode, sh_degree, rec, rect, counts, depth_keys);
    count_launches(1);
}

void launch_deform6d(const float* params6, int64_t N, float t, float* params3, cudaStream_t stream) {
    if (N == 0) return;
    if (((reinterpret_cast<uintptr_t>(params6) | reinterpret_cast<uintptr_t>(params3)) & 15u) == 0)
        launch_pdl(k_deform6d<true>, ceil_div(N, 256), 256, 0, stream, params6, N, t, params3);
    else
        launch_pdl(k_deform6d<false>, ceil_div(N, 256), 256, 0, stream, params6, N, t, params3);
    count_launches(1);
}

void launch_deform6d_backward(const float* params6, int64_t N, float t, const float* g3, float* g6, int accumulate,
                              cudaStream_t stream) {
    if (N == 0) return;
    const uintptr_t ptrs = reinterpret_cast<uintptr_t>(params6) | reinterpret_cast<uintptr_t>(g3) |
                           reinterpret_cast<uintptr_t>(g6);
    if ((ptrs & 15u) == 0)
        launch_pdl(k_deform6d_backward<true>, ceil_div(N, 256), 256, 0, stream, params6, N, t, g3, g6, accumulate);
    else
        launch_pdl(k_deform6d_backward<false>, ceil_div(N, 256), 256, 0, stream, params6, N, t, g3, g6, accumulate);
    count_launches(1);
}

}  // namespace wipes
