/*
 * WIPES oracle: a plain, slow, brute-force CPU reference of the wavelet rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg load this file.  The product library never links, includes or calls it, and it shares no
 * code with the CUDA path.
 *
 * What it computes (paper: "WIPES: Wavelet-based Visual Primitives", ICCV 2025):
 *   - the wavelet primitive  W(x) = 1/2 [cos(f.(x-mu)) + 1] G(x; mu, Sigma)     (Sec. 4.1, Eq. 5),
 *     with G the Gaussian of Sec. 3.1 (Eq. 1) and Sigma = R S S^T R^T;
 *   - the 2D image field  C(x) = sum_i c_i W'_i(x)   (Eq. 4 with G' replaced by W', Sec. 4.3);
 *   - the 3D splat: EWA projection Sigma' = [J W Sigma W^T J^T]_{2x2} (Sec. 3.1), the frequency
 *     carried by the same ray-space map (Sec. 4.1), and front-to-back alpha blending of W'
 *     (Eq. 3 with G' replaced by W', Sec. 4.1);
 *   - the analytic gradient of a scalar loss L = sum_x g(x).C(x) with respect to every
 *     primitive parameter (the paper states that explicit gradients exist, Sec. 1).
 * Values are computed in IEEE binary64, by a double loop over every pixel and every primitive.
 *
 * Readings of the paper (where it is silent or inconsistent):
 *   - frequency f is given in cycles per pixel (2D) or cycles per world unit (3D), so the cosine
 *     argument is 2 pi f.d; an extra phase phi is added inside the cosine (phi = 0 is the paper);
 *   - 2D primitives carry no separate opacity (alpha folded into the colour, as in GaussianImage);
 *   - pixel (u, v) is sampled at (u + 0.5, v + 0.5);
 *   - the projected frequency is the phase gradient on the fronto-parallel plane through the
 *     primitive's centre: f' = (fc_x tz / fx, fc_y tz / fy), fc = W f (camera frame);
 *   - 3D: dilation 0.3 px^2, alpha clamped at alpha_max, skipped below alpha_min, blending stops
 *     before a primitive that would take the transmittance below T_min; depth order by camera z.
 *
 * Decisions that floating point turns into integers (is a pixel inside a primitive's 3-sigma
 * footprint, which tiles a primitive covers, the depth order) are taken in binary32 by the
 * "footprint rule" below, so that they are the same decisions the kernels take.  This file is
 * compiled with -ffp-contract=off: every binary32 expression is a sequence of single IEEE
 * operations in source order, and a fused multiply-add occurs only where fmaf is written.
 * The alpha and transmittance thresholds depend on exp and cos and cannot be reproduced bit for
 * bit; pixels where one of them is within a small margin of its threshold are reported as
 * ambiguous.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TILE 16
#define EXT_MARGIN 1.0009765625f /* 1 + 2^-10: footprint half-extent safety factor */
#define INV_TWO_PI_F 0.15915494309189535f /* 1 / (2 pi) rounded to binary32: phase in cycles */
#define DAMP_EXP2_F 28.47765864997501f   /* 2 pi^2 log2(e) rounded to binary32: kappa = 2^-(this fn^2 / c) */

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------------ */
/* binary32 footprint rule                                                                     */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    float mx, my;          /* centre in pixels */
    float l11, l21, l22;   /* lower Cholesky factor of the inverse covariance */
    float ex, ey;          /* half extents of the cutoff ellipse, with margin */
    float depth;           /* camera z (3D), 0 (2D) */
    int u0, v0, u1, v1;    /* covered pixel range (inclusive); empty if u0 > u1 */
    int valid;
    /* 3D only: the record's binary32 projected frequency (cycles/px) under each frequency map
     * (index 0: phase gradient on the fronto-parallel plane, 1: literal J W f, 2: integrated along
     * the viewing ray), its phase in cycles, the opacity, and for map 2 the exponent kx of the
     * damping of the oscillation, kappa = 2^kx.  They take part in no integer decision of the rule
     * itself; the threshold decisions of the blend are evaluated from them (see alpha_decision). */
    float fp[3][2], phc, op, kx;
} fp32_footprint;

static int finite4(float a, float b, float c, float d) { return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d); }

static void footprint_pixrect(fp32_footprint* k, int W, int H) {
    float xlo = (k->mx - k->ex) - 0.5f;
    float xhi = (k->mx + k->ex) - 0.5f;
    float ylo = (k->my - k->ey) - 0.5f;
    float yhi = (k->my + k->ey) - 0.5f;
    xlo = fminf(fmaxf(xlo, -1.0f), (float)W);
    xhi = fminf(fmaxf(xhi, -1.0f), (float)W);
    ylo = fminf(fmaxf(ylo, -1.0f), (float)H);
    yhi = fminf(fmaxf(yhi, -1.0f), (float)H);
    int u0 = (int)ceilf(xlo), u1 = (int)floorf(xhi);
    int v0 = (int)ceilf(ylo), v1 = (int)floorf(yhi);
    if (u0 < 0) u0 = 0;
    if (v0 < 0) v0 = 0;
    if (u1 > W - 1) u1 = W - 1;
    if (v1 > H - 1) v1 = H - 1;
    k->u0 = u0; k->u1 = u1; k->v0 = v0; k->v1 = v1;
    if (u0 > u1 || v0 > v1) { k->u0 = 1; k->u1 = 0; k->v0 = 1; k->v1 = 0; }
}

/* cos and sin of the 2D rotation angle for the footprint rule, as a fixed sequence of IEEE
 * operations (no library transcendental, so that any two IEEE implementations of the rule return
 * the same bits).  The angle is the record's binary32 value.
 * |th| <= 2^16: binary32 arithmetic with fused multiply-adds written as fmaf.  Cody and Waite's
 * reduction: k = nearest integer to th * (2/pi rounded), r = th - k pi/2 with pi/2 split into three
 * binary32 parts P1 + P2 + P3 (within 1e-23 of pi/2).  th - k P1 is exact in one fmaf: both are
 * multiples of 2^-23 (of 2^-24 when |th| < 1, where |k| <= 1) and their difference is below 1.
 * Then the Taylor series of sin r through r^11 and of cos r through r^10 (|r| <= pi/4 + 0.01:
 * truncation below 2e-10), in Horner form in z = r^2; the quadrant k mod 4 picks the signs and the
 * swap.  Each result is within one binary32 ulp of the correctly rounded cosine or sine.
 * 2^16 < |th| <= 1e15: the same steps in binary64 (pi/2 in parts of 33, 33 and 53 significant
 * bits, so k times the first two is exact for |k| < 2^20; Taylor series through r^17 and r^18),
 * rounded once to binary32: the correctly rounded cosine and sine up to |th| = 2^20 pi/2.
 * |th| > 1e15 (or not finite) gives NaN, which makes the primitive invalid. */
static void rule_cos_sin_wide(double th, float* c, float* s) {
    const double k = nearbyint(th * 0x1.45f306dc9c883p-1);
    const double r = ((th - k * 0x1.921fb544p+0) - k * 0x1.0b4611a6p-34) - k * 0x1.3198a2e037073p-69;
    const double z = r * r;
    double ps = 0x1.952c77030ad4ap-49;           /*  1/17! */
    ps = ps * z - 0x1.ae7f3e733b81fp-41;         /* -1/15! */
    ps = ps * z + 0x1.6124613a86d09p-33;         /*  1/13! */
    ps = ps * z - 0x1.ae64567f544e4p-26;         /* -1/11! */
    ps = ps * z + 0x1.71de3a556c734p-19;         /*  1/9!  */
    ps = ps * z - 0x1.a01a01a01a01ap-13;         /* -1/7!  */
    ps = ps * z + 0x1.1111111111111p-7;          /*  1/5!  */
    ps = ps * z - 0x1.5555555555555p-3;          /* -1/3!  */
    const double sr = r + (r * z) * ps;
    double pc = -0x1.6827863b97d97p-53;          /* -1/18! */
    pc = pc * z + 0x1.ae7f3e733b81fp-45;         /*  1/16! */
    pc = pc * z - 0x1.93974a8c07c9dp-37;         /* -1/14! */
    pc = pc * z + 0x1.1eed8eff8d898p-29;         /*  1/12! */
    pc = pc * z - 0x1.27e4fb7789f5cp-22;         /* -1/10! */
    pc = pc * z + 0x1.a01a01a01a01ap-16;         /*  1/8!  */
    pc = pc * z - 0x1.6c16c16c16c17p-10;         /* -1/6!  */
    pc = pc * z + 0x1.5555555555555p-5;          /*  1/4!  */
    pc = pc * z - 0.5;                           /* -1/2!  */
    const double cr = 1.0 + z * pc;
    switch ((int)((long long)k & 3)) {
        case 0: *c = (float)cr; *s = (float)sr; break;
        case 1: *c = (float)(-sr); *s = (float)cr; break;
        case 2: *c = (float)(-cr); *s = (float)(-sr); break;
        default: *c = (float)sr; *s = (float)(-cr); break;
    }
}

static void rule_cos_sin(float th, float* c, float* s) {
    if (!(fabsf(th) <= 0x1p16f)) {
        if (!(fabs((double)th) <= 1e15)) { *c = *s = (float)NAN; return; }
        rule_cos_sin_wide((double)th, c, s);
        return;
    }
    const float k = rintf(th * 0x1.45f306p-1f);  /* th 2/pi */
    float r = fmaf(-k, 0x1.921fb6p+0f, th);      /* - k P1, exact */
    r = fmaf(-k, -0x1.777a5cp-25f, r);           /* - k P2 */
    r = fmaf(-k, -0x1.ee59dap-50f, r);           /* - k P3 */
    const float z = r * r;
    float ps = -0x1.ae6456p-26f;                 /* -1/11! */
    ps = fmaf(ps, z, 0x1.71de3ap-19f);           /*  1/9!  */
    ps = fmaf(ps, z, -0x1.a01a02p-13f);          /* -1/7!  */
    ps = fmaf(ps, z, 0x1.111112p-7f);            /*  1/5!  */
    ps = fmaf(ps, z, -0x1.555556p-3f);           /* -1/3!  */
    const float sr = fmaf(r * z, ps, r);
    float pc = -0x1.27e4fcp-22f;                 /* -1/10! */
    pc = fmaf(pc, z, 0x1.a01a02p-16f);           /*  1/8!  */
    pc = fmaf(pc, z, -0x1.6c16c2p-10f);          /* -1/6!  */
    pc = fmaf(pc, z, 0x1.555556p-5f);            /*  1/4!  */
    pc = fmaf(pc, z, -0.5f);                     /* -1/2!  */
    const float cr = fmaf(z, pc, 1.0f);
    switch ((int)k & 3) {
        case 0: *c = cr; *s = sr; break;
        case 1: *c = -sr; *s = cr; break;
        case 2: *c = -cr; *s = -sr; break;
        default: *c = sr; *s = -cr; break;
    }
}

/* exported for its pin: out[n,2] = the rule's (cos, sin) of th[n] */
int wo_rule_cos_sin(const float* th, int64_t n, float* out) {
    for (int64_t i = 0; i < n; ++i) rule_cos_sin(th[i], &out[2 * i], &out[2 * i + 1]);
    return 0;
}

/* 2D record: mu(2) s(2) theta f(2) phi c(3) */
static void footprint2d(const float* p, float cutoff, int W, int H, fp32_footprint* k) {
    float sx = p[2], sy = p[3];
    float c, s;
    rule_cos_sin(p[4], &c, &s);
    float sx2 = sx * sx, sy2 = sy * sy;
    float ix = 1.0f / sx2, iy = 1.0f / sy2;
    float cc = c * c, ss = s * s, cs = c * s;
    float A = cc * ix + ss * iy;
    float B = cs * (ix - iy);
    float l11 = sqrtf(A);
    float l21 = B / l11;
    float l22 = 1.0f / ((sx * sy) * l11);
    float vxx = cc * sx2 + ss * sy2;
    float vyy = ss * sx2 + cc * sy2;
    k->mx = p[0];
    k->my = p[1];
    k->l11 = l11; k->l21 = l21; k->l22 = l22;
    k->ex = (cutoff * sqrtf(vxx)) * EXT_MARGIN;
    k->ey = (cutoff * sqrtf(vyy)) * EXT_MARGIN;
    k->depth = 0.0f;
    k->valid = finite4(k->mx, k->my, l11, l21) && finite4(l22, k->ex, k->ey, 1.0f) && sx > 0.0f && sy > 0.0f &&
               l11 > 0.0f && l22 > 0.0f;
    if (k->valid) footprint_pixrect(k, W, H);
    else { k->u0 = 1; k->u1 = 0; k->v0 = 1; k->v1 = 0; }
}

/* 2D Cholesky record (GaussianImage's second construction, Sec. 5.1): mu(2) l1 l2 l3 f(2) phi c(3),
 * Sigma = L L^T with L = [[l1, 0], [l2, l3]], so Sigma = [[l1^2, l1 l2], [l1 l2, l2^2 + l3^2]] and
 * Sigma^-1 = [[u, -l1 l2], [-l1 l2, l1^2]] / (l1 l3)^2 with u = l2^2 + l3^2.  Its lower Cholesky
 * factor: l11 = sqrt(u) / |l1 l3|, l21 = -l1 l2 / (|l1 l3| sqrt(u)), l22 = 1 / sqrt(u). */
static void footprint2d_chol(const float* p, float cutoff, int W, int H, fp32_footprint* k) {
    float a = p[2], b = p[3], c = p[4];
    float u = b * b + c * c;
    float su = sqrtf(u);
    float aac = fabsf(a * c);
    float l11 = su / aac;
    float l21 = -(a * b) / (aac * su);
    float l22 = 1.0f / su;
    float vxx = a * a;
    k->mx = p[0];
    k->my = p[1];
    k->l11 = l11; k->l21 = l21; k->l22 = l22;
    k->ex = (cutoff * sqrtf(vxx)) * EXT_MARGIN;
    k->ey = (cutoff * su) * EXT_MARGIN;
    k->depth = 0.0f;
    k->valid = finite4(k->mx, k->my, l11, l21) && finite4(l22, k->ex, k->ey, 1.0f) && aac > 0.0f && l11 > 0.0f &&
               l22 > 0.0f;
    if (k->valid) footprint_pixrect(k, W, H);
    else { k->u0 = 1; k->u1 = 0; k->v0 = 1; k->v1 = 0; }
}

/* Record kinds of the functions below: KIND_2D_RS = 2 (mu s theta f phi c), KIND_3D = 3,
 * KIND_2D_CHOL = 4 (mu l1 l2 l3 f phi c). */
#define KIND_2D_RS 2
#define KIND_3D 3
#define KIND_2D_CHOL 4
#define KIND_3D_SH 5 /* 3D record followed by spherical-harmonic coefficients: 68 floats */
#define P3D_SH 68

static void footprint_of(int kind, const float* params, int64_t i, const float* cam, float cutoff, float dil, int W,
                         int H, fp32_footprint* k);

/* 3D record: mu(3) s(3) q(4: w,x,y,z) f(3) phi opacity c(3); camera: V[12] fx fy cx cy near */
static void footprint3d(const float* p, const float* cam, float cutoff, float dil, int W, int H, fp32_footprint* k) {
    const float* V = cam;
    float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15], near_z = cam[16];
    float tx = ((V[0] * p[0] + V[1] * p[1]) + V[2] * p[2]) + V[3];
    float ty = ((V[4] * p[0] + V[5] * p[1]) + V[6] * p[2]) + V[7];
    float tz = ((V[8] * p[0] + V[9] * p[1]) + V[10] * p[2]) + V[11];
    k->u0 = 1; k->u1 = 0; k->v0 = 1; k->v1 = 0;
    k->valid = 0;
    if (!(tz > near_z) || !isfinite(tz) || !isfinite(tx) || !isfinite(ty)) return;
    float qw = p[6], qx = p[7], qy = p[8], qz = p[9];
    float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    float r = sqrtf(n2);
    qw = qw / r; qx = qx / r; qy = qy / r; qz = qz / r;
    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz);        R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);        R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);        R[7] = 2.0f * (yz + wx);        R[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i * 3 + j] = R[i * 3 + j] * p[3 + j];
    float Q[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Q[i * 3 + j] = (V[i * 4 + 0] * M[0 * 3 + j] + V[i * 4 + 1] * M[1 * 3 + j]) + V[i * 4 + 2] * M[2 * 3 + j];
    float limx = 1.3f * ((0.5f * (float)W) / fx);
    float limy = 1.3f * ((0.5f * (float)H) / fy);
    float txz = fminf(limx, fmaxf(-limx, tx / tz));
    float tyz = fminf(limy, fmaxf(-limy, ty / tz));
    float j00 = fx / tz, j02 = -((fx * txz) / tz);
    float j11 = fy / tz, j12 = -((fy * tyz) / tz);
    float P0[3], P1[3];
    for (int j = 0; j < 3; ++j) {
        P0[j] = j00 * Q[0 * 3 + j] + j02 * Q[2 * 3 + j];
        P1[j] = j11 * Q[1 * 3 + j] + j12 * Q[2 * 3 + j];
    }
    float n0 = (P0[0] * P0[0] + P0[1] * P0[1]) + P0[2] * P0[2];
    float n1 = (P1[0] * P1[0] + P1[1] * P1[1]) + P1[2] * P1[2];
    float s01 = (P0[0] * P1[0] + P0[1] * P1[1]) + P0[2] * P1[2];
    float c0 = P0[1] * P1[2] - P0[2] * P1[1];
    float c1 = P0[2] * P1[0] - P0[0] * P1[2];
    float c2 = P0[0] * P1[1] - P0[1] * P1[0];
    float S00 = n0 + dil, S11 = n1 + dil;
    float D = (((c0 * c0 + c1 * c1) + c2 * c2) + dil * (n0 + n1)) + dil * dil;
    float l22 = 1.0f / sqrtf(S11);
    float l11 = sqrtf(S11 / D);
    float l21 = -(s01 / sqrtf(S11 * D));
    k->mx = ((fx * tx) / tz) + cx;
    k->my = ((fy * ty) / tz) + cy;
    k->l11 = l11; k->l21 = l21; k->l22 = l22;
    k->ex = (cutoff * sqrtf(S00)) * EXT_MARGIN;
    k->ey = (cutoff * sqrtf(S11)) * EXT_MARGIN;
    k->depth = tz;
    {
        float fcx = (V[0] * p[10] + V[1] * p[11]) + V[2] * p[12];
        float fcy = (V[4] * p[10] + V[5] * p[11]) + V[6] * p[12];
        float fcz = (V[8] * p[10] + V[9] * p[11]) + V[10] * p[12];
        k->fp[0][0] = fcx * tz / fx;
        k->fp[0][1] = fcy * tz / fy;
        k->fp[1][0] = j00 * fcx + j02 * fcz;
        k->fp[1][1] = j11 * fcy + j12 * fcz;
        k->phc = p[13] * INV_TWO_PI_F;
        k->op = p[14];
        /* map 2 (Sec. 4.1, the integral along z): with n = (txz, tyz, 1) the viewing direction of
         * the affine ray space (J n = 0) and A = V R the camera-frame principal axes,
         * m = A^T n, w = S^-2 m, c = n^T Sigma_c^-1 n = m . w, b = Sigma_c^-1 n = A w, fn = fc . n;
         * f' = P0^T (fc - (fn / c) b) with P0^T v = (v_x tz / fx, v_y tz / fy), and
         * kappa = exp(-2 pi^2 fn^2 / c) = 2^kx.  binary32, in this order of operations. */
        float A[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                A[i * 3 + j] = (V[i * 4 + 0] * R[0 * 3 + j] + V[i * 4 + 1] * R[1 * 3 + j]) + V[i * 4 + 2] * R[2 * 3 + j];
        float m[3], w[3];
        for (int j = 0; j < 3; ++j) m[j] = (A[0 * 3 + j] * txz + A[1 * 3 + j] * tyz) + A[2 * 3 + j];
        for (int j = 0; j < 3; ++j) w[j] = m[j] / (p[3 + j] * p[3 + j]);
        float cq = (m[0] * w[0] + m[1] * w[1]) + m[2] * w[2];
        float bx = (A[0] * w[0] + A[1] * w[1]) + A[2] * w[2];
        float by = (A[3] * w[0] + A[4] * w[1]) + A[5] * w[2];
        float fn = (fcx * txz + fcy * tyz) + fcz;
        float rr = fn / cq;
        k->fp[2][0] = ((fcx - rr * bx) * tz) / fx;
        k->fp[2][1] = ((fcy - rr * by) * tz) / fy;
        k->kx = -((DAMP_EXP2_F * fn) * rr);
    }
    k->valid = finite4(k->mx, k->my, l11, l21) && finite4(l22, k->ex, k->ey, D) && D > 0.0f && S11 > 0.0f &&
               l11 > 0.0f && l22 > 0.0f;
    if (k->valid) footprint_pixrect(k, W, H);
    else { k->u0 = 1; k->u1 = 0; k->v0 = 1; k->v1 = 0; }
}

/* binary32 squared Mahalanobis distance of pixel (u, v) from the footprint centre */
static void footprint_of(int kind, const float* params, int64_t i, const float* cam, float cutoff, float dil, int W,
                         int H, fp32_footprint* k) {
    if (kind == KIND_2D_RS) footprint2d(params + i * 16, cutoff, W, H, k);
    else if (kind == KIND_2D_CHOL) footprint2d_chol(params + i * 16, cutoff, W, H, k);
    else footprint3d(params + i * (kind == KIND_3D_SH ? P3D_SH : 20), cam, cutoff, dil, W, H, k);
}

static float q32(const fp32_footprint* k, int u, int v) {
    float dx = ((float)u + 0.5f) - k->mx;
    float dy = ((float)v + 0.5f) - k->my;
    float a = fmaf(k->l11, dx, k->l21 * dy);
    float b = k->l22 * dy;
    return fmaf(a, a, b * b);
}

/* Does the cutoff ellipse, widened by a 1 % margin on cutoff^2, reach the rectangle spanned by the
 * pixel centres of columns x0..x1 and rows y0..y1?  With q = A dx^2 + 2 B dx dy + C dy^2
 * (A = l11^2, B = l11 l21, C = l21^2 + l22^2) the minimum over the rectangle is 0 when the centre
 * lies inside, else the least of the four edge minima: on an edge of fixed dx the minimiser is
 * dy = -(B/C) dx clamped to the edge, on an edge of fixed dy it is dx = -(B/A) dy clamped.  Every
 * pixel centre that passes the binary32 cutoff test lies in a rectangle this returns 1 for (the
 * margin exceeds the rounding of q32). */
typedef struct { float rBA, rBC; } edge_ratios;

static edge_ratios footprint_ratios(const fp32_footprint* k) {
    float A = k->l11 * k->l11, B = k->l11 * k->l21, C = k->l21 * k->l21 + k->l22 * k->l22;
    edge_ratios r = {-(B / A), -(B / C)};
    return r;
}

static int rect_touched(const fp32_footprint* k, edge_ratios rr, int x0, int x1, int y0, int y1, float lim) {
    float dx0 = ((float)x0 + 0.5f) - k->mx, dx1 = ((float)x1 + 0.5f) - k->mx;
    float dy0 = ((float)y0 + 0.5f) - k->my, dy1 = ((float)y1 + 0.5f) - k->my;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 1;
    float best = 0.0f;
    for (int e = 0; e < 4; ++e) {
        float dx, dy;
        if (e < 2) {
            dx = e == 0 ? dx0 : dx1;
            dy = fminf(fmaxf(rr.rBC * dx, dy0), dy1);
        } else {
            dy = e == 2 ? dy0 : dy1;
            dx = fminf(fmaxf(rr.rBA * dy, dx0), dx1);
        }
        float a = k->l11 * dx + k->l21 * dy;
        float b = k->l22 * dy;
        float q = a * a + b * b;
        best = e == 0 ? q : fminf(best, q);
    }
    return best <= lim;
}

static float touch_limit(float cutoff) { return (cutoff * cutoff) * 1.01f; }

/* number of tiles of the covered pixel range that the cutoff ellipse touches */
static int64_t touched_tiles(const fp32_footprint* k, float lim, uint32_t* tiles, int tiles_x) {
    if (!k->valid || k->u0 > k->u1) return 0;
    edge_ratios rr = footprint_ratios(k);
    int64_t n = 0;
    for (int ty = k->v0 / TILE; ty <= k->v1 / TILE; ++ty)
        for (int tx = k->u0 / TILE; tx <= k->u1 / TILE; ++tx) {
            int x0 = tx * TILE > k->u0 ? tx * TILE : k->u0, x1 = tx * TILE + TILE - 1 < k->u1 ? tx * TILE + TILE - 1 : k->u1;
            int y0 = ty * TILE > k->v0 ? ty * TILE : k->v0, y1 = ty * TILE + TILE - 1 < k->v1 ? ty * TILE + TILE - 1 : k->v1;
            if (!rect_touched(k, rr, x0, x1, y0, y1, lim)) continue;
            if (tiles) tiles[n] = (uint32_t)(ty * tiles_x + tx);
            ++n;
        }
    return n;
}

static uint32_t f32_bits(float x) { uint32_t b; memcpy(&b, &x, 4); return b; }

/* Exported view of the footprint rule: rec[N,8] = mx,my,l11,l21,l22,ex,ey,depth; rect[N,4] = u0,v0,u1,v1;
 * valid[N].  kind = KIND_2D_RS, KIND_3D or KIND_2D_CHOL; cam and dil are ignored in 2D. */
int wo_footprints(int kind, const float* params, int64_t N, const float* cam, int H, int W, float cutoff, float dil,
                  float* rec, int32_t* rect, int32_t* valid) {
    for (int64_t i = 0; i < N; ++i) {
        fp32_footprint k;
        footprint_of(kind, params, i, cam, cutoff, dil, W, H, &k);
        if (rec) {
            float* r = rec + i * 8;
            r[0] = k.mx; r[1] = k.my; r[2] = k.l11; r[3] = k.l21; r[4] = k.l22; r[5] = k.ex; r[6] = k.ey; r[7] = k.depth;
        }
        if (rect) { rect[i * 4 + 0] = k.u0; rect[i * 4 + 1] = k.v0; rect[i * 4 + 2] = k.u1; rect[i * 4 + 3] = k.v1; }
        if (valid) valid[i] = k.valid;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* tile lists: every (tile, primitive) pair whose tile meets the primitive's covered pixel     */
/* range, ordered by tile, then depth (3D), then primitive index                               */
/* ------------------------------------------------------------------------------------------ */

typedef struct { uint32_t tile, depth, prim; } tile_entry;

static int cmp_entry(const void* a, const void* b) {
    const tile_entry* x = (const tile_entry*)a;
    const tile_entry* y = (const tile_entry*)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    if (x->prim != y->prim) return x->prim < y->prim ? -1 : 1;
    return 0;
}

static fp32_footprint* all_footprints(int kind, const float* params, int64_t N, const float* cam, int H, int W,
                                      float cutoff, float dil) {
    fp32_footprint* k = (fp32_footprint*)malloc(sizeof(fp32_footprint) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) footprint_of(kind, params, i, cam, cutoff, dil, W, H, &k[i]);
    return k;
}

/* Returns the number of entries (also when it exceeds cap; then only cap are written). */
int64_t wo_tile_lists(int kind, const float* params, int64_t N, const float* cam, int H, int W, float cutoff, float dil,
                      uint32_t* tile_out, uint32_t* prim_out, int64_t cap) {
    const int dims = kind == KIND_3D || kind == KIND_3D_SH ? 3 : 2;
    fp32_footprint* k = all_footprints(kind, params, N, cam, H, W, cutoff, dil);
    int tiles_x = (W + TILE - 1) / TILE;
    float lim = touch_limit(cutoff);
    int64_t total = 0;
    for (int64_t i = 0; i < N; ++i) total += touched_tiles(&k[i], lim, NULL, tiles_x);
    tile_entry* e = (tile_entry*)malloc(sizeof(tile_entry) * (size_t)(total > 0 ? total : 1));
    uint32_t* tl = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)((W + TILE - 1) / TILE) * (size_t)((H + TILE - 1) / TILE));
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t m = touched_tiles(&k[i], lim, tl, tiles_x);
        for (int64_t j = 0; j < m; ++j) {
            e[n].tile = tl[j];
            e[n].depth = dims == 3 ? f32_bits(k[i].depth) : 0u;
            e[n].prim = (uint32_t)i;
            ++n;
        }
    }
    free(tl);
    qsort(e, (size_t)n, sizeof(tile_entry), cmp_entry);
    for (int64_t j = 0; j < n && j < cap; ++j) {
        tile_out[j] = e[j].tile;
        prim_out[j] = e[j].prim;
    }
    free(e);
    free(k);
    return total;
}

/* ------------------------------------------------------------------------------------------ */
/* small dense helpers (binary64)                                                              */
/* ------------------------------------------------------------------------------------------ */

static void mat2_inv(const double a[4], double out[4]) {
    double det = a[0] * a[3] - a[1] * a[2];
    out[0] = a[3] / det;
    out[1] = -a[1] / det;
    out[2] = -a[2] / det;
    out[3] = a[0] / det;
}

/* C = A (m x k) * B (k x n) */
static void matmul(const double* A, const double* B, double* C, int m, int k, int n) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * n + j];
            C[i * n + j] = s;
        }
}

static void transpose(const double* A, double* At, int m, int n) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) At[j * m + i] = A[i * n + j];
}

/* ------------------------------------------------------------------------------------------ */
/* the projected (image-plane) wavelet of one primitive, binary64                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int valid;
    double mu[2];    /* mu' (pixels) */
    double K[4];     /* inverse of Sigma' (row-major 2x2) */
    double f[2];     /* f' (cycles per pixel) */
    double kap;      /* damping of the oscillation (1 except under frequency map 2) */
    double phi;      /* phase (radians) */
    double o;        /* opacity (3D) */
    double c[3];     /* colour */
    /* 3D chain-rule intermediates */
    double t[3], R[9], M[9], V[9], Sc[9], J[6], fc[3], qn[4], qnorm, s[3];
    int unclamped_x, unclamped_y;
    int fmode;       /* frequency projection mode of project3d */
    double lim[2];   /* view-angle clamp of the Jacobian (|tx / tz|, |ty / tz|) */
    int sh;          /* SH degree of the colour (0: the record's RGB) */
    double dir[3], dist, raw[3];  /* SH colour: unit direction camera -> centre, its length, unclamped colour */
} proj;

/* cov2d = 0: record mu s(2) theta ..., Sigma = R diag(sx^2, sy^2) R^T (Sec. 3.1, Sigma = R S S^T R^T);
 * cov2d = 1: record mu l1 l2 l3 ..., Sigma = L L^T with L = [[l1, 0], [l2, l3]] (Cholesky, Sec. 5.1). */
static void project2d(const float* p, int cov2d, proj* w) {
    double Sig[4];
    memset(w, 0, sizeof(*w));
    if (cov2d) {
        double a = p[2], b = p[3], c = p[4];
        Sig[0] = a * a; Sig[1] = a * b; Sig[2] = a * b; Sig[3] = b * b + c * c;
        w->valid = a != 0.0 && c != 0.0 && isfinite(a) && isfinite(b) && isfinite(c);
    } else {
        double sx = p[2], sy = p[3], th = p[4];
        double c = cos(th), s = sin(th);
        Sig[0] = c * c * sx * sx + s * s * sy * sy;
        Sig[1] = c * s * (sx * sx - sy * sy);
        Sig[2] = Sig[1];
        Sig[3] = s * s * sx * sx + c * c * sy * sy;
        w->valid = sx > 0 && sy > 0 && isfinite(sx) && isfinite(sy);
    }
    mat2_inv(Sig, w->K);
    w->mu[0] = p[0]; w->mu[1] = p[1];
    w->f[0] = p[5]; w->f[1] = p[6];
    w->kap = 1.0;
    w->phi = p[7];
    w->o = 1.0;
    w->c[0] = p[8]; w->c[1] = p[9]; w->c[2] = p[10];
    w->s[0] = p[2]; w->s[1] = p[3];
}

static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* fmode 0: f' = (fc_x tz / fx, fc_y tz / fy), the phase gradient on the fronto-parallel plane through
 * the centre (reading of Sec. 4.1); fmode 1: f' = J fc, the frequency put through the same W and J
 * as the covariance, read literally (Sec. 4.1). */
/* Real spherical harmonics up to degree 3 at the unit vector d = (x, y, z), Condon-Shortley phase,
 * ordered l = 0..3 and m = -l..l within a degree (the view-dependent colour of 3DGS that the paper's
 * 3D primitives carry, Sec. 3.1), and their partial derivatives with respect to x, y, z (the
 * polynomials differentiated as functions on R^3). */
static void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
    const double x = d[0], y = d[1], z = d[2];
    const double k0 = 0.5 * sqrt(1.0 / PI), k1 = sqrt(3.0 / (4.0 * PI));
    const double k2a = 0.5 * sqrt(15.0 / PI), k2b = 0.25 * sqrt(5.0 / PI), k2c = 0.25 * sqrt(15.0 / PI);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI)), k3b = 0.5 * sqrt(105.0 / PI);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI)), k3d = 0.25 * sqrt(7.0 / PI), k3e = 0.25 * sqrt(105.0 / PI);
    const double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k0;
    Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
    Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (2 * zz - xx - yy); Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    Y[9] = -k3a * y * (3 * xx - yy); Y[10] = k3b * x * y * z; Y[11] = -k3c * y * (4 * zz - xx - yy);
    Y[12] = k3d * z * (2 * zz - 3 * xx - 3 * yy); Y[13] = -k3c * x * (4 * zz - xx - yy); Y[14] = k3e * z * (xx - yy);
    Y[15] = -k3a * x * (xx - 3 * yy);
    const double g[16][3] = {{0, 0, 0},
                             {0, -k1, 0}, {0, 0, k1}, {-k1, 0, 0},
                             {k2a * y, k2a * x, 0}, {0, -k2a * z, -k2a * y}, {-2 * k2b * x, -2 * k2b * y, 4 * k2b * z},
                             {-k2a * z, 0, -k2a * x}, {2 * k2c * x, -2 * k2c * y, 0},
                             {-6 * k3a * x * y, -3 * k3a * (xx - yy), 0},
                             {k3b * y * z, k3b * x * z, k3b * x * y},
                             {2 * k3c * x * y, -k3c * (4 * zz - xx - 3 * yy), -8 * k3c * y * z},
                             {-6 * k3d * x * z, -6 * k3d * y * z, k3d * (6 * zz - 3 * xx - 3 * yy)},
                             {-k3c * (4 * zz - 3 * xx - yy), 2 * k3c * x * y, -8 * k3c * x * z},
                             {2 * k3e * x * z, -2 * k3e * y * z, k3e * (xx - yy)},
                             {-3 * k3a * (xx - yy), 6 * k3a * x * y, 0}};
    if (dY) memcpy(dY, g, sizeof(g));
}

/* exported for tests: Y[n,16] at n unit vectors */
int wo_sh_basis(const double* dirs, int64_t n, double* Y) {
    for (int64_t i = 0; i < n; ++i) sh_basis(dirs + 3 * i, Y + 16 * i, NULL);
    return 0;
}

/* view-dependent colour of an SH record: the coefficient of basis k for channel ch */
static double sh_coef(const float* p, int k, int ch) { return k == 0 ? (double)p[15 + ch] : (double)p[20 + 3 * (k - 1) + ch]; }

/* Frequency map 2, the oscillation integrated along the viewing ray (Sec. 4.1 integrates the 3D
 * wavelet over z).  In the affine ray space of the EWA projection a camera-frame offset from the
 * centre is y - t = P0 a + n z: a is the image-plane offset in pixels, n = (txz, tyz, 1) the viewing
 * direction (J n = 0, with the Jacobian's clamped view angles) and P0 the right inverse of J with
 * P0 a = (a_x tz / fx, a_y tz / fy, 0).  With Q = B^T Sigma_c^-1 B, B = [P0 | n], completing the
 * square in z turns the integral over z of cos(2 pi fc.(y - t) + phi) G into
 *   kappa cos(2 pi f'.a + phi) G'(a) (times the constant of the Gaussian integral),
 *   f' = P0^T fc - (fc.n) Q_az / Q_zz,   kappa = exp(-2 pi^2 (fc.n)^2 / Q_zz),
 * where G' is the marginal the covariance projection gives; the constant is dropped as for G' (the
 * opacity carries it).  Q_zz = n^T Sigma_c^-1 n and Q_az = P0^T Sigma_c^-1 n, with Sigma_c = V Sigma V^T.
 * Written over complex numbers so that the complex step gives its exact derivatives (chain3d);
 * real inputs give the value.  out = (f'_x, f'_y, kappa). */
static void quat_to_rot_c(const double complex q[4], double complex R[9]) {
    double complex w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void damped_freq(const double complex t[3], const double complex s[3], const double complex qn[4],
                        const double complex fc[3], const double V[9], double fx, double fy, const double lim[2],
                        double complex out[3]) {
    double complex R[9], M[9], Sig[9], VS[9], Sc[9], adj[9], n[3], b[3];
    quat_to_rot_c(qn, R);
    /* Sigma_c = V R S S^T R^T V^T, the camera-frame covariance of the covariance projection */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i * 3 + j] = R[i * 3 + j] * s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Sig[i * 3 + j] = M[i * 3 + 0] * M[j * 3 + 0] + M[i * 3 + 1] * M[j * 3 + 1] + M[i * 3 + 2] * M[j * 3 + 2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) VS[i * 3 + j] = V[i * 3 + 0] * Sig[0 * 3 + j] + V[i * 3 + 1] * Sig[1 * 3 + j] + V[i * 3 + 2] * Sig[2 * 3 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Sc[i * 3 + j] = VS[i * 3 + 0] * V[j * 3 + 0] + VS[i * 3 + 1] * V[j * 3 + 1] + VS[i * 3 + 2] * V[j * 3 + 2];
    /* b = Sigma_c^-1 n by the adjugate */
    adj[0] = Sc[4] * Sc[8] - Sc[5] * Sc[7]; adj[1] = Sc[2] * Sc[7] - Sc[1] * Sc[8]; adj[2] = Sc[1] * Sc[5] - Sc[2] * Sc[4];
    adj[3] = Sc[5] * Sc[6] - Sc[3] * Sc[8]; adj[4] = Sc[0] * Sc[8] - Sc[2] * Sc[6]; adj[5] = Sc[2] * Sc[3] - Sc[0] * Sc[5];
    adj[6] = Sc[3] * Sc[7] - Sc[4] * Sc[6]; adj[7] = Sc[1] * Sc[6] - Sc[0] * Sc[7]; adj[8] = Sc[0] * Sc[4] - Sc[1] * Sc[3];
    const double complex det = Sc[0] * adj[0] + Sc[1] * adj[3] + Sc[2] * adj[6];
    n[0] = t[0] / t[2];
    n[1] = t[1] / t[2];
    n[2] = 1.0;
    for (int a = 0; a < 2; ++a) {
        if (creal(n[a]) < -lim[a]) n[a] = -lim[a];
        if (creal(n[a]) > lim[a]) n[a] = lim[a];
    }
    for (int i = 0; i < 3; ++i) b[i] = (adj[i * 3 + 0] * n[0] + adj[i * 3 + 1] * n[1] + adj[i * 3 + 2] * n[2]) / det;
    const double complex c = n[0] * b[0] + n[1] * b[1] + n[2] * b[2];  /* Q_zz */
    const double complex fn = fc[0] * n[0] + fc[1] * n[1] + fc[2] * n[2];
    const double complex r = fn / c;
    for (int a = 0; a < 2; ++a) out[a] = (fc[a] - r * b[a]) * t[2] / (a == 0 ? fx : fy);
    out[2] = cexp(-2.0 * PI * PI * fn * r);
}

/* the map's value at the projection's inputs (real) and, when d is not NULL, its derivatives
 * d[k][0..2] by input k of (t(3), s(3), qn(4), fc(3)), each from one complex step of 1e-30 */
static void damped_freq_eval(const proj* w, double fx, double fy, double val[3], double d[13][3]) {
    double complex in[13], out[3];
    for (int j = 0; j < 3; ++j) { in[j] = w->t[j]; in[3 + j] = w->s[j]; in[10 + j] = w->fc[j]; }
    for (int m = 0; m < 4; ++m) in[6 + m] = w->qn[m];
    damped_freq(in, in + 3, in + 6, in + 10, w->V, fx, fy, w->lim, out);
    for (int a = 0; a < 3; ++a) val[a] = creal(out[a]);
    if (!d) return;
    const double h = 1e-30;
    for (int k = 0; k < 13; ++k) {
        double complex x[13];
        memcpy(x, in, sizeof(x));
        x[k] += h * I;
        damped_freq(x, x + 3, x + 6, x + 10, w->V, fx, fy, w->lim, out);
        for (int a = 0; a < 3; ++a) d[k][a] = cimag(out[a]) / h;
    }
}

static void project3d(const float* p, const float* cam, int H, int W, double dil, int fmode, int valid32, proj* w) {
    memset(w, 0, sizeof(*w));
    w->valid = valid32;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) w->V[i * 3 + j] = cam[i * 4 + j];
    for (int i = 0; i < 3; ++i)
        w->t[i] = w->V[i * 3 + 0] * p[0] + w->V[i * 3 + 1] * p[1] + w->V[i * 3 + 2] * p[2] + (double)cam[i * 4 + 3];
    double tx = w->t[0], ty = w->t[1], tz = w->t[2];
    double qr[4] = {p[6], p[7], p[8], p[9]};
    w->qnorm = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    for (int i = 0; i < 4; ++i) w->qn[i] = qr[i] / w->qnorm;
    quat_to_rot(w->qn, w->R);
    for (int j = 0; j < 3; ++j) w->s[j] = p[3 + j];
    /* Sigma = R S S^T R^T, camera frame Sc = V Sigma V^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) w->M[i * 3 + j] = w->R[i * 3 + j] * w->s[j];
    double Mt[9], Sig[9], Vt[9], tmp[9];
    transpose(w->M, Mt, 3, 3);
    matmul(w->M, Mt, Sig, 3, 3, 3);
    transpose(w->V, Vt, 3, 3);
    matmul(w->V, Sig, tmp, 3, 3, 3);
    matmul(tmp, Vt, w->Sc, 3, 3, 3);
    /* local affine Jacobian of the perspective map, with the usual clamp of the view angle */
    double limx = 1.3 * (0.5 * W / fx), limy = 1.3 * (0.5 * H / fy);
    w->lim[0] = limx;
    w->lim[1] = limy;
    double txz = tx / tz, tyz = ty / tz;
    w->unclamped_x = txz > -limx && txz < limx;
    w->unclamped_y = tyz > -limy && tyz < limy;
    if (txz < -limx) txz = -limx;
    if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy;
    if (tyz > limy) tyz = limy;
    double J[6] = {fx / tz, 0.0, -fx * txz / tz, 0.0, fy / tz, -fy * tyz / tz};
    memcpy(w->J, J, sizeof(J));
    double Jt[6], JS[6], S2[4];
    transpose(J, Jt, 2, 3);
    matmul(J, w->Sc, JS, 2, 3, 3);
    matmul(JS, Jt, S2, 2, 3, 2);
    S2[0] += dil;
    S2[3] += dil;
    mat2_inv(S2, w->K);
    w->mu[0] = fx * tx / tz + cx;
    w->mu[1] = fy * ty / tz + cy;
    for (int i = 0; i < 3; ++i) w->fc[i] = w->V[i * 3 + 0] * p[10] + w->V[i * 3 + 1] * p[11] + w->V[i * 3 + 2] * p[12];
    w->kap = 1.0;
    if (fmode == 2) {
        double val[3];
        damped_freq_eval(w, fx, fy, val, NULL);
        w->f[0] = val[0];
        w->f[1] = val[1];
        w->kap = val[2];
    } else if (fmode) {
        w->f[0] = J[0] * w->fc[0] + J[1] * w->fc[1] + J[2] * w->fc[2];
        w->f[1] = J[3] * w->fc[0] + J[4] * w->fc[1] + J[5] * w->fc[2];
    } else {
        w->f[0] = w->fc[0] * tz / fx;
        w->f[1] = w->fc[1] * tz / fy;
    }
    w->fmode = fmode;
    w->phi = p[13];
    w->o = p[14];
    w->c[0] = p[15]; w->c[1] = p[16]; w->c[2] = p[17];
}

/* SH colour (degree sh >= 1): c = max(0, 1/2 + sum_k Y_k(dir) sh_k), dir the unit vector from the
 * camera centre -V^T t0 to mu (as 3DGS evaluates it) */
static void sh_colour(const float* p, const float* cam, int sh, proj* w) {
    double cpos[3];
    for (int j = 0; j < 3; ++j)
        cpos[j] = -((double)cam[0 * 4 + j] * cam[3] + (double)cam[1 * 4 + j] * cam[7] + (double)cam[2 * 4 + j] * cam[11]);
    double v[3] = {p[0] - cpos[0], p[1] - cpos[1], p[2] - cpos[2]};
    w->dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int j = 0; j < 3; ++j) w->dir[j] = v[j] / w->dist;
    double Y[16];
    sh_basis(w->dir, Y, NULL);
    const int nk = (sh + 1) * (sh + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double r = 0.5;
        for (int k = 0; k < nk; ++k) r += Y[k] * sh_coef(p, k, ch);
        w->raw[ch] = r;
        w->c[ch] = r > 0.0 ? r : 0.0;
    }
    w->sh = sh;
}

/* W'(x) and its pieces at pixel (u, v) */
typedef struct { double d[2], Kd[2], q, G, ca, sa, M, W; } wval;

static void eval_wavelet(const proj* w, int u, int v, wval* e) {
    e->d[0] = (u + 0.5) - w->mu[0];
    e->d[1] = (v + 0.5) - w->mu[1];
    e->Kd[0] = w->K[0] * e->d[0] + w->K[1] * e->d[1];
    e->Kd[1] = w->K[2] * e->d[0] + w->K[3] * e->d[1];
    e->q = e->d[0] * e->Kd[0] + e->d[1] * e->Kd[1];
    e->G = exp(-0.5 * e->q);
    double arg = 2.0 * PI * (w->f[0] * e->d[0] + w->f[1] * e->d[1]) + w->phi;
    e->ca = cos(arg);
    e->sa = sin(arg);
    e->M = 0.5 * (1.0 + w->kap * e->ca);
    e->W = e->M * e->G;
}

/* per-primitive image-plane gradient accumulator: dL/d(mu', K (full 2x2), f', phi, o, c) */
typedef struct { double mu[2], K[4], f[2], phi, o, c[3], kap; } pgrad;

/* add gW * dW'/d(mu', K, f', phi) */
static void accum_wavelet_grad(const proj* w, const wval* e, double gW, pgrad* g) {
    /* W = (1 + kappa cos(arg)) G / 2:  dW/dmu = W K d + pi kappa G sin(arg) f ;
       dW/df = -pi kappa G sin(arg) d ;  dW/dphi = -kappa G sin(arg) / 2 ;  dW/dK_ab = -W d_a d_b / 2 ;
       dW/dkappa = cos(arg) G / 2 */
    const double kGs = w->kap * e->G * e->sa;
    for (int a = 0; a < 2; ++a) {
        g->mu[a] += gW * (e->W * e->Kd[a] + PI * kGs * w->f[a]);
        g->f[a] += gW * (-PI * kGs * e->d[a]);
    }
    g->phi += gW * (-0.5 * kGs);
    g->kap += gW * 0.5 * e->ca * e->G;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) g->K[a * 2 + b] += gW * (-0.5 * e->W * e->d[a] * e->d[b]);
}

/* ------------------------------------------------------------------------------------------ */
/* 2D: summed field                                                                            */
/* ------------------------------------------------------------------------------------------ */

static int pixel_of(const int32_t* pix, int64_t j, int W, int* u, int* v) {
    if (pix) { *u = pix[2 * j]; *v = pix[2 * j + 1]; }
    else { *u = (int)(j % W); *v = (int)(j / W); }
    return 0;
}

/* out[npix,3] (or [H*W,3] when pix is NULL).  truncated: include a primitive at a pixel only if the
 * binary32 footprint rule puts the pixel inside its cutoff ellipse; otherwise every primitive counts. */
int wo_render2d(const float* params, int64_t N, int H, int W, float cutoff, int truncated, const int32_t* pix,
                int64_t npix, int cov2d, double* out) {
    fp32_footprint* k = all_footprints(cov2d ? KIND_2D_CHOL : KIND_2D_RS, params, N, NULL, H, W, cutoff, 0.0f);
    proj* w = (proj*)malloc(sizeof(proj) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) project2d(params + i * 16, cov2d, &w[i]);
    float k2 = cutoff * cutoff;
    int64_t np = pix ? npix : (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < np; ++j) {
        int u, v;
        pixel_of(pix, j, W, &u, &v);
        double C[3] = {0, 0, 0};
        for (int64_t i = 0; i < N; ++i) {
            if (truncated) {
                if (!k[i].valid || !(q32(&k[i], u, v) <= k2)) continue;
            } else if (!w[i].valid) continue;
            wval e;
            eval_wavelet(&w[i], u, v, &e);
            for (int ch = 0; ch < 3; ++ch) C[ch] += w[i].c[ch] * e.W;
        }
        for (int ch = 0; ch < 3; ++ch) out[j * 3 + ch] = C[ch];
    }
    free(w);
    free(k);
    return 0;
}

/* the gradient with respect to the Cholesky record entries (l1, l2, l3): K = Sigma^-1, so for each
 * entry dK = -K dSigma K with dSigma/dl1 = [[2 l1, l2], [l2, 0]], dSigma/dl2 = [[0, l1], [l1, 2 l2]],
 * dSigma/dl3 = [[0, 0], [0, 2 l3]] */
static void chain2d_chol(const float* p, const pgrad* g, double gl[3]) {
    double a = p[2], b = p[3], c = p[4];
    double Sig[4] = {a * a, a * b, a * b, b * b + c * c}, K[4];
    mat2_inv(Sig, K);
    double dS[3][4] = {{2 * a, b, b, 0}, {0, a, a, 2 * b}, {0, 0, 0, 2 * c}};
    for (int j = 0; j < 3; ++j) {
        double t1[4], dK[4];
        matmul(K, dS[j], t1, 2, 2, 2);
        matmul(t1, K, dK, 2, 2, 2);
        gl[j] = 0.0;
        for (int m = 0; m < 4; ++m) gl[j] -= g->K[m] * dK[m];
    }
}

/* chain the image-plane gradient of a 2D primitive to its record: mu(2) s(2) theta f(2) phi c(3)
 * (cov2d = 0) or mu(2) l1 l2 l3 f(2) phi c(3) (cov2d = 1) */
static void chain2d(const float* p, int cov2d, const pgrad* g, double* out) {
    if (cov2d) {
        double gl[3];
        chain2d_chol(p, g, gl);
        memset(out, 0, sizeof(double) * 16);
        out[0] = g->mu[0]; out[1] = g->mu[1];
        out[2] = gl[0]; out[3] = gl[1]; out[4] = gl[2];
        out[5] = g->f[0]; out[6] = g->f[1];
        out[7] = g->phi;
        out[8] = g->c[0]; out[9] = g->c[1]; out[10] = g->c[2];
        return;
    }
    double sx = p[2], sy = p[3], th = p[4];
    double c = cos(th), s = sin(th);
    double R[4] = {c, -s, s, c}, Rt[4] = {c, s, -s, c};
    double dR[4] = {-s, -c, c, -s}, dRt[4] = {-s, c, -c, -s};
    double Dinv[4] = {1.0 / (sx * sx), 0, 0, 1.0 / (sy * sy)};
    double t1[4], t2[4], dK[4];
    /* K = R D^-1 R^T:  dK/dtheta = R' D^-1 R^T + R D^-1 R'^T */
    matmul(dR, Dinv, t1, 2, 2, 2);
    matmul(t1, Rt, t2, 2, 2, 2);
    matmul(R, Dinv, t1, 2, 2, 2);
    matmul(t1, dRt, dK, 2, 2, 2);
    double gth = 0.0;
    for (int a = 0; a < 4; ++a) gth += g->K[a] * (t2[a] + dK[a]);
    double gs[2];
    for (int j = 0; j < 2; ++j) {
        double sj = j == 0 ? sx : sy;
        double Dj[4] = {0, 0, 0, 0};
        Dj[j * 3] = -2.0 / (sj * sj * sj);
        matmul(R, Dj, t1, 2, 2, 2);
        matmul(t1, Rt, t2, 2, 2, 2);
        gs[j] = 0.0;
        for (int a = 0; a < 4; ++a) gs[j] += g->K[a] * t2[a];
    }
    memset(out, 0, sizeof(double) * 16);
    out[0] = g->mu[0]; out[1] = g->mu[1];
    out[2] = gs[0]; out[3] = gs[1];
    out[4] = gth;
    out[5] = g->f[0]; out[6] = g->f[1];
    out[7] = g->phi;
    out[8] = g->c[0]; out[9] = g->c[1]; out[10] = g->c[2];
}

/* grad[N,16] of L = sum_pixels dldimg . C.  When gabs is not NULL it receives, per parameter, the
 * sum over pixels of the absolute value of that pixel's contribution to the gradient: the scale
 * against which the rounding error of a summed gradient is measured. */
int wo_grad2d(const float* params, int64_t N, int H, int W, float cutoff, int truncated, const float* dldimg,
              int cov2d, double* grad, double* gabs) {
    fp32_footprint* k = all_footprints(cov2d ? KIND_2D_CHOL : KIND_2D_RS, params, N, NULL, H, W, cutoff, 0.0f);
    proj* w = (proj*)malloc(sizeof(proj) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) project2d(params + i * 16, cov2d, &w[i]);
    pgrad* acc = (pgrad*)calloc((size_t)(N > 0 ? N : 1), sizeof(pgrad));
    float k2 = cutoff * cutoff;
    /* primitive-major so that each accumulator has one writer */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        if (!w[i].valid) continue;
        if (truncated && !k[i].valid) continue;
        pgrad g;
        memset(&g, 0, sizeof(g));
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                if (truncated && !(q32(&k[i], u, v) <= k2)) continue;
                const float* gp = dldimg + ((int64_t)v * W + u) * 3;
                wval e;
                eval_wavelet(&w[i], u, v, &e);
                double gW = 0.0;
                pgrad one;
                memset(&one, 0, sizeof(one));
                for (int ch = 0; ch < 3; ++ch) {
                    one.c[ch] = gp[ch] * e.W;
                    gW += gp[ch] * w[i].c[ch];
                }
                accum_wavelet_grad(&w[i], &e, gW, &one);
                for (int m = 0; m < 2; ++m) { g.mu[m] += one.mu[m]; g.f[m] += one.f[m]; }
                for (int m = 0; m < 4; ++m) g.K[m] += one.K[m];
                for (int m = 0; m < 3; ++m) g.c[m] += one.c[m];
                g.phi += one.phi;
                if (gabs) {
                    double t[16];
                    chain2d(params + i * 16, cov2d, &one, t);
                    for (int m = 0; m < 16; ++m) gabs[i * 16 + m] += fabs(t[m]);
                }
            }
        acc[i] = g;
    }
    for (int64_t i = 0; i < N; ++i) {
        /* a degenerate primitive (non-positive scale, or dropped by the cutoff rule) contributes
           nothing to the image, so its gradient is zero */
        if (!w[i].valid || (truncated && !k[i].valid)) memset(grad + i * 16, 0, sizeof(double) * 16);
        else chain2d(params + i * 16, cov2d, &acc[i], grad + i * 16);
    }
    free(acc);
    free(w);
    free(k);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* 3D: projection and front-to-back alpha blending                                             */
/* ------------------------------------------------------------------------------------------ */

/* opts[10] = cutoff, alpha_min, alpha_max, T_min, dilation, bg_r, bg_g, bg_b, frequency projection
 * mode (0: phase gradient on the fronto-parallel plane; 1: the literal f' = (J W f)_xy; 2: the
 * oscillation integrated along the viewing ray, with its damping kappa), degree of
 * the spherical-harmonic colour (0: the record's RGB colour; 1..3: SH records of P3D_SH floats) */
typedef struct { float cutoff, amin, amax, Tmin, dil; double bg[3]; int fmode, sh; } blend_opts;

static blend_opts read_opts(const float* o) {
    blend_opts b = {o[0], o[1], o[2], o[3], o[4], {o[5], o[6], o[7]}, (int)o[8], (int)o[9]};
    return b;
}

typedef struct { uint32_t depth, prim; } order_entry;

static int cmp_order(const void* a, const void* b) {
    const order_entry* x = (const order_entry*)a;
    const order_entry* y = (const order_entry*)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return x->prim < y->prim ? -1 : (x->prim > y->prim);
}

typedef struct {
    fp32_footprint* k;
    proj* w;
    uint32_t* order; /* valid primitives, front to back */
    int64_t nvalid;
} scene3;

static int rec3_stride(const blend_opts* o) { return o->sh ? P3D_SH : 20; }

static void scene3_build(const float* params, int64_t N, const float* cam, int H, int W, const blend_opts* o, scene3* s) {
    const int P = rec3_stride(o);
    s->k = all_footprints(o->sh ? KIND_3D_SH : KIND_3D, params, N, cam, H, W, o->cutoff, o->dil);
    s->w = (proj*)malloc(sizeof(proj) * (size_t)(N > 0 ? N : 1));
    order_entry* e = (order_entry*)malloc(sizeof(order_entry) * (size_t)(N > 0 ? N : 1));
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) {
        project3d(params + i * P, cam, H, W, o->dil, o->fmode, s->k[i].valid, &s->w[i]);
        if (o->sh) sh_colour(params + i * P, cam, o->sh, &s->w[i]);
        if (s->k[i].valid) { e[n].depth = f32_bits(s->k[i].depth); e[n].prim = (uint32_t)i; ++n; }
    }
    qsort(e, (size_t)n, sizeof(order_entry), cmp_order);
    s->order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) s->order[j] = e[j].prim;
    s->nvalid = n;
    free(e);
}

static void scene3_free(scene3* s) { free(s->k); free(s->w); free(s->order); }

/* Threshold decisions (alpha_min skip, alpha_max clamp, T_min stop: Eq. 3 with the 3DGS constants).
 * A decision that floating point turns into a branch is taken, on both sides, from the values the
 * kernels decide with: the primitive's binary32 projected record (centre, Cholesky factor of
 * Sigma'^-1, frequency, phase in cycles, opacity; bit-exact with the kernels' footprint rule).
 * The oracle evaluates alpha from that record exactly (binary64), and decides with it.  The
 * kernels evaluate the same expression in binary32 with approximate exp2 and cos; the bound below
 * follows their operations one by one, so a decision whose exact value lies farther than the bound
 * from its threshold is the kernels' decision too.  Pixels with a decision inside its bound are
 * reported as ambiguous.  The colour values themselves are still accumulated from the binary64
 * projection (proj), so the image keeps the full precision of the method.
 *
 * Error constants of the approximate instructions, taken conservatively from their documented
 * accuracy: cos.approx.f32 absolute error <= 2^-20 on [-pi, pi]; ex2.approx.f32 relative error
 * <= 2^-21.  U = 2^-24 is the unit roundoff of binary32. */
#define U32 5.9604644775390625e-08
#define EPS_COS 9.5367431640625e-07
#define EPS_EX2 4.76837158203125e-07
#define AMB_SAFETY 1.5
#define AMB_ALPHA_MIN 1 /* bit 0: the alpha_min skip could go either way */
#define AMB_T_MIN 2     /* bit 1: the T_min stop could go either way */
#define AMB_ALPHA_MAX 4 /* bit 2: the alpha_max clamp could go either way (a kink, not a jump) */

/* alpha before the clamp, o W'(x), from the binary32 record, in binary64; *bound receives an upper
 * bound of |kernel value - exact value|.  The kernel computes, in binary32:
 *   dx = px - mx, dy = py - my;  a = fma(l11, dx, l21 dy);  b = l22 dy;  q = fma(a, a, b b);
 *   G = ex2(q * (-log2(e) / 2));  t = fma(fx, dx, fma(fy, dy, phc));
 *   ang = (t - rint(t)) * 2pi;  M = fma(hk, cos(ang), 1/2);  raw = o (M G),
 * with hk = 1/2, or under frequency map 2 hk = ex2(kx) / 2 = kappa / 2 from the record's exponent
 * (ex2's relative error on top; a result below the smallest normal binary32 may be flushed). */
static double alpha_decision(const fp32_footprint* k, int fmode, int u, int v, double* bound) {
    const double dx = ((double)u + 0.5) - (double)k->mx, dy = ((double)v + 0.5) - (double)k->my;
    const double l11 = k->l11, l21 = k->l21, l22 = k->l22;
    const double fx = k->fp[fmode][0], fy = k->fp[fmode][1], phc = k->phc, o = k->op;
    const double a = l11 * dx + l21 * dy, b = l22 * dy;
    const double q = a * a + b * b;
    const double G = exp(-0.5 * q);
    const double s1 = fy * dy + phc, t = fx * dx + s1;
    const double ang = 2.0 * PI * (t - nearbyint(t));
    const double ca = cos(ang), sa = sin(ang);
    const double hk = fmode == 2 ? 0.5 * exp2((double)k->kx) : 0.5;
    const double dhk = fmode == 2 ? hk * EPS_EX2 + 0x1p-126 : 0.0;
    const double M = 0.5 + hk * ca, raw = o * M * G;
    /* rounding of the kernel's steps, first order, with every term taken in absolute value */
    const double ddx = U32 * fabs(dx), ddy = U32 * fabs(dy);
    const double da = fabs(l11) * ddx + fabs(l21) * ddy + U32 * (fabs(l21 * dy) + fabs(a));
    const double db = fabs(l22) * ddy + U32 * fabs(b);
    const double dq = 2.0 * fabs(a) * da + 2.0 * fabs(b) * db + da * da + db * db + U32 * (b * b + q);
    const double e = 0.5 * q * 1.4426950408889634;          /* |q * (-log2(e) / 2)| */
    const double de = 0.7213475204444817 * dq + 2.0 * U32 * e; /* the constant's and the product's rounding */
    const double dG = G * (EPS_EX2 + 0.6931471805599453 * de);
    const double dt = fabs(fx) * ddx + fabs(fy) * ddy + U32 * (fabs(s1) + fabs(t));
    const double dang = 2.0 * PI * dt + 2.0 * U32 * fabs(ang);
    const double dcos = fabs(sa) * dang + 0.5 * dang * dang + EPS_COS;
    const double dM = hk * dcos + fabs(ca) * dhk + U32 * M;
    const double dW = M * dG + G * dM + dM * dG + U32 * M * G;
    *bound = AMB_SAFETY * (o * dW + U32 * raw) + 1e-15;
    return raw;
}

typedef struct { uint32_t prim; double alpha, T, Wv; int clamped; wval e; } contrib;

/* Blend one pixel front to back.  Writes the contributors (when list != NULL), returns their count.
 * *amb collects the AMB_* bits of the threshold decisions taken within their error bounds.
 * The decisions use the record's alpha (alpha_decision) and the transmittance built from it,
 * T_dec, whose relative error in the kernels is at most Trel: per contributor its alpha's bound
 * over 1 - alpha plus the rounding of 1 - alpha and of the product. */
static int64_t blend_pixel(const scene3* s, int u, int v, const blend_opts* o, int truncated, double C[3],
                           double* Tout, int* amb, contrib* list) {
    double T = 1.0, Tdec = 1.0, Trel = 0.0;
    float k2 = o->cutoff * o->cutoff;
    int64_t n = 0;
    C[0] = C[1] = C[2] = 0.0;
    *amb = 0;
    for (int64_t j = 0; j < s->nvalid; ++j) {
        uint32_t i = s->order[j];
        if (truncated && !(q32(&s->k[i], u, v) <= k2)) continue;
        double bound;
        const double rdec = alpha_decision(&s->k[i], o->fmode, u, v, &bound);
        if (o->amin > 0.0f && fabs(rdec - (double)o->amin) <= bound) *amb |= AMB_ALPHA_MIN;
        if (fabs(rdec - (double)o->amax) <= bound) *amb |= AMB_ALPHA_MAX;
        const int clamped = rdec > (double)o->amax;
        const double adec = clamped ? (double)o->amax : rdec;
        if (adec < (double)o->amin) continue;
        const double testTdec = Tdec * (1.0 - adec);
        const double rel = Trel + (clamped ? 0.0 : bound / (1.0 - adec)) + 2.0 * U32;
        if (o->Tmin > 0.0f && fabs(testTdec - (double)o->Tmin) <= AMB_SAFETY * rel * testTdec) *amb |= AMB_T_MIN;
        if (testTdec < (double)o->Tmin) break;
        /* the value: the binary64 projection */
        wval e;
        eval_wavelet(&s->w[i], u, v, &e);
        const double alpha = clamped ? (double)o->amax : s->w[i].o * e.W;
        for (int ch = 0; ch < 3; ++ch) C[ch] += s->w[i].c[ch] * alpha * T;
        if (list) {
            list[n].prim = i; list[n].alpha = alpha; list[n].T = T; list[n].Wv = e.W;
            list[n].clamped = clamped; list[n].e = e;
        }
        ++n;
        T *= 1.0 - alpha;
        Tdec = testTdec;
        Trel = rel;
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] += T * o->bg[ch];
    *Tout = T;
    return n;
}

/* out[npix,3], Tout[npix], ncontrib[npix], ambiguous[npix] = AMB_* bits (any may be NULL except out) */
int wo_render3d(const float* params, int64_t N, const float* cam, int H, int W, const float* opts, int truncated,
                const int32_t* pix, int64_t npix, double* out, double* Tout, int32_t* ncontrib, uint8_t* ambiguous) {
    blend_opts o = read_opts(opts);
    scene3 s;
    scene3_build(params, N, cam, H, W, &o, &s);
    int64_t np = pix ? npix : (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < np; ++j) {
        int u, v, amb;
        pixel_of(pix, j, W, &u, &v);
        double C[3], T;
        int64_t n = blend_pixel(&s, u, v, &o, truncated, C, &T, &amb, NULL);
        for (int ch = 0; ch < 3; ++ch) out[j * 3 + ch] = C[ch];
        if (Tout) Tout[j] = T;
        if (ncontrib) ncontrib[j] = (int32_t)n;
        if (ambiguous) ambiguous[j] = (uint8_t)amb;
    }
    scene3_free(&s);
    return 0;
}

/* d(entry of R(q))/d(q) for a unit quaternion q = (w, x, y, z); dR[e*4 + m] = dR_e / dq_m */
static void quat_rot_jac(const double q[4], double dR[36]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double J[36] = {
        /* R00 */ 0, 0, -4 * y, -4 * z,
        /* R01 */ -2 * z, 2 * y, 2 * x, -2 * w,
        /* R02 */ 2 * y, 2 * z, 2 * w, 2 * x,
        /* R10 */ 2 * z, 2 * y, 2 * x, 2 * w,
        /* R11 */ 0, -4 * x, 0, -4 * z,
        /* R12 */ -2 * x, -2 * w, 2 * z, 2 * y,
        /* R20 */ -2 * y, 2 * z, -2 * w, 2 * x,
        /* R21 */ 2 * x, 2 * w, 2 * z, 2 * y,
        /* R22 */ 0, -4 * x, -4 * y, 0};
    memcpy(dR, J, sizeof(J));
}

/* chain the image-plane gradient of a 3D primitive to its record:
 * mu(3) s(3) q(4) f(3) phi opacity c(3) */
static void chain3d(const proj* w, const float* p, const float* cam, const pgrad* g, double* out) {
    double fx = cam[12], fy = cam[13];
    double tx = w->t[0], ty = w->t[1], tz = w->t[2];
    memset(out, 0, sizeof(double) * (w->sh ? P3D_SH : 20));
    /* frequency map 2: (f', kappa) depend on t, s, the unit quaternion and fc; dmap[k] holds their
       derivatives by input k (t(3), s(3), qn(4), fc(3)) and gmap[k] the gradient they pass on */
    double gmap[13] = {0};
    if (w->fmode == 2) {
        double val[3], dmap[13][3];
        damped_freq_eval(w, fx, fy, val, dmap);
        for (int k = 0; k < 13; ++k) gmap[k] = g->f[0] * dmap[k][0] + g->f[1] * dmap[k][1] + g->kap * dmap[k][2];
    }
    /* K = Sigma'^-1:  dL/dSigma' = -K (dL/dK) K */
    double t1[4], gS2[4];
    matmul(w->K, g->K, t1, 2, 2, 2);
    matmul(t1, w->K, gS2, 2, 2, 2);
    for (int a = 0; a < 4; ++a) gS2[a] = -gS2[a];
    /* Sigma' = J Sc J^T + dil I:  dL/dJ = (G + G^T) J Sc,  dL/dSc = J^T G J */
    double Gs[4] = {gS2[0] + gS2[0], gS2[1] + gS2[2], gS2[2] + gS2[1], gS2[3] + gS2[3]};
    double JSc[6], gJ[6], Jt[6], tmp[6], gSc[9];
    matmul(w->J, w->Sc, JSc, 2, 3, 3);
    matmul(Gs, JSc, gJ, 2, 2, 3);
    transpose(w->J, Jt, 2, 3);
    matmul(Jt, gS2, tmp, 3, 2, 2);
    matmul(tmp, w->J, gSc, 3, 2, 3);
    /* Sc = V Sigma V^T:  dL/dSigma = V^T gSc V */
    double Vt[9], t9[9], gSig[9];
    transpose(w->V, Vt, 3, 3);
    matmul(Vt, gSc, t9, 3, 3, 3);
    matmul(t9, w->V, gSig, 3, 3, 3);
    /* Sigma = M M^T:  dL/dM = (gSig + gSig^T) M */
    double gSym[9], gM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gSym[i * 3 + j] = gSig[i * 3 + j] + gSig[j * 3 + i];
    matmul(gSym, w->M, gM, 3, 3, 3);
    /* M = R S */
    double gR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            gR[i * 3 + j] = gM[i * 3 + j] * w->s[j];
            out[3 + j] += gM[i * 3 + j] * w->R[i * 3 + j];
        }
    /* R(qn), qn = q / |q| */
    double dR[36], gqn[4] = {0, 0, 0, 0};
    quat_rot_jac(w->qn, dR);
    for (int e = 0; e < 9; ++e)
        for (int m = 0; m < 4; ++m) gqn[m] += gR[e] * dR[e * 4 + m];
    for (int m = 0; m < 4; ++m) gqn[m] += gmap[6 + m];
    for (int j = 0; j < 3; ++j) out[3 + j] += gmap[3 + j];
    double dot = 0.0;
    for (int m = 0; m < 4; ++m) dot += w->qn[m] * gqn[m];
    for (int m = 0; m < 4; ++m) out[6 + m] = (gqn[m] - w->qn[m] * dot) / w->qnorm;
    /* camera-frame centre t: through mu', f' and J */
    double gt[3] = {0, 0, 0};
    gt[0] += g->mu[0] * fx / tz;
    gt[2] += -g->mu[0] * fx * tx / (tz * tz);
    gt[1] += g->mu[1] * fy / tz;
    gt[2] += -g->mu[1] * fy * ty / (tz * tz);
    double gfc[3];
    if (w->fmode == 2) {
        for (int k = 0; k < 3; ++k) {
            gt[k] += gmap[k];
            gfc[k] = gmap[10 + k];
        }
    } else if (w->fmode) {
        /* f' = J fc: dL/dfc = J^T dL/df', and dL/dJ gains dL/df' fc^T */
        for (int k = 0; k < 3; ++k) {
            gfc[k] = w->J[k] * g->f[0] + w->J[3 + k] * g->f[1];
            gJ[k] += g->f[0] * w->fc[k];
            gJ[3 + k] += g->f[1] * w->fc[k];
        }
    } else {
        gfc[0] = g->f[0] * tz / fx;
        gfc[1] = g->f[1] * tz / fy;
        gfc[2] = 0.0;
        gt[2] += g->f[0] * w->fc[0] / fx + g->f[1] * w->fc[1] / fy;
    }
    /* J = [[fx/tz, 0, -fx txz/tz], [0, fy/tz, -fy tyz/tz]], txz = clamp(tx/tz) */
    double txz = -w->J[2] * tz / fx, tyz = -w->J[5] * tz / fy;
    gt[2] += gJ[0] * (-fx / (tz * tz));
    gt[2] += gJ[4] * (-fy / (tz * tz));
    gt[2] += gJ[2] * (fx * txz / (tz * tz));
    gt[2] += gJ[5] * (fy * tyz / (tz * tz));
    if (w->unclamped_x) {
        /* d txz/dtx = 1/tz, d txz/dtz = -tx/tz^2 */
        gt[0] += gJ[2] * (-fx / tz) * (1.0 / tz);
        gt[2] += gJ[2] * (-fx / tz) * (-tx / (tz * tz));
    }
    if (w->unclamped_y) {
        gt[1] += gJ[5] * (-fy / tz) * (1.0 / tz);
        gt[2] += gJ[5] * (-fy / tz) * (-ty / (tz * tz));
    }
    /* t = V mu + t0,  fc = V f */
    for (int j = 0; j < 3; ++j) {
        out[j] = Vt[j * 3 + 0] * gt[0] + Vt[j * 3 + 1] * gt[1] + Vt[j * 3 + 2] * gt[2];
        out[10 + j] = Vt[j * 3 + 0] * gfc[0] + Vt[j * 3 + 1] * gfc[1] + Vt[j * 3 + 2] * gfc[2];
    }
    out[13] = g->phi;
    out[14] = g->o;
    out[15] = g->c[0]; out[16] = g->c[1]; out[17] = g->c[2];
    if (w->sh) {
        /* c_ch = max(0, 1/2 + sum_k Y_k(dir) sh_k,ch): dL/dsh_k,ch = dL/dc_ch Y_k where unclamped, and the
           centre gains dL/ddir (I - dir dir^T) / |mu - camera centre| */
        double Y[16], dY[16][3], gdir[3] = {0, 0, 0};
        sh_basis(w->dir, Y, dY);
        const int nk = (w->sh + 1) * (w->sh + 1);
        for (int ch = 0; ch < 3; ++ch) {
            const double gc = w->raw[ch] > 0.0 ? g->c[ch] : 0.0;
            for (int k = 0; k < nk; ++k) {
                const double v = gc * Y[k];
                if (k == 0) out[15 + ch] = v;
                else out[20 + 3 * (k - 1) + ch] = v;
                const double a = gc * sh_coef(p, k, ch);
                for (int j = 0; j < 3; ++j) gdir[j] += a * dY[k][j];
            }
        }
        const double dd = gdir[0] * w->dir[0] + gdir[1] * w->dir[1] + gdir[2] * w->dir[2];
        for (int j = 0; j < 3; ++j) out[j] += (gdir[j] - dd * w->dir[j]) / w->dist;
    }
}

static void pgrad_add(pgrad* g, const pgrad* a) {
    for (int m = 0; m < 2; ++m) { g->mu[m] += a->mu[m]; g->f[m] += a->f[m]; }
    for (int m = 0; m < 4; ++m) g->K[m] += a->K[m];
    for (int m = 0; m < 3; ++m) g->c[m] += a->c[m];
    g->phi += a->phi;
    g->o += a->o;
    g->kap += a->kap;
}

/* grad[N,20] (or [N,P3D_SH] with SH colour) of L = sum_pixels dldimg . C.  Pixels with a zero upstream
 * gradient are skipped.
 * gabs (optional) as in wo_grad2d. */
int wo_grad3d(const float* params, int64_t N, const float* cam, int H, int W, const float* opts, int truncated,
              const float* dldimg, double* grad, double* gabs) {
    blend_opts o = read_opts(opts);
    scene3 s;
    scene3_build(params, N, cam, H, W, &o, &s);
    int nthreads = 1;
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    nthreads = omp_get_max_threads();
#endif
    const int P = rec3_stride(&o);
    pgrad* acc = (pgrad*)calloc((size_t)nthreads * (size_t)(N > 0 ? N : 1), sizeof(pgrad));
    double* abs_acc = gabs ? (double*)calloc((size_t)nthreads * (size_t)(N > 0 ? N : 1) * P, sizeof(double)) : NULL;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        extern int omp_get_thread_num(void);
        tid = omp_get_thread_num();
#endif
        pgrad* my = acc + (size_t)tid * (size_t)(N > 0 ? N : 1);
        contrib* list = (contrib*)malloc(sizeof(contrib) * (size_t)(s.nvalid > 0 ? s.nvalid : 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < (int64_t)H * W; ++j) {
            int u = (int)(j % W), v = (int)(j / W);
            const float* gp = dldimg + j * 3;
            if (gp[0] == 0.0f && gp[1] == 0.0f && gp[2] == 0.0f) continue;
            double C[3], T;
            int amb;
            int64_t n = blend_pixel(&s, u, v, &o, truncated, C, &T, &amb, list);
            /* S = sum over later contributors of c alpha T, plus the background term */
            double S[3] = {T * o.bg[0], T * o.bg[1], T * o.bg[2]};
            for (int64_t m = n - 1; m >= 0; --m) {
                contrib* cb = &list[m];
                proj* w = &s.w[cb->prim];
                pgrad one;
                memset(&one, 0, sizeof(one));
                double galpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    one.c[ch] = gp[ch] * cb->alpha * cb->T;
                    galpha += gp[ch] * (w->c[ch] * cb->T - S[ch] / (1.0 - cb->alpha));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += w->c[ch] * cb->alpha * cb->T;
                if (!cb->clamped) {
                    one.o = galpha * cb->Wv;
                    accum_wavelet_grad(w, &cb->e, galpha * w->o, &one);
                }
                pgrad_add(&my[cb->prim], &one);
                if (abs_acc) {
                    double t[P3D_SH];
                    chain3d(w, params + (size_t)cb->prim * P, cam, &one, t);
                    double* a = abs_acc + ((size_t)tid * (size_t)N + cb->prim) * P;
                    for (int q = 0; q < P; ++q) a[q] += fabs(t[q]);
                }
            }
        }
        free(list);
    }
    for (int64_t i = 0; i < N; ++i) {
        pgrad g;
        memset(&g, 0, sizeof(g));
        for (int t = 0; t < nthreads; ++t) {
            pgrad* a = &acc[(size_t)t * (size_t)N + (size_t)i];
            for (int m = 0; m < 2; ++m) { g.mu[m] += a->mu[m]; g.f[m] += a->f[m]; }
            for (int m = 0; m < 4; ++m) g.K[m] += a->K[m];
            for (int m = 0; m < 3; ++m) g.c[m] += a->c[m];
            g.phi += a->phi;
            g.o += a->o;
            g.kap += a->kap;
        }
        if (s.w[i].valid) chain3d(&s.w[i], params + i * P, cam, &g, grad + i * P);
        else memset(grad + i * P, 0, sizeof(double) * P);
        if (gabs) {
            for (int q = 0; q < P; ++q) {
                double a = 0.0;
                for (int t = 0; t < nthreads; ++t) a += abs_acc[((size_t)t * (size_t)N + (size_t)i) * P + q];
                gabs[i * P + q] = a;
            }
        }
    }
    free(abs_acc);
    free(acc);
    scene3_free(&s);
    return 0;
}

/* Binary64 projection of each primitive, out[N,16]:
 * valid, tz, mu'x, mu'y, Sigma'00, Sigma'01, Sigma'11, f'x, f'y, phi, opacity, c(3), kappa, 0 */
int wo_project3d(const float* params, int64_t N, const float* cam, int H, int W, const float* opts, double* out) {
    blend_opts o = read_opts(opts);
    const int P = rec3_stride(&o);
    for (int64_t i = 0; i < N; ++i) {
        fp32_footprint k;
        footprint3d(params + i * P, cam, o.cutoff, o.dil, W, H, &k);
        proj w;
        project3d(params + i * P, cam, H, W, o.dil, o.fmode, k.valid, &w);
        if (o.sh) sh_colour(params + i * P, cam, o.sh, &w);
        double S2[4];
        mat2_inv(w.K, S2);
        double* r = out + i * 16;
        memset(r, 0, sizeof(double) * 16);
        r[0] = w.valid; r[1] = w.t[2]; r[2] = w.mu[0]; r[3] = w.mu[1];
        r[4] = S2[0]; r[5] = S2[1]; r[6] = S2[3];
        r[7] = w.f[0]; r[8] = w.f[1]; r[9] = w.phi; r[10] = w.o;
        r[11] = w.c[0]; r[12] = w.c[1]; r[13] = w.c[2];
        r[14] = w.kap;
    }
    return 0;
}

/* The threshold-decision values of (primitive, pixel) pairs: out[n,4] = the record's binary32
 * values the decision reads are in rec[N,10] (mx, my, l11, l21, l22, f'x, f'y, phase in cycles,
 * opacity, and under frequency map 2 the damping exponent kx, else 0; zeros for an invalid
 * primitive); per pair (prim, u, v) in pairs[n,3]: out[n,3] = the
 * record's alpha before the clamp, its kernel error bound, and the alpha of the binary64 projection. */
int wo_alpha_decisions(const float* params, int64_t N, const float* cam, int H, int W, const float* opts,
                       const int32_t* pairs, int64_t n, float* rec, double* out) {
    blend_opts o = read_opts(opts);
    const int P = rec3_stride(&o);
    fp32_footprint* k = all_footprints(o.sh ? KIND_3D_SH : KIND_3D, params, N, cam, H, W, o.cutoff, o.dil);
    if (rec)
        for (int64_t i = 0; i < N; ++i) {
            float* r = rec + i * 10;
            memset(r, 0, sizeof(float) * 10);
            if (!k[i].valid) continue;
            r[0] = k[i].mx; r[1] = k[i].my; r[2] = k[i].l11; r[3] = k[i].l21; r[4] = k[i].l22;
            r[5] = k[i].fp[o.fmode][0]; r[6] = k[i].fp[o.fmode][1]; r[7] = k[i].phc; r[8] = k[i].op;
            r[9] = o.fmode == 2 ? k[i].kx : 0.0f;
        }
    for (int64_t j = 0; j < n; ++j) {
        const int32_t i = pairs[j * 3], u = pairs[j * 3 + 1], v = pairs[j * 3 + 2];
        double* r = out + j * 3;
        r[0] = r[1] = r[2] = 0.0;
        if (i < 0 || i >= N || !k[i].valid) continue;
        r[0] = alpha_decision(&k[i], o.fmode, u, v, &r[1]);
        proj w;
        project3d(params + (int64_t)i * P, cam, H, W, o.dil, o.fmode, 1, &w);
        wval e;
        eval_wavelet(&w, u, v, &e);
        r[2] = w.o * e.W;
    }
    free(k);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* 6D: per-primitive linear time model                                                         */
/* ------------------------------------------------------------------------------------------ */

/* Reading of the 6D deformation (Sec. 4.3 gives it only as an MLP of unstated architecture):
 * mu(t) = mu0 + v t, f(t) = f0 + df t, phi(t) = phi0 + dphi t, log s(t) = log s0 + dlog_s t.
 * in[N,32] -> out[N,20] */
int wo_deform6d(const float* params6, int64_t N, double t, double* out3) {
    for (int64_t i = 0; i < N; ++i) {
        const float* p = params6 + i * 32;
        double* o = out3 + i * 20;
        for (int j = 0; j < 20; ++j) o[j] = p[j];
        for (int j = 0; j < 3; ++j) {
            o[j] = (double)p[j] + (double)p[20 + j] * t;
            o[3 + j] = (double)p[3 + j] * exp((double)p[27 + j] * t);
            o[10 + j] = (double)p[10 + j] + (double)p[23 + j] * t;
        }
        o[13] = (double)p[13] + (double)p[26] * t;
    }
    return 0;
}

/* chain dL/d(deformed record)[N,20] to dL/d(record6)[N,32] */
int wo_deform6d_grad(const float* params6, int64_t N, double t, const double* g3, double* g6) {
    for (int64_t i = 0; i < N; ++i) {
        const float* p = params6 + i * 32;
        const double* g = g3 + i * 20;
        double* o = g6 + i * 32;
        memset(o, 0, sizeof(double) * 32);
        for (int j = 0; j < 20; ++j) o[j] = g[j];
        for (int j = 0; j < 3; ++j) {
            double e = exp((double)p[27 + j] * t);
            o[20 + j] = g[j] * t;
            o[3 + j] = g[3 + j] * e;
            o[27 + j] = g[3 + j] * (double)p[3 + j] * e * t;
            o[23 + j] = g[10 + j] * t;
        }
        o[26] = g[13] * t;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* footprint check: every (pixel, primitive) pair that passes the binary32 cutoff test must     */
/* lie inside the primitive's covered pixel range (so tile lists lose no contribution)          */
/* ------------------------------------------------------------------------------------------ */

/* counts[0] = pairs inside the cutoff ellipse, counts[1] = of those, pairs outside the pixel range,
 * counts[2] = pixels inside the pixel ranges, counts[3] = cutoff pairs whose tile (or whose own
 * one-pixel rectangle) the ellipse test rejects */
int wo_cutoff_coverage(int kind, const float* params, int64_t N, const float* cam, int H, int W, float cutoff,
                       float dil, int64_t* counts) {
    fp32_footprint* k = all_footprints(kind, params, N, cam, H, W, cutoff, dil);
    float k2 = cutoff * cutoff;
    float lim = touch_limit(cutoff);
    int64_t inside = 0, outside = 0, rect_px = 0, untouched = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : inside, outside, rect_px, untouched)
    for (int64_t i = 0; i < N; ++i) {
        if (!k[i].valid) continue;
        if (k[i].u0 <= k[i].u1) rect_px += (int64_t)(k[i].u1 - k[i].u0 + 1) * (k[i].v1 - k[i].v0 + 1);
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                if (!(q32(&k[i], u, v) <= k2)) continue;
                ++inside;
                if (u < k[i].u0 || u > k[i].u1 || v < k[i].v0 || v > k[i].v1) { ++outside; continue; }
                int tx = u / TILE, ty = v / TILE;
                int x0 = tx * TILE > k[i].u0 ? tx * TILE : k[i].u0;
                int x1 = tx * TILE + TILE - 1 < k[i].u1 ? tx * TILE + TILE - 1 : k[i].u1;
                int y0 = ty * TILE > k[i].v0 ? ty * TILE : k[i].v0;
                int y1 = ty * TILE + TILE - 1 < k[i].v1 ? ty * TILE + TILE - 1 : k[i].v1;
                edge_ratios rr = footprint_ratios(&k[i]);
                if (!rect_touched(&k[i], rr, x0, x1, y0, y1, lim) || !rect_touched(&k[i], rr, u, u, v, v, lim)) ++untouched;
            }
    }
    counts[0] = inside;
    counts[1] = outside;
    counts[2] = rect_px;
    counts[3] = untouched;
    free(k);
    return 0;
}
