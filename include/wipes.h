/*
 * wipes.h — C ABI of the GB300 (sm_103a) wavelet rasterizer.
 *
 * The library renders wavelet primitives (Zhang et al., "WIPES: Wavelet-based Visual Primitives",
 * ICCV 2025) and differentiates the rendering:
 *   W(x) = 1/2 [cos(2 pi f.(x - mu) + phi) + 1] exp(-1/2 (x - mu)^T Sigma^-1 (x - mu))
 * (Sec. 4.1, Eq. 5; the phase phi is an added parameter, phi = 0 is the paper's primitive).
 *   2D image task:  C(x) = sum_i c_i W_i(x)                          (Eq. 4 with W, Sec. 4.3)
 *   3D view synthesis: project each primitive to the image plane (EWA, Sec. 3.1; frequency by the
 *   same ray-space map, Sec. 4.1) and alpha-blend front to back       (Eq. 3 with W', Sec. 4.1)
 *   Backward: the gradient of a scalar loss with respect to every primitive parameter, given
 *   dL/dimage (explicit gradients, Sec. 1).
 *
 * Conventions shared by every call:
 *   - All arrays are row-major float32 (uint32 where stated).  Unless a call says otherwise a
 *     pointer is a DEVICE pointer on the context's device, owned by the caller; the library never
 *     frees caller memory and keeps no pointer to it after the call returns (except as stated for
 *     wipes_state).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls enqueue
 *     work on it and return; WIPES_OK means "enqueued".  wipes_render2d/3d (and the prepare calls)
 *     read one value back to the host (the number of tile instances): each waits once for the work
 *     on `stream` up to the scan that produces it (the emission that follows is already enqueued
 *     and keeps running), then enqueues the rest.
 *   - Pixel (u, v) (column u, row v) is sampled at (u + 0.5, v + 0.5).  Images are [H, W, 3].
 *   - Frequencies are in cycles per pixel (2D) or cycles per world unit (3D); phases in radians.
 *   - On failure a call returns a non-zero wipes_status and wipes_last_error() describes it.
 *
 * Record layouts:
 *   2D [N,16]: mu_x, mu_y, s_x, s_y, theta, f_x, f_y, phi, c_r, c_g, c_b, (5 unused)
 *              Sigma = R(theta) diag(s_x^2, s_y^2) R(theta)^T (RS form, Sec. 5.1), or with
 *              wipes_opts.cov2d = 1: mu_x, mu_y, l1, l2, l3, f_x, f_y, phi, c_r, c_g, c_b, (5 unused),
 *              Sigma = L L^T with L = [[l1, 0], [l2, l3]], l1 l3 != 0 (Cholesky form, Sec. 5.1)
 *   3D [N,20]: mu(3), s(3), q(w,x,y,z), f(3), phi, opacity, c(3), (2 unused)
 *              Sigma = R(q/|q|) S S^T R^T (Sec. 3.1); q need not be normalised
 *   3D with spherical-harmonic colour (wipes_opts.sh_degree = d in 1..3) [N,68]: the 3D record, whose
 *              c(3) are the degree-0 coefficients, then the coefficients of basis functions
 *              k = 1..15 (degree l = 1..3, order m = -l..l), three channels each: [20 + 3 (k-1) + ch];
 *              coefficients above degree d are ignored (and get zero gradient).  Colour per channel:
 *              max(0, 1/2 + sum_k Y_k(dir) sh_k) with the real spherical harmonics Y_k (Condon-Shortley
 *              phase) at the unit vector dir from the camera centre to mu (the colour of 3DGS, Sec. 3.1)
 *   6D [N,32]: the 3D record followed by v(3), df(3), dphi, dlog_s(3), (2 unused)
 */
#ifndef WIPES_H
#define WIPES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WIPES_TILE 16      /* tile edge in pixels */
#define WIPES_P2D 16       /* floats per 2D record */
#define WIPES_P3D 20       /* floats per 3D record */
#define WIPES_P6D 32       /* floats per 6D record */
#define WIPES_P3D_SH 68    /* floats per 3D record with spherical-harmonic colour */

typedef enum {
    WIPES_OK = 0,
    WIPES_ERR_INVALID = 1,   /* bad argument (null pointer, size out of range, wrong call order) */
    WIPES_ERR_CAPACITY = 2,  /* the tile-instance count exceeds 2^31 - 1 */
    WIPES_ERR_CUDA = 3,      /* a CUDA runtime call failed; see wipes_last_error() */
    WIPES_ERR_TIMEOUT = 4,   /* a bounded device wait gave up */
    WIPES_ERR_OOM = 5        /* device allocation for the workspace failed */
} wipes_status;

typedef struct wipes_ctx wipes_ctx;      /* one device; owns no rendering buffers */
typedef struct wipes_state wipes_state;  /* the workspace of one forward pass, kept for its backward */

/* Pinhole camera (17 floats).  viewmat: world->camera [R|t], 3x4 row-major, OpenCV axes
 * (x right, y down, z forward).  A primitive with camera z <= near_z is culled. */
typedef struct {
    float viewmat[12];
    float fx, fy, cx, cy;
    float near_z;
} wipes_camera;

/* Rendering options.  Defaults (wipes_default_opts): cutoff_sigma 3, alpha_min 1/255,
 * alpha_max 0.99, T_min 1e-4, dilation 0.3 px^2 (3D) / 0 (2D), bg 0, freq_proj_mode 0, cov2d 0,
 * sh_degree 0. */
typedef struct {
    float cutoff_sigma;     /* a primitive counts at a pixel iff its squared Mahalanobis distance <= cutoff^2;
                             * 2^-10 <= cutoff_sigma <= 2^10, else WIPES_ERR_INVALID */
    float alpha_min;        /* 3D: alpha below this is skipped */
    float alpha_max;        /* 3D: alpha is clamped to this */
    float T_min;            /* 3D: blending stops before a primitive that takes T below this */
    float dilation;         /* 3D: added to the diagonal of Sigma' (px^2); ignored in 2D */
    float bg[3];            /* 3D: background colour, weighted by the final transmittance */
    int32_t freq_proj_mode; /* 3D: 0 = phase gradient on the fronto-parallel plane through the centre,
                               f' = (fc_x t_z / f_x, fc_y t_z / f_y) with fc = W f; 1 = the literal
                               f' = J W f (the covariance's ray-space map, Sec. 4.1); 2 = the
                               oscillation integrated along the viewing ray (Sec. 4.1's integral
                               over z, in the EWA ray space): f' = P0^T fc - (fc.n) Q_az / Q_zz and
                               W' = (1 + kappa cos(2 pi f'.x' + phi)) G' / 2 with the damping
                               kappa = exp(-2 pi^2 (fc.n)^2 / Q_zz), n the ray direction, P0 the
                               right inverse of J, Q = [P0|n]^T Sigma_c^-1 [P0|n] */
    int32_t cov2d;          /* 2D: 0 = RS record (s_x, s_y, theta), 1 = Cholesky record (l1, l2, l3) */
    int32_t sh_degree;      /* 3D: 0 = RGB colour of the [N,20] record; 1..3 = spherical-harmonic colour of
                               that degree from [N,68] records (params and dL/dparams) */
} wipes_opts;

/* Fill `out` with the defaults for dims = 2 or 3. */
void wipes_default_opts(int dims, wipes_opts* out);

/* Create a context on CUDA device `device`.  Errors: INVALID (bad device), CUDA.  A context holds
 * one host readback word pair, one event and the loss's reduction buffer: calls that use one
 * context are made from one host thread at a time (separate contexts serve concurrent threads or
 * concurrently running streams, as the bench's 6D samples do). */
wipes_status wipes_create(int device, wipes_ctx** out);
/* Destroy a context; fails with WIPES_ERR_INVALID (and destroys nothing) while states created on
 * it are alive. */
wipes_status wipes_destroy(wipes_ctx* ctx);

/* A state holds the device workspace of one forward pass (projected records, sorted tile lists,
 * tile ranges, and in 3D the final transmittance and contributor count per pixel).  Buffers grow
 * on demand (cudaMalloc) and are reused by later forward passes on the same state.  A state must
 * not be used by two calls that overlap on the GPU. */
wipes_status wipes_state_create(wipes_ctx* ctx, wipes_state** out);
wipes_status wipes_state_destroy(wipes_state* st);

/* 2D forward (summed field, Eq. 4 with W, Sec. 4.3).
 *   params [N,16] device, out [H,W,3] device (overwritten).  N >= 0, 1 <= H, W <= 16384.
 *   The state records N, H, W and options for wipes_render_backward. */
wipes_status wipes_render2d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, int H, int W,
                            const wipes_opts* opts, float* out, void* stream);

/* 3D forward (EWA projection, Sec. 3.1; frequency projection, Sec. 4.1; front-to-back blending of
 * W', Eq. 3 with W').  params [N,20] device, out [H,W,3] device (overwritten). */
wipes_status wipes_render3d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N,
                            const wipes_camera* cam, int H, int W, const wipes_opts* opts, float* out,
                            void* stream);

/* The forward passes split in two for batching: wipes_prepare2d/3d run everything but the blend
 * (projection, footprints, tile binning, sort) into `st`; wipes_blend_batch then renders any number
 * of prepared states, of any mix of 2D and 3D frames and image sizes, in persistent launches
 * (up to 128 frames per launch): every block takes (frame, tile) items from a device counter.  A
 * frame renders to the same bits alone (wipes_render2d/3d = prepare + one-frame blend) and in a
 * batch, because both paths run the same per-pixel code.  A state stays valid for further blends
 * until it is prepared again (and a 2D state for wipes_render_backward); outs[i] is [H_i, W_i, 3]
 * device memory.  At most 64 batch launches may be in flight on one context. */
wipes_status wipes_prepare2d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, int H, int W,
                             const wipes_opts* opts, void* stream);
wipes_status wipes_prepare3d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N,
                             const wipes_camera* cam, int H, int W, const wipes_opts* opts, void* stream);
wipes_status wipes_blend_batch(wipes_ctx* ctx, const wipes_state* const* states, float* const* outs, int n,
                               void* stream);

/* Backward of the last forward pass on `st` (explicit gradients, Sec. 1).
 *   params: the same [N,16|20] array the forward pass read, unchanged since.
 *   dL_dout [H,W,3] device.  dL_dparams [N,16|20] device, overwritten (unused columns are 0).
 *   3D: the walk back along a pixel's list runs in chunks of 256 entries at once, each from the
 *   pixel's transmittance and colour that the one-frame forward recorded at the chunk's end; so a
 *   3D backward needs wipes_render3d as the last forward on `st` (not prepare + batch).
 *   Errors: INVALID if `st` holds no forward pass, or (3D) its lists were not blended by
 *   wipes_render3d since they were prepared. */
wipes_status wipes_render_backward(wipes_ctx* ctx, wipes_state* st, const float* params, const float* dL_dout,
                                   float* dL_dparams, void* stream);

/* 6D time model (reading of the deformation of Sec. 4.3; the paper gives it only as an MLP):
 * mu(t) = mu0 + v t, f(t) = f0 + df t, phi(t) = phi0 + dphi t, log s(t) = log s0 + dlog_s t.
 *   params6 [N,32] device -> params3 [N,20] device. */
wipes_status wipes_deform6d(const float* params6, int64_t N, float t, float* params3, void* stream);
/* dL/dparams3 [N,20] -> dL/dparams6 [N,32]; accumulate != 0 adds into dL_dparams6. */
wipes_status wipes_deform6d_backward(const float* params6, int64_t N, float t, const float* dL_dparams3,
                                     float* dL_dparams6, int accumulate, void* stream);

/* Mean squared error between img and target (n floats each, device):
 * loss[0] = sum (img - target)^2 / n (device scalar), dL_dimg = 2 (img - target) / n.
 * Uses a small reduction buffer owned by ctx: calls on one ctx must not overlap on the GPU. */
wipes_status wipes_l2_loss(wipes_ctx* ctx, const float* img, const float* target, int64_t n, float* loss,
                           float* dL_dimg, void* stream);

/* The same loss without allocating device memory (the paper has no counterpart; this serves
 * callers that cannot call cudaMalloc: code whose allocator owns all device memory, hosts that
 * forbid device allocation after start-up).  Runs on the calling thread's
 * current device and needs no context.  Its scratch is a fixed 256 KB array inside the library's
 * device image (one partial sum per 4096 elements), held by every GPU that loads the library until
 * the process exits.  Limits: 1 <= n <= 268,435,456 (65,536 x 4,096); larger n returns
 * WIPES_ERR_INVALID.  Every call outside stream capture looks up the array's device address in
 * the current context (cudaGetSymbolAddress); a call on a capturing stream reuses the address of
 * the last call outside capture on that device, so make a first call on each device before any
 * stream capture (without one, the call fails with WIPES_ERR_CUDA).  The call does not switch
 * devices: img, target, loss and dL_dimg must be on the calling thread's current device.  The
 * array is per process and per device (other processes hold their own).  All calls on a device
 * in this process share it: calls that overlap on the GPU race.  Each call writes every partial
 * sum before reading it, so the array needs no clearing. */
wipes_status wipes_l2_loss_noalloc(const float* img, const float* target, int64_t n, float* loss, float* dL_dimg,
                                   void* stream);

/* Introspection of the last forward pass on a state (host-side values). */
typedef struct {
    int32_t dims;          /* 2, 3, or 0 if no forward pass */
    int32_t H, W, tiles_x, tiles_y;
    int64_t N;
    int64_t n_instances;   /* (tile, primitive) pairs in the sorted lists */
    int64_t bytes_reserved;/* device bytes held by the state */
} wipes_state_info;
wipes_status wipes_state_get_info(const wipes_state* st, wipes_state_info* info);

/* Copy the sorted tile lists of the last forward pass into caller device buffers:
 * tile_ids[n_instances], prim_ids[n_instances] (ordered by tile, then depth in 3D, then primitive
 * index) and tile_ranges[tiles_x * tiles_y * 2] ([start, end) per tile).  Any pointer may be NULL. */
wipes_status wipes_state_copy_lists(const wipes_state* st, uint32_t* tile_ids, uint32_t* prim_ids,
                                    uint32_t* tile_ranges, void* stream);
/* 3D: copy the final transmittance [H,W] and the per-pixel count of tile-list entries processed
 * up to the last contributor [H,W] into caller device buffers.  Either pointer may be NULL. */
wipes_status wipes_state_copy_pixel_state(const wipes_state* st, float* T_final, uint32_t* last_index,
                                          void* stream);

/* Count, over the sorted tile lists of the last forward pass, the (pixel, primitive) pairs a
 * kernel visits (pixel inside the image, primitive in the pixel's tile list) and the pairs inside
 * the cutoff ellipse (the terms of the sum of Eq. 4; in 3D the entries of Eq. 3 up to each pixel's
 * last contributor).  Synchronises `stream`; results are host values. */
wipes_status wipes_state_count_pairs(wipes_ctx* ctx, const wipes_state* st, int64_t* visited, int64_t* inside,
                                     void* stream);

/* Stage timing with CUDA events, for measurement.  When enabled on a context, every call on it
 * brackets each stage with events on the call's stream; wipes_get_timing synchronises the device,
 * adds the elapsed times of the completed brackets to per-stage totals, writes the totals
 * (milliseconds) and bracket counts for the WIPES_STAGE_COUNT stages, and resets them if asked. */
enum {
    WIPES_STAGE_FOOTPRINT = 0,   /* per-primitive projection, extents, tile counts */
    WIPES_STAGE_DEPTH_SORT = 1,  /* 3D: sort of the primitives by camera depth */
    WIPES_STAGE_SCAN = 2,        /* scan of tile counts and readback of the instance total */
    WIPES_STAGE_EMIT = 3,        /* emission of (tile, primitive) pairs */
    WIPES_STAGE_TILE_SORT = 4,   /* stable radix sort of the pairs by tile */
    WIPES_STAGE_RANGES = 5,      /* per-tile ranges */
    WIPES_STAGE_BLEND = 6,       /* forward rasterization (summed field or alpha blend) */
    WIPES_STAGE_BWD_RASTER = 7,  /* backward rasterization */
    WIPES_STAGE_BWD_CHAIN = 8,   /* backward reduction and chain to the record parameters */
    WIPES_STAGE_LOSS = 9,        /* wipes_l2_loss */
    WIPES_STAGE_MLP_FWD = 10,    /* wipes_deform_mlp */
    WIPES_STAGE_MLP_BWD = 11,    /* wipes_deform_mlp_backward */
    WIPES_STAGE_SORT = 12,       /* wipes_sort_pairs */
    WIPES_STAGE_COUNT = 13
};
wipes_status wipes_set_timing(wipes_ctx* ctx, int enable);
wipes_status wipes_get_timing(wipes_ctx* ctx, double* ms, int64_t* brackets, int reset);

/* Device memory of a context's workspaces (all its states).  With a limit set (bytes > 0; 0 removes
 * it), a call that would grow the workspaces past the limit fails with WIPES_ERR_OOM before
 * allocating; the caller can free states and retry.  Reserved bytes count every state buffer. */
wipes_status wipes_set_memory_limit(wipes_ctx* ctx, int64_t bytes);
wipes_status wipes_get_memory_reserved(wipes_ctx* ctx, int64_t* bytes);

/* Number of kernels this library has launched since it was loaded (all contexts, all threads). */
int64_t wipes_kernel_launches(void);

/* Static description of a status code. */
const char* wipes_status_string(wipes_status s);
/* Message of the last failure on the calling thread ("" if none). */
const char* wipes_last_error(void);
/* Synchronise `stream` and report any pending CUDA error, then any error latched on the device
 * since the last check: WIPES_ERR_TIMEOUT when a bounded device wait (the radix sort's look-back
 * over earlier tiles) ran out; the results of the calls enqueued since are then undefined.  A
 * latched error is reported once. */
wipes_status wipes_sync_status(wipes_ctx* ctx, void* stream);

/* 6D deformation network F_theta (Sec. 4.3): (dx, df, dSigma) = F_theta(gamma(x), gamma(t)).  The paper
 * gives only an MLP with positional encoding gamma; the network here: gamma(p) = (p, sin(2^k p),
 * cos(2^k p)) with k < 10 for the centre and k < 6 for t (76 inputs, padded to 80), 8 ReLU layers of
 * width 256, layer 5 taking (gamma, h_4), and 13 outputs (dx, dq, dlog s, df).  The deformed record
 * is mu + dx, q + dq, s exp(dlog s), f + df, the other fields unchanged.  theta: packed float32
 * parameters, per layer (out x in: 256x80, 4 x 256x256, 256x336, 2 x 256x256, 13x256) W row-major
 * then b; wipes_deform_mlp_param_count() floats.  The products run in bfloat16 with fp32
 * accumulation (cuBLASLt; the hidden layers' biases are applied in bfloat16, the output layer's in
 * fp32); activations are kept in `st` for the backward. */
int64_t wipes_deform_mlp_param_count(void);
/* params3: canonical [N,20] records; params_out: deformed [N,20] records (device, 16-byte aligned). */
wipes_status wipes_deform_mlp(wipes_ctx* ctx, wipes_state* st, const float* params3, int64_t N, float t,
                              const float* theta, float* params_out, void* stream);
/* From dL/d(deformed records) [N,20] of the last wipes_deform_mlp on `st` (same params3): dL/dtheta
 * [param_count] and dL/dparams3 [N,20], accumulated into the outputs when accumulate != 0, else
 * overwritten. */
wipes_status wipes_deform_mlp_backward(wipes_ctx* ctx, wipes_state* st, const float* params3, const float* dL_dout,
                                       float* dL_dtheta, float* dL_dparams3, int accumulate, void* stream);

/* The path's sort (Sec. 1: the GPU sort that orders the tile lists; also the depth sort of the 3D
 * primitives) as a call of its own, for tests and measurement.  Sorts the n (key, value) pairs in
 * keys[n], vals[n] (device, uint32, caller-owned) in place by the low key_bits bits of the key
 * (1..32), stably: pairs with equal low bits keep their input order; the high bits ride along.
 * One pass per 8 bits or fewer (the bits split evenly over ceil(key_bits / 8) passes) after one
 * histogram kernel.  `st` provides the second buffers (2 n words, kept for reuse) and the look-back
 * workspace; its render data are untouched.  An odd pass count ends with one device copy back.
 * Errors: WIPES_ERR_INVALID for n outside 0..2^31-1, key_bits outside 1..32 or null buffers;
 * WIPES_ERR_OOM under the context's memory limit.  Asynchronous on `stream`; a look-back wait that
 * ran out is reported by the next wipes_sync_status() as WIPES_ERR_TIMEOUT. */
wipes_status wipes_sort_pairs(wipes_ctx* ctx, wipes_state* st, uint32_t* keys, uint32_t* vals, int64_t n,
                              int key_bits, void* stream);

/* Diagnostic: run one radix-sort pass on scratch data in which the tile before the block's tile
 * never publishes its counts, so that the block's bounded look-back runs out (after well under a
 * second).  Returns WIPES_ERR_TIMEOUT when the wait ran out and was reported, as it should; the
 * context stays usable.  Allocates and frees about 140 KB of scratch; synchronises `stream`. */
wipes_status wipes_selftest_sort_timeout(wipes_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WIPES_H */
