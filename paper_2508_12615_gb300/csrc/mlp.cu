// 6D deformation network (Sec. 4.3): (dx, df, dSigma) = F_theta(gamma(x), gamma(t)) per primitive,
// and its backward to the network parameters and the canonical records.
//
// Network (the paper gives only "an MLP with positional encoding, as Deformable 3D Gaussians"):
//   gamma(p) = (p, sin(2^k p), cos(2^k p), k < L) per coordinate, L = 10 for the centre, 6 for t:
//     76 inputs, zero-padded to 80;
//   8 ReLU layers of width 256; layer 5 takes (gamma, h_4) (skip connection);
//   13 outputs: dx (3), dq (4), dlog s (3), df (3);
//   deformed record: mu + dx, q + dq, s exp(dlog s), f + df (phase, opacity, colour kept).
// Parameters theta: packed float32, per layer W (out x in, row-major) then b (out).
//
// The products are dense contractions over 200k-row activation matrices: they run on the tensor
// cores through cuBLASLt (bfloat16 operands, fp32 accumulation, bias + ReLU fused in the epilogue
// for the hidden layers, whose biases are used in bfloat16 like their weights).  Activations are kept in bfloat16 for the backward pass.  Layouts: every
// activation matrix is row-major [N, width]; in cuBLASLt's column-major terms that is a
// [width, N] matrix, so Y = X W^T + b is  Y^T (out x N) = W (out x in, i.e. column-major in x out
// read transposed) * X^T (in x N).  The skip input lives in one [N, 336] buffer: columns 0..79 the
// encoding (written by the encoder), columns 80..335 the output h_4 of layer 4.
#include <cublasLt.h>
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"

namespace wipes {

namespace {

constexpr int kLx = 10, kLt = 6;
constexpr int kIn = 3 * (1 + 2 * kLx) + (1 + 2 * kLt);  // 76
constexpr int kInPad = 80;
constexpr int kWidth = 256;
constexpr int kHidden = 8;
constexpr int kSkipLayer = 5;
constexpr int kOut = 13;
constexpr int kOutPad = 16;
constexpr int kX5 = kInPad + kWidth;  // 336

struct LayerShape {
    int out, in;
};
constexpr LayerShape kShapes[kHidden + 1] = {{kWidth, kInPad}, {kWidth, kWidth}, {kWidth, kWidth}, {kWidth, kWidth},
                                             {kWidth, kWidth}, {kWidth, kX5},    {kWidth, kWidth}, {kWidth, kWidth},
                                             {kOut, kWidth}};

int64_t layer_offset(int l) {
    int64_t k = 0;
    for (int i = 0; i < l; ++i) k += (int64_t)kShapes[i].out * kShapes[i].in + kShapes[i].out;
    return k;
}

// gamma(mu, t) into columns 0..79 of the [N, 336] bf16 buffer; one thread per (row, column).
__global__ void __launch_bounds__(256) k_mlp_encode(const float* __restrict__ params3, int64_t N, float t,
                                                    __nv_bfloat16* __restrict__ x5) {
    pdl_enter();
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * kInPad) return;
    const int64_t row = idx / kInPad;
    const int c = (int)(idx - row * kInPad);
    float v = 0.f;
    if (c < 3) {
        v = params3[row * WIPES_P3D + c];
    } else if (c < 3 + 6 * kLx) {
        const int k = (c - 3) / 6, r = (c - 3) % 6;
        const float x = params3[row * WIPES_P3D + (r % 3)] * (float)(1 << k);
        v = r < 3 ? sinf(x) : cosf(x);
    } else if (c == 3 + 6 * kLx) {
        v = t;
    } else if (c < kIn) {
        const int k = (c - 4 - 6 * kLx) / 2, r = (c - 4 - 6 * kLx) % 2;
        const float x = t * (float)(1 << k);
        v = r == 0 ? sinf(x) : cosf(x);
    }
    x5[row * kX5 + c] = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(256) k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                                 int64_t n) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// deformed record from the canonical record and the network outputs d [N, 16] (13 used): the
// output layer's bias b is added here, and d keeps the biased outputs for the backward.  VEC: the
// caller's record rows are 16-byte aligned and move in 16-byte pieces (d always does).
template <bool VEC>
__global__ void __launch_bounds__(256) k_mlp_apply(const float* __restrict__ params3, int64_t N,
                                                   float* __restrict__ d, const float* __restrict__ b,
                                                   float* __restrict__ out) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float p[WIPES_P3D], e[kOutPad], o[WIPES_P3D];
    load_row<VEC, WIPES_P3D>(p, params3 + i * WIPES_P3D);
    load_row<true, kOutPad>(e, d + i * kOutPad);
#pragma unroll
    for (int k = 0; k < kOut; ++k) e[k] += b[k];
    store_row<true, kOutPad>(d + i * kOutPad, e);
#pragma unroll
    for (int k = 0; k < WIPES_P3D; ++k) o[k] = p[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o[k] = p[k] + e[k];
        o[3 + k] = p[3 + k] * expf(e[7 + k]);
        o[10 + k] = p[10 + k] + e[10 + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) o[6 + k] = p[6 + k] + e[3 + k];
    store_row<VEC, WIPES_P3D>(out + i * WIPES_P3D, o);
}

// dL/dd (bfloat16, the backward's product operand) and the direct part of dL/dparams3; the output
// bias gradient is the column sum of the rounded dL/dd (summed over the warp, then the block)
template <bool VEC>
__global__ void __launch_bounds__(256) k_mlp_apply_backward(const float* __restrict__ params3, int64_t N,
                                                            const float* __restrict__ d,
                                                            const float* __restrict__ g_out,
                                                            __nv_bfloat16* __restrict__ gd,
                                                            float* __restrict__ g_params3, int accumulate,
                                                            float* __restrict__ db_head) {
    pdl_enter();
    __shared__ float s_db[kOutPad];
    if (threadIdx.x < kOutPad) s_db[threadIdx.x] = 0.f;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float gdr[kOutPad];  // the rounded dL/dd of this row (0 past N)
#pragma unroll
    for (int k = 0; k < kOutPad; ++k) gdr[k] = 0.f;
    if (i < N) {
        float p[WIPES_P3D], e[kOutPad], g[WIPES_P3D];
        load_row<VEC, WIPES_P3D>(p, params3 + i * WIPES_P3D);
        load_row<true, kOutPad>(e, d + i * kOutPad);
        load_row<VEC, WIPES_P3D>(g, g_out + i * WIPES_P3D);
        float gdv[kOutPad];
#pragma unroll
        for (int k = 0; k < kOutPad; ++k) gdv[k] = 0.f;
        float gp[WIPES_P3D];
#pragma unroll
        for (int k = 0; k < WIPES_P3D; ++k) gp[k] = g[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float es = expf(e[7 + k]);
            gdv[k] = g[k];
            gdv[7 + k] = g[3 + k] * p[3 + k] * es;
            gdv[10 + k] = g[10 + k];
            gp[3 + k] = g[3 + k] * es;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) gdv[3 + k] = g[6 + k];
        uint32_t packed[kOutPad / 2];
#pragma unroll
        for (int k = 0; k < kOutPad; k += 2) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(gdv[k], gdv[k + 1]);
            packed[k / 2] = *reinterpret_cast<const uint32_t*>(&b2);
            const float2 f2v = __bfloat1622float2(b2);
            gdr[k] = f2v.x;
            gdr[k + 1] = f2v.y;
        }
        uint4* gd4 = reinterpret_cast<uint4*>(gd + i * kOutPad);
        gd4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        gd4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        float* go = g_params3 + i * WIPES_P3D;
        if (accumulate) {
            float prev[WIPES_P3D];
            load_row<VEC, WIPES_P3D>(prev, go);
#pragma unroll
            for (int k = 0; k < WIPES_P3D; ++k) gp[k] = prev[k] + gp[k];
        }
        store_row<VEC, WIPES_P3D>(go, gp);
    }
#pragma unroll
    for (int k = 0; k < kOut; ++k) {
        float v = gdr[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_db[k], v);
    }
    __syncthreads();
    if (threadIdx.x < kOut) atomicAdd(&db_head[threadIdx.x], s_db[threadIdx.x]);
}

// the output layer's weights += rows 0..12 of the padded [16, 256] weight gradient
__global__ void __launch_bounds__(256) k_mlp_add_head_dw(const float* __restrict__ dw_head16,
                                                         float* __restrict__ g_theta, int64_t head_off) {
    pdl_enter();
    const int c = threadIdx.x;
    for (int o = 0; o < kOut; ++o) g_theta[head_off + (int64_t)o * kWidth + c] += dw_head16[o * kWidth + c];
}

// the output layer's weights in bfloat16, zero-padded from 13 to 16 rows (aligned product shapes)
__global__ void __launch_bounds__(256) k_mlp_head16(const float* __restrict__ w_head, __nv_bfloat16* __restrict__ out) {
    pdl_enter();
    const int c = threadIdx.x;
    for (int o = 0; o < kOutPad; ++o) out[o * kWidth + c] = __float2bfloat16_rn(o < kOut ? w_head[o * kWidth + c] : 0.f);
}

// dz = dh where the layer's activation was positive (its ReLU bit-mask from the forward product)
// and the bias gradient (column sums of dz) of a 256-wide layer: a warp takes a row, each lane 8
// columns with a 16-byte access and one mask byte; the block sums its column totals in shared
// memory and adds them with one atomic per column
constexpr int kReluBlocks = 152 * 4;
constexpr int kReluRows = 4;  // rows a warp has in flight: its loads are issued before any is used
__global__ void __launch_bounds__(256) k_relu_backward(const __nv_bfloat16* __restrict__ dh, int ld_dh,
                                                       const uint8_t* __restrict__ mask, int64_t N,
                                                       __nv_bfloat16* __restrict__ dz, float* __restrict__ db) {
    pdl_enter();
    __shared__ float s_db[8][kWidth];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    const int64_t stride = (int64_t)gridDim.x * 8;
    for (int64_t r0 = (int64_t)blockIdx.x * 8 + g; r0 < N; r0 += kReluRows * stride) {
        uint4 vd[kReluRows];
        uint32_t mb[kReluRows];
#pragma unroll
        for (int j = 0; j < kReluRows; ++j) {
            const int64_t r = r0 + j * stride;
            vd[j] = make_uint4(0u, 0u, 0u, 0u);
            mb[j] = 0u;
            if (r < N) {
                mb[j] = mask[r * (kWidth / 8) + lane];  // activations 8 lane .. 8 lane + 7 of row r
                vd[j] = *reinterpret_cast<const uint4*>(dh + r * ld_dh + 8 * lane);
            }
        }
#pragma unroll
        for (int j = 0; j < kReluRows; ++j) {
            const int64_t r = r0 + j * stride;
            const __nv_bfloat162* pd = reinterpret_cast<const __nv_bfloat162*>(&vd[j]);
            uint4 vo;
            __nv_bfloat162* po = reinterpret_cast<__nv_bfloat162*>(&vo);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 fd = __bfloat1622float2(pd[k]);
                fd.x = (mb[j] >> (2 * k)) & 1u ? fd.x : 0.f;
                fd.y = (mb[j] >> (2 * k + 1)) & 1u ? fd.y : 0.f;
                po[k] = __floats2bfloat162_rn(fd.x, fd.y);  // exact: fd is a bfloat16 value or 0
                acc[2 * k] += fd.x;
                acc[2 * k + 1] += fd.y;
            }
            if (r < N) *reinterpret_cast<uint4*>(dz + r * kWidth + 8 * lane) = vo;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s_db[g][8 * lane + k] = acc[k];
    __syncthreads();
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += s_db[q][threadIdx.x];
    atomicAdd(&db[threadIdx.x], sum);
}

// dL/dmu through gamma: d/dx (x, sin(2^k x), cos(2^k x)) = (1, 2^k cos, -2^k sin); the encoding's
// gradient is the sum of layer 0's (dg0 [N, 80]) and layer 5's through its skip input (dgs [N, 80])
__global__ void __launch_bounds__(256) k_mlp_encode_backward(const float* __restrict__ params3, int64_t N,
                                                             const __nv_bfloat16* __restrict__ dg0,
                                                             const __nv_bfloat16* __restrict__ dgs,
                                                             float* __restrict__ g_params3) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // columns 0 .. 63 of both rows (the centre's encoding is columns 0 .. 62), in 16-byte pieces
    constexpr int kCols = 64;
    static_assert(3 + 6 * kLx <= kCols && kInPad % 8 == 0, "the centre's encoding fits the loaded columns");
    float ab[kCols];  // the encoding's gradient: layer 0's part plus the skip input's
#pragma unroll
    for (int q = 0; q < kCols / 8; ++q) {
        const uint4 va = reinterpret_cast<const uint4*>(dg0 + i * kInPad)[q];
        const uint4 vb = reinterpret_cast<const uint4*>(dgs + i * kInPad)[q];
        const uint32_t wa[4] = {va.x, va.y, va.z, va.w}, wb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wa[h]));
            const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wb[h]));
            ab[8 * q + 2 * h] = fa.x + fb.x, ab[8 * q + 2 * h + 1] = fa.y + fb.y;
        }
    }
    float gm[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) gm[j] = ab[j];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float x = params3[i * WIPES_P3D + j];
#pragma unroll
        for (int k = 0; k < kLx; ++k) {
            const float f = (float)(1 << k);
            const float gs = ab[3 + 6 * k + j];
            const float gc = ab[6 + 6 * k + j];
            float sn, cs;
            sincosf(f * x, &sn, &cs);
            gm[j] += f * (gs * cs - gc * sn);
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) g_params3[i * WIPES_P3D + j] += gm[j];
}

// ---------------------------------------------------------------------------------------------
// cuBLASLt products (column-major views, see the header comment)
// ---------------------------------------------------------------------------------------------

#define LT_TRY(x)                                                                                        \
    do {                                                                                                 \
        cublasStatus_t st_ = (x);                                                                        \
        if (st_ != CUBLAS_STATUS_SUCCESS) return std::string("cuBLASLt: " #x " failed with status ") + \
                                                 std::to_string((int)st_);                               \
    } while (0)

struct GemmKey {
    int ta, tb, m, n, k, lda, ldb, ldc, dtype, epi;
    bool operator<(const GemmKey& o) const {
        return std::tie(ta, tb, m, n, k, lda, ldb, ldc, dtype, epi) <
               std::tie(o.ta, o.tb, o.m, o.n, o.k, o.lda, o.ldb, o.ldc, o.dtype, o.epi);
    }
};

}  // namespace

struct MlpLt {
    cublasLtHandle_t h = nullptr;
    void* ws = nullptr;
    size_t ws_size = 32u << 20;
    std::map<GemmKey, cublasLtMatmulHeuristicResult_t> algos;
    std::mutex mu;
};

namespace {

// D (m x n, column-major, type dtype) = alpha op(A) op(B) (+ beta D) [+ bias, ReLU]; A, B bfloat16.
// The bias (when given) has the type of D: bfloat16 for the hidden layers, fp32 for the output layer.
std::string gemm(MlpLt& lt, bool ta, bool tb, int m, int n, int k, const void* A, int lda, const void* B, int ldb,
                 void* D, int ldc, cudaDataType_t dtype, float beta, cublasLtEpilogue_t epi, const void* bias,
                 cudaStream_t stream, void* aux = nullptr) {
    cublasLtMatmulDesc_t desc = nullptr;
    cublasLtMatrixLayout_t la = nullptr, lb = nullptr, lc = nullptr;
    LT_TRY(cublasLtMatmulDescCreate(&desc, CUBLAS_COMPUTE_32F, CUDA_R_32F));
    const cublasOperation_t opa = ta ? CUBLAS_OP_T : CUBLAS_OP_N, opb = tb ? CUBLAS_OP_T : CUBLAS_OP_N;
    LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_TRANSA, &opa, sizeof(opa)));
    LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_TRANSB, &opb, sizeof(opb)));
    LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_EPILOGUE, &epi, sizeof(epi)));
    if (bias) LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_BIAS_POINTER, &bias, sizeof(bias)));
    if (aux) {
        // ReLU bit-mask, one bit per element of D (m rows), leading dimension in bits
        const int64_t aux_ld = kWidth;
        LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_EPILOGUE_AUX_POINTER, &aux, sizeof(aux)));
        LT_TRY(cublasLtMatmulDescSetAttribute(desc, CUBLASLT_MATMUL_DESC_EPILOGUE_AUX_LD, &aux_ld, sizeof(aux_ld)));
    }
    LT_TRY(cublasLtMatrixLayoutCreate(&la, CUDA_R_16BF, ta ? k : m, ta ? m : k, lda));
    LT_TRY(cublasLtMatrixLayoutCreate(&lb, CUDA_R_16BF, tb ? n : k, tb ? k : n, ldb));
    LT_TRY(cublasLtMatrixLayoutCreate(&lc, dtype, m, n, ldc));
    const GemmKey key{ta, tb, m, n, k, lda, ldb, ldc, (int)dtype, (int)epi};
    cublasLtMatmulHeuristicResult_t res{};
    {
        std::lock_guard<std::mutex> g(lt.mu);
        auto it = lt.algos.find(key);
        if (it != lt.algos.end()) {
            res = it->second;
        } else {
            cublasLtMatmulPreference_t pref = nullptr;
            LT_TRY(cublasLtMatmulPreferenceCreate(&pref));
            LT_TRY(cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &lt.ws_size,
                                                        sizeof(lt.ws_size)));
            // the heuristic's candidates are timed once on this product and the fastest is kept:
            // its first choice is slow for some epilogues
            constexpr int kCandidates = 12;
            cublasLtMatmulHeuristicResult_t cand[kCandidates];
            int found = 0;
            const cublasStatus_t hs =
                cublasLtMatmulAlgoGetHeuristic(lt.h, desc, la, lb, lc, lc, pref, kCandidates, cand, &found);
            cublasLtMatmulPreferenceDestroy(pref);
            if (hs != CUBLAS_STATUS_SUCCESS || found == 0)
                return "cuBLASLt: no algorithm for the product (m=" + std::to_string(m) + ", n=" + std::to_string(n) +
                       ", k=" + std::to_string(k) + ")";
            res = cand[0];
            if (found > 1) {
                // trials write D (and the epilogue outputs) with beta 0: into a scratch copy when the
                // call accumulates (beta != 0), else into D itself, which the real call rewrites
                void* Dt = D;
                const size_t d_bytes = (size_t)ldc * n * (dtype == CUDA_R_32F ? 4 : 2);
                if (beta != 0.f && cudaMallocAsync(&Dt, d_bytes, stream) != cudaSuccess) Dt = nullptr;
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                const float one = 1.f, zero = 0.f;
                float best = 1e30f;
                for (int c = 0; Dt && c < found; ++c) {
                    float ms_sum = 0.f;
                    bool ok = true;
                    for (int rep = 0; rep < 3 && ok; ++rep) {
                        cudaEventRecord(e0, stream);
                        ok = cublasLtMatmul(lt.h, desc, &one, A, la, B, lb, &zero, Dt, lc, Dt, lc, &cand[c].algo, lt.ws,
                                            lt.ws_size, stream) == CUBLAS_STATUS_SUCCESS;
                        cudaEventRecord(e1, stream);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (rep > 0) ms_sum += ms;  // the first run warms up
                    }
                    if (ok && ms_sum < best) {
                        best = ms_sum;
                        res = cand[c];
                    }
                }
                cudaGetLastError();
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (Dt && Dt != D) cudaFreeAsync(Dt, stream);
            }
            lt.algos[key] = res;
        }
    }
    const float alpha = 1.f;
    const cublasStatus_t st = cublasLtMatmul(lt.h, desc, &alpha, A, la, B, lb, &beta, D, lc, D, lc, &res.algo, lt.ws,
                                             lt.ws_size, stream);
    cublasLtMatrixLayoutDestroy(la);
    cublasLtMatrixLayoutDestroy(lb);
    cublasLtMatrixLayoutDestroy(lc);
    cublasLtMatmulDescDestroy(desc);
    if (st != CUBLAS_STATUS_SUCCESS) return "cuBLASLt: matmul failed with status " + std::to_string((int)st);
    count_launches(1);
    return "";
}

// forward product of layer l: Y [N, out] (row-major, ldy) = X [N, in] (ldx) W^T + b, ReLU for hidden
// layers (bias b in bfloat16 for them, fp32 for the output layer), whose ReLU bit-mask goes to mask
std::string layer_forward(MlpLt& lt, int l, const __nv_bfloat16* w, const void* b, const void* x, int ldx, void* y,
                          int ldy, int64_t N, void* mask, cudaStream_t s) {
    const LayerShape sh = kShapes[l];
    if (l == kHidden)  // output layer: the padded [16, 256] weights, bias added by k_mlp_apply
        return gemm(lt, true, false, kOutPad, (int)N, kWidth, w, kWidth, x, ldx, y, ldy, CUDA_R_32F, 0.f,
                    CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
    return gemm(lt, true, false, sh.out, (int)N, sh.in, w, sh.in, x, ldx, y, ldy, CUDA_R_16BF, 0.f,
                CUBLASLT_EPILOGUE_RELU_AUX_BIAS, b, s, mask);
}

}  // namespace

MlpLt* mlp_lt_create(std::string* err) {
    MlpLt* lt = new MlpLt();
    if (cublasLtCreate(&lt->h) != CUBLAS_STATUS_SUCCESS) {
        *err = "cublasLtCreate failed";
        delete lt;
        return nullptr;
    }
    if (cudaMalloc(&lt->ws, lt->ws_size) != cudaSuccess) {
        *err = "cuBLASLt workspace allocation failed";
        cublasLtDestroy(lt->h);
        delete lt;
        return nullptr;
    }
    return lt;
}

void mlp_lt_destroy(MlpLt* lt) {
    if (!lt) return;
    cudaFree(lt->ws);
    cublasLtDestroy(lt->h);
    delete lt;
}

int64_t mlp_param_count() { return layer_offset(kHidden + 1); }

namespace {
// bytes of one hidden layer's ReLU bit-mask: 256 bits (32 bytes) per row, rows padded to 128
size_t mask_bytes(int64_t N) { return (size_t)((N + 127) / 128 * 128) * (kWidth / 8); }
}  // namespace

// element offset of the padded output layer in the bfloat16 parameter buffer (8 elements = 16 bytes)
int64_t head16_offset() { return (mlp_param_count() + 7) / 8 * 8; }

MlpSizes mlp_sizes(int64_t N) {
    MlpSizes z;
    // activations: x5 and seven 256-wide layers, then the eight hidden layers' ReLU bit-masks
    z.act = (size_t)N * (kX5 + 7 * kWidth) * sizeof(__nv_bfloat16) + mask_bytes(N) * kHidden;
    // dh [N, 256], dz [N, 256], encoding gradients [N, 80] x 2, dL/dd [N, 16]; the padded output
    // layer's weight gradient [16, 256] (fp32)
    z.scratch = (size_t)N * (2 * kWidth + 2 * kInPad + kOutPad) * sizeof(__nv_bfloat16) +
                kOutPad * kWidth * sizeof(float);
    z.out = (size_t)N * kOutPad * sizeof(float);
    // the bfloat16 parameters, then (16-byte aligned) the padded [16, 256] output layer
    z.theta16 = (size_t)(head16_offset() + kOutPad * kWidth) * sizeof(__nv_bfloat16);
    return z;
}

namespace {
// activation buffer: x5 [N, 336] then h0..h3, h5..h7 [N, 256] each
__nv_bfloat16* act_x5(void* act) { return static_cast<__nv_bfloat16*>(act); }
__nv_bfloat16* act_h(void* act, int64_t N, int l) {
    const int slot = l < 4 ? l : l - 1;  // h0..h3 -> 0..3, h5..h7 -> 4..6 (h4 lives in x5)
    return act_x5(act) + (size_t)N * kX5 + (size_t)slot * N * kWidth;
}
// ReLU bit-mask of hidden layer l, written by its forward product: bit m + 256 n is set when
// activation m of row n is positive (row n's 256 bits are bytes 32 n .. 32 n + 31)
uint8_t* act_mask(void* act, int64_t N, int l) {
    return reinterpret_cast<uint8_t*>(act_x5(act) + (size_t)N * (kX5 + 7 * kWidth)) + (size_t)l * mask_bytes(N);
}
}  // namespace

std::string mlp_forward(MlpLt& lt, const float* params3, int64_t N, float t, const float* theta, void* theta16_buf,
                        void* act, float* d, float* params_out, cudaStream_t s) {
    if (N == 0) return "";
    __nv_bfloat16* w16 = static_cast<__nv_bfloat16*>(theta16_buf);
    const int64_t P = mlp_param_count();
    launch_pdl(k_to_bf16, (unsigned)std::min<int64_t>(ceil_div(P, 256), 1024), 256, 0, s, theta, w16, P);
    launch_pdl(k_mlp_head16, 1u, kWidth, 0, s, theta + layer_offset(kHidden), w16 + head16_offset());
    count_launches(2);
    __nv_bfloat16* x5 = act_x5(act);
    launch_pdl(k_mlp_encode, ceil_div(N * kInPad, 256), 256, 0, s, params3, N, t, x5);
    count_launches(1);
    for (int l = 0; l <= kHidden; ++l) {
        // input: the encoding (layer 0, the first 80 columns of x5), (gamma, h4) (layer 5, all of
        // x5), else the previous layer's output; layer 4 writes h4 into columns 80.. of x5
        const void* x = (l == 0 || l == kSkipLayer) ? (const void*)x5 : (const void*)act_h(act, N, l - 1);
        const int ldx = (l == 0 || l == kSkipLayer) ? kX5 : kWidth;
        void* y = l == kHidden ? (void*)d : (l == 4 ? (void*)(x5 + kInPad) : (void*)act_h(act, N, l));
        const int ldy = l == kHidden ? kOutPad : (l == 4 ? kX5 : kWidth);
        const int64_t boff = layer_offset(l) + (int64_t)kShapes[l].out * kShapes[l].in;
        const __nv_bfloat16* wl = l == kHidden ? w16 + head16_offset() : w16 + layer_offset(l);
        const std::string e =
            layer_forward(lt, l, wl, w16 + boff, x, ldx, y, ldy, N, l == kHidden ? nullptr : act_mask(act, N, l), s);
        if (!e.empty()) return e;
    }
    const float* b_head = theta + layer_offset(kHidden) + (int64_t)kOut * kWidth;
    if (((reinterpret_cast<uintptr_t>(params3) | reinterpret_cast<uintptr_t>(params_out)) & 15u) == 0)
        launch_pdl(k_mlp_apply<true>, ceil_div(N, 256), 256, 0, s, params3, N, d, b_head, params_out);
    else
        launch_pdl(k_mlp_apply<false>, ceil_div(N, 256), 256, 0, s, params3, N, d, b_head, params_out);
    count_launches(1);
    return "";
}

std::string mlp_backward(MlpLt& lt, const float* params3, int64_t N, const void* theta16_buf, const void* act,
                         const float* d, void* scratch, const float* g_out, float* g_theta, float* g_params3,
                         int accumulate, cudaStream_t s) {
    if (N == 0) return "";
    const __nv_bfloat16* w16 = static_cast<const __nv_bfloat16*>(theta16_buf);
    const __nv_bfloat16* whead16 = w16 + head16_offset();  // [16, 256], rows 13..15 zero
    void* actm = const_cast<void*>(act);
    const __nv_bfloat16* x5 = act_x5(actm);
    // scratch layout (see mlp_sizes)
    __nv_bfloat16* dh = static_cast<__nv_bfloat16*>(scratch);  // [N, 256] before the ReLU mask
    __nv_bfloat16* dz = dh + (size_t)N * kWidth;                // [N, 256] after it
    __nv_bfloat16* dg0 = dz + (size_t)N * kWidth;               // [N, 80] through layer 0
    __nv_bfloat16* dgs = dg0 + (size_t)N * kInPad;              // [N, 80] through the skip input of layer 5
    __nv_bfloat16* gd = dgs + (size_t)N * kInPad;               // [N, 16]
    float* dw_head16 = reinterpret_cast<float*>(gd + (size_t)N * kOutPad);  // [16, 256]
    if (!accumulate) cudaMemsetAsync(g_theta, 0, sizeof(float) * (size_t)mlp_param_count(), s);
    float* db_head = g_theta + layer_offset(kHidden) + (int64_t)kOut * kWidth;
    const uintptr_t rows = reinterpret_cast<uintptr_t>(params3) | reinterpret_cast<uintptr_t>(g_out) |
                           reinterpret_cast<uintptr_t>(g_params3);
    if ((rows & 15u) == 0)
        launch_pdl(k_mlp_apply_backward<true>, ceil_div(N, 256), 256, 0, s, params3, N, d, g_out, gd, g_params3,
                   accumulate, db_head);
    else
        launch_pdl(k_mlp_apply_backward<false>, ceil_div(N, 256), 256, 0, s, params3, N, d, g_out, gd, g_params3,
                   accumulate, db_head);
    count_launches(1);
    std::string e;
    // output layer (padded to 16 rows): dW_8 = gd^T h7 into [16, 256]; dh7 = gd W_8
    e = gemm(lt, false, true, kWidth, kOutPad, (int)N, act_h(actm, N, 7), kWidth, gd, kOutPad, dw_head16, kWidth,
             CUDA_R_32F, 0.f, CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
    if (!e.empty()) return e;
    e = gemm(lt, false, false, kWidth, (int)N, kOutPad, whead16, kWidth, gd, kOutPad, dh, kWidth, CUDA_R_16BF, 0.f,
             CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
    if (!e.empty()) return e;
    for (int l = kHidden - 1; l >= 0; --l) {
        const LayerShape sh = kShapes[l];
        const __nv_bfloat16* wl = w16 + layer_offset(l);
        float* gb = g_theta + layer_offset(l) + (int64_t)sh.out * sh.in;
        launch_pdl(k_relu_backward, (unsigned)std::min<int64_t>(kReluBlocks, ceil_div(N, 8)), 256, 0, s,
                   (const __nv_bfloat16*)dh, kWidth, (const uint8_t*)act_mask(actm, N, l), N, dz, gb);
        count_launches(1);
        // dW_l += dz_l^T x_l  (column-major [in, out] = x^T (in x N) dz (N x out))
        const void* xin = (l == 0 || l == kSkipLayer) ? (const void*)x5 : (const void*)act_h(actm, N, l - 1);
        const int ldx = (l == 0 || l == kSkipLayer) ? kX5 : kWidth;
        e = gemm(lt, false, true, sh.in, sh.out, (int)N, xin, ldx, dz, kWidth, g_theta + layer_offset(l), sh.in,
                 CUDA_R_32F, 1.f, CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
        if (!e.empty()) return e;
        // input gradient dz_l W_l (W_l row-major [out, in] = column-major [in, out]) into dh for layer
        // l - 1; layer 5 splits it into the encoding's part and h4's, layer 0 has only the encoding's
        if (l == 0) {
            e = gemm(lt, false, false, kInPad, (int)N, kWidth, wl, kInPad, dz, kWidth, dg0, kInPad, CUDA_R_16BF, 0.f,
                     CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
        } else if (l == kSkipLayer) {
            e = gemm(lt, false, false, kInPad, (int)N, kWidth, wl, kX5, dz, kWidth, dgs, kInPad, CUDA_R_16BF, 0.f,
                     CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
            if (!e.empty()) return e;
            e = gemm(lt, false, false, kWidth, (int)N, kWidth, wl + kInPad, kX5, dz, kWidth, dh, kWidth, CUDA_R_16BF,
                     0.f, CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
        } else {
            e = gemm(lt, false, false, kWidth, (int)N, kWidth, wl, kWidth, dz, kWidth, dh, kWidth, CUDA_R_16BF, 0.f,
                     CUBLASLT_EPILOGUE_DEFAULT, nullptr, s);
        }
        if (!e.empty()) return e;
    }
    launch_pdl(k_mlp_add_head_dw, 1u, kWidth, 0, s, (const float*)dw_head16, g_theta, layer_offset(kHidden));
    launch_pdl(k_mlp_encode_backward, ceil_div(N, 256), 256, 0, s, params3, N, (const __nv_bfloat16*)dg0,
               (const __nv_bfloat16*)dgs, g_params3);
    count_launches(2);
    return "";
}

}  // namespace wipes
