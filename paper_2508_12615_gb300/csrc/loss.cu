// Mean squared error and its gradient in one pass (deterministic two-stage reduction).
#include "common.cuh"

namespace wipes {
namespace {

// One launch: every block adds the squared differences of its grid-stride share and writes the
// gradient; the last block to finish (a counter after the partials) sums the block partials in a
// fixed order in binary64, writes the loss and puts the counter back to zero.
__global__ void __launch_bounds__(256) k_l2_loss(const float* __restrict__ img, const float* __restrict__ target,
                                                 int64_t n, float* __restrict__ grad, float* __restrict__ partials,
                                                 float* __restrict__ loss) {
    pdl_enter();
    __shared__ float s_warp[8];
    __shared__ double s_sum[256];
    __shared__ bool s_last;
    const float scale = 2.0f / (float)n;
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;  // elements handled four at a time
    const uintptr_t ptrs = reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(target) |
                           reinterpret_cast<uintptr_t>(grad);
    if ((ptrs & 15u) == 0) {
        const int64_t n4 = n >> 2;
        for (int64_t i = first; i < n4; i += stride) {
            const float4 a = reinterpret_cast<const float4*>(img)[i];
            const float4 t = reinterpret_cast<const float4*>(target)[i];
            const float4 d = make_float4(a.x - t.x, a.y - t.y, a.z - t.z, a.w - t.w);
            reinterpret_cast<float4*>(grad)[i] = make_float4(scale * d.x, scale * d.y, scale * d.z, scale * d.w);
            acc = fmaf(d.x, d.x, acc);
            acc = fmaf(d.y, d.y, acc);
            acc = fmaf(d.z, d.z, acc);
            acc = fmaf(d.w, d.w, acc);
        }
        done = n4 << 2;
    }
    for (int64_t i = done + first; i < n; i += stride) {
        const float d = img[i] - target[i];
        grad[i] = scale * d;
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    unsigned int* counter = reinterpret_cast<unsigned int*>(partials + kLossBlocks);
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += s_warp[w];
        partials[blockIdx.x] = s;
        __threadfence();  // the partial is visible before the count says so
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nb = (int)gridDim.x;
    double t = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) t += (double)__ldcg(partials + i);
    s_sum[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *loss = (float)(s_sum[0] / (double)n);
        *counter = 0u;
    }
}

}  // namespace

void launch_l2_loss(const float* img, const float* target, int64_t n, float* loss, float* grad, float* partials,
                    cudaStream_t stream) {
    const int nb = (int)std::min<int64_t>(kLossBlocks, std::max<int64_t>(1, ceil_div(n, 256)));
    launch_pdl(k_l2_loss, nb, 256, 0, stream, img, target, n, grad, partials, loss);
    count_launches(1);
}

}  // namespace wipes
