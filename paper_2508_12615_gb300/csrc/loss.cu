// Mean squared error and its gradient in one pass (deterministic two-stage reduction).
#include "common.cuh"

namespace wipes {
namespace {

__global__ void __launch_bounds__(256) k_l2_loss(const float* __restrict__ img, const float* __restrict__ target,
                                                 int64_t n, float* __restrict__ grad, float* __restrict__ partials) {
    pdl_enter();
    __shared__ float s_warp[8];
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
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += s_warp[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_l2_finish(const float* __restrict__ partials, int nb, int64_t n, float* __restrict__ loss) {
    pdl_enter();
    __shared__ double s[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) acc += partials[i];
    s[threadIdx.x] = acc;
    __syncwarp();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 32; ++i) t += s[i];
        *loss = (float)(t / (double)n);
    }
}

}  // namespace

void launch_l2_loss(const float* img, const float* target, int64_t n, float* loss, float* grad, float* partials,
                    cudaStream_t stream) {
    const int nb = (int)std::min<int64_t>(kLossBlocks, std::max<int64_t>(1, ceil_div(n, 256)));
    launch_pdl(k_l2_loss, nb, 256, 0, stream, img, target, n, grad, partials); count_launches(1);
    launch_pdl(k_l2_finish, 1, 32, 0, stream, partials, nb, n, loss); count_launches(1);
}

}  // namespace wipes
