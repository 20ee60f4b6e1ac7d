// Mean squared error and its gradient without any device allocation.
//
// Some callers cannot call cudaMalloc: code running under an allocator that owns all device
// memory (a framework's caching allocator or a fixed arena), and embedded hosts that forbid
// device allocation after start-up.  This entry point serves them: its only scratch is the file-scope array below,
// part of the library's device image, so every GPU that loads the library holds it (256 KB) until
// the process exits.
//
// The array is shared by every call on a device and keeps the last call's contents.  Each call
// writes every partial sum it later reads, so nothing in it has to start at zero; two calls that
// overlap on the GPU (different streams, no ordering between them) race on it.  The array belongs
// to this process's copy of the library on each device: other processes have their own.
#include <mutex>

#include "common.cuh"

namespace wipes {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItems = 16;                                   // elements per thread
constexpr int64_t kNoAllocBlockElems = kNoAllocThreads * kNoAllocItems;  // 4096 per block
constexpr int kNoAllocMaxBlocks = 65536;                            // scratch: one float per block
constexpr int64_t kNoAllocMaxElems = kNoAllocBlockElems * kNoAllocMaxBlocks;  // 268,435,456

static __device__ __align__(256) float g_loss_scratch[kNoAllocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
float* g_scratch_ptr[kMaxDevices] = {};

// One partial sum of squared differences per block; grad = 2 (img - target) / n.
__global__ void __launch_bounds__(kNoAllocThreads) k_l2_loss_blocks(const float* __restrict__ img,
                                                                    const float* __restrict__ target, int64_t n,
                                                                    float* __restrict__ grad,
                                                                    float* __restrict__ partials) {
    pdl_enter();
    __shared__ float s_warp[kNoAllocThreads / 32];
    const float scale = 2.0f / (float)n;
    const int64_t base = (int64_t)blockIdx.x * kNoAllocBlockElems + threadIdx.x;
    float acc = 0.f;
#pragma unroll 4
    for (int k = 0; k < kNoAllocItems; ++k) {
        const int64_t i = base + (int64_t)k * kNoAllocThreads;
        if (i < n) {
            const float d = img[i] - target[i];
            grad[i] = scale * d;
            acc = fmaf(d, d, acc);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) s += s_warp[w];
        partials[blockIdx.x] = s;
    }
}

// Sum the block partials in a fixed order (binary64 accumulation) and divide by n.
__global__ void __launch_bounds__(kNoAllocThreads) k_l2_loss_total(const float* __restrict__ partials, int nb,
                                                                   int64_t n, float* __restrict__ loss) {
    pdl_enter();
    __shared__ double s[kNoAllocThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kNoAllocThreads) acc += partials[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(s[0] / (double)n);
}

// Device address of the scratch array for the current device.  Host code cannot use the array's
// name as a device address; cudaGetSymbolAddress gives the address in the context that is current.
// Outside stream capture it is looked up on every call, so a reset device (whose library image
// may load elsewhere) or another current context never leaves a stale address behind; while
// `stream` is capturing, the address from the last call outside capture on this device is used, and
// a device with none yet returns cudaErrorStreamCaptureUnsupported.
cudaError_t scratch_for_current_device(cudaStream_t stream, float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> guard(g_setup_lock);
    if (cap == cudaStreamCaptureStatusNone) {
        float* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_loss_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

int64_t l2_loss_noalloc_max_elements() { return kNoAllocMaxElems; }

cudaError_t l2_loss_noalloc(const float* img, const float* target, int64_t n, float* loss, float* grad,
                            cudaStream_t stream) {
    float* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(stream, &scratch);
    if (e != cudaSuccess) return e;
    const int nb = (int)ceil_div(n, kNoAllocBlockElems);
    // this call's own launch results: an error left behind by unrelated earlier work stays for
    // its owner to read
    e = launch_pdl(k_l2_loss_blocks, nb, kNoAllocThreads, 0, stream, img, target, n, grad, scratch);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_l2_loss_total, 1, kNoAllocThreads, 0, stream, scratch, nb, n, loss);
    count_launches(2);
    return e;
}

}  // namespace wipes
