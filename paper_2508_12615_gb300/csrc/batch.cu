// Batched forward rasterization: the tiles of many prepared frames (2D or 3D, any primitive count
// and image size) in one persistent launch.  Every block loops: it takes the next (frame, tile)
// item from a device counter, renders that tile with the same per-tile function as the one-frame
// kernels, and stops when the items run out.  Short frames do not leave the GPU idle while long
// ones finish, and one launch replaces one launch per frame.
#include "blend_tile.cuh"

namespace wipes {
namespace {

struct BatchTable {
    int n_jobs;
    unsigned int start[kMaxBatchJobs + 1];  // first item of each frame; start[n_jobs] = all items
    BlendJob jobs[kMaxBatchJobs];
};

__global__ void __launch_bounds__(kTilePixels) k_blend_batch(const __grid_constant__ BatchTable table,
                                                             unsigned int* __restrict__ counter) {
    pdl_enter();
    __shared__ unsigned int s_item;
    __shared__ int s_job;
    const unsigned int total = table.start[table.n_jobs];
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int item = atomicAdd(counter, 1u);
            int lo = 0, hi = table.n_jobs;  // largest j with start[j] <= item
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (table.start[mid] <= item) lo = mid;
                else hi = mid;
            }
            s_item = item;
            s_job = lo;
        }
        __syncthreads();
        const unsigned int item = s_item;
        const int j = s_job;
        __syncthreads();  // every thread has read the item before thread 0 takes the next one
        if (item >= total) break;
        const BlendJob& job = table.jobs[j];
        const int tile = (int)(item - table.start[j]);
        if (job.dims == 2) blend2d_tile(job, tile);
        else blend3d_tile(job, tile);
    }
}

}  // namespace

void launch_blend_batch(const BlendJob* jobs, const int* tiles_y, int n_jobs, unsigned int* counter,
                        cudaStream_t stream) {
    BatchTable t;
    t.n_jobs = n_jobs;
    unsigned int s = 0;
    for (int j = 0; j < n_jobs; ++j) {
        t.start[j] = s;
        t.jobs[j] = jobs[j];
        s += (unsigned int)(jobs[j].tiles_x * tiles_y[j]);
    }
    t.start[n_jobs] = s;
    if (s == 0) return;
    cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_blend_batch, kTilePixels, 0);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>((long long)std::max(1, per_sm) * std::max(1, sms), s);
    launch_pdl(k_blend_batch, grid, kTilePixels, 0, stream, t, counter);
    count_launches(1);
}

}  // namespace wipes
