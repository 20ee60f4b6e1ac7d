// C ABI of the wavelet rasterizer: contexts, workspaces (states) and the orchestration of the
// forward and backward passes.  Every numeric step runs in the kernels of footprint.cu,
// binning.cu, raster2d.cu, raster3d.cu and loss.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>
#include <string>

#include <mutex>

#include "common.cuh"

using namespace wipes;

namespace {

thread_local std::string g_last_error;

wipes_status fail(wipes_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define WIPES_CUDA(call)                                                                                  \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? WIPES_ERR_OOM : WIPES_ERR_CUDA,                \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

#define WIPES_TRY(expr)                   \
    do {                                  \
        wipes_status s_ = (expr);         \
        if (s_ != WIPES_OK) return s_;    \
    } while (0)

// Device bytes held by the workspaces of one context, and the optional limit on them.
struct MemAccount {
    std::atomic<int64_t> reserved{0};
    std::atomic<int64_t> limit{0};  // 0: no limit
    cudaMemPool_t pool = nullptr;   // stream-ordered pool of the context's workspace buffers
};

// Workspace buffers come from the context's memory pool in stream order, on the stream of the call
// that grows them (set by AllocStream at the entry points): a new state costs no cudaMalloc.
// Frees wait for the whole device first, as cudaFree does, because a buffer may be in use by work
// on any stream.
thread_local cudaStream_t t_alloc_stream = nullptr;
struct AllocStream {
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
    ~AllocStream() { t_alloc_stream = prev; }
};

// Grow-only device buffer, accounted to its context.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    MemAccount* acct = nullptr;
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

void free_buf(DevBuf& b, bool device_idle = false) {
    if (b.p) {
        if (b.acct && b.acct->pool) {
            if (!device_idle) cudaDeviceSynchronize();
            cudaFreeAsync(b.p, nullptr);
        } else {
            cudaFree(b.p);
        }
    }
    if (b.acct) b.acct->reserved -= (int64_t)b.cap;
    b.p = nullptr;
    b.cap = 0;
}

wipes_status ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return WIPES_OK;
    size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    const int64_t limit = b.acct ? b.acct->limit.load() : 0;
    if (limit > 0 && b.acct->reserved.load() - (int64_t)b.cap + (int64_t)want > limit) {
        // a tighter request that still fits the limit is taken without headroom
        want = bytes;
        if (b.acct->reserved.load() - (int64_t)b.cap + (int64_t)want > limit)
            return fail(WIPES_ERR_OOM, "workspace memory limit of " + std::to_string(limit) + " bytes reached (" +
                                           std::to_string(b.acct->reserved.load()) + " reserved, " +
                                           std::to_string(want) + " more wanted)");
    }
    free_buf(b);
    cudaError_t e = b.acct && b.acct->pool ? cudaMallocFromPoolAsync(&b.p, want, b.acct->pool, t_alloc_stream)
                                           : cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(WIPES_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed: " + cudaGetErrorString(e));
    }
    b.cap = want;
    if (b.acct) b.acct->reserved += (int64_t)want;
    return WIPES_OK;
}

void release(DevBuf& b, bool device_idle = false) { free_buf(b, device_idle); }

int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

std::atomic<int64_t> g_launches{0};

// Batch launches in flight on one context use distinct work counters, taken round-robin.
constexpr unsigned int kBatchCounterSlots = 64;

}  // namespace

void wipes::count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct wipes_ctx {
    int device = 0;
    MemAccount mem;
    std::atomic<int64_t> live_states{0};  // a context is not destroyed while states refer to it
    unsigned long long* h_total = nullptr;  // pinned readback: [0] instance count, [1] device error word
    unsigned long long* d_readback = nullptr;  // h_total's device address (mapped pinned memory)
    cudaEvent_t scan_done = nullptr;           // recorded after the scan writes h_total; the host waits on it
    unsigned int* d_error = nullptr;        // device error word: bit 0 = a bounded device wait ran out
    float* d_loss_partials = nullptr;
    unsigned long long* d_counters = nullptr;  // pair counters
    unsigned int* d_batch_counters = nullptr;  // work counters of in-flight batch launches (a ring)
    unsigned int batch_slot = 0;
    // stage timing
    bool timing = false;
    struct Bracket {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Bracket> pending;
    std::vector<cudaEvent_t> free_events;
    double stage_ms[WIPES_STAGE_COUNT] = {};
    int64_t stage_n[WIPES_STAGE_COUNT] = {};

    cudaEvent_t take_event() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

namespace {

// Brackets one stage with CUDA events on `s` when timing is enabled on the context.
struct StageTimer {
    wipes_ctx* ctx;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(wipes_ctx* c, int st, cudaStream_t stream) : ctx(c), stage(st), s(stream) {
        if (ctx && ctx->timing) {
            a = ctx->take_event();
            cudaEventRecord(a, s);
        }
    }
    void stop() {
        if (!a) return;
        cudaEvent_t b = ctx->take_event();
        cudaEventRecord(b, s);
        ctx->pending.push_back({stage, a, b});
        a = nullptr;
    }
    ~StageTimer() { stop(); }
};

}  // namespace

struct wipes_state {
    wipes_ctx* ctx = nullptr;
    int dims = 0;
    int64_t N = 0;
    int H = 0, W = 0, tiles_x = 0, tiles_y = 0;
    wipes_opts opts{};
    wipes_camera cam{};
    int64_t n_inst = 0;
    int sorted = 0;  // which ping-pong buffer holds the sorted lists
    DevBuf rec, rect, counts, offsets, dkeys[2], dvals[2], block_sums, total, keys[2], vals[2], inst_prim, hist, ranges;
    DevBuf sprim, order, T_final, last, partial, grad_img;
    DevBuf mlp_act, mlp_scratch, mlp_d, mlp_theta16;  // deformation network: activations kept for the backward
    int64_t mlp_N = -1;                               // primitives of the last network forward (-1: none)
    DevBuf sort_k, sort_v;                            // second buffers of wipes_sort_pairs
    // 3D backward in chunks: its items (tile, chunk), each tile's first item, the item count, and
    // the pixels' state at chunk boundaries and final colour recorded by the one-frame forward
    DevBuf bwd_items, item_base, n_items, bnd, cfin;
    int64_t max_items = 0;
    bool bnd_valid = false;  // the last forward on this state recorded bnd and cfin

    DevBuf* all[34] = {&rec,     &rect,    &counts,    &offsets, &dkeys[0], &dkeys[1], &dvals[0], &dvals[1],
                       &block_sums, &total, &keys[0], &keys[1],   &vals[0],   &vals[1],   &inst_prim, &hist,
                       &ranges,  &sprim,   &order,     &T_final, &last,     &partial,  &grad_img, &mlp_act,
                       &mlp_scratch, &mlp_d, &mlp_theta16, &sort_k, &sort_v, &bwd_items, &item_base,
                       &n_items,  &bnd,     &cfin};
    size_t reserved() const {
        size_t s = 0;
        for (DevBuf* b : all) s += b->cap;
        return s;
    }
    TileLists lists() const {
        TileLists t;
        t.sorted = vals[sorted].as<uint32_t>();
        t.prim = sprim.as<uint32_t>();
        t.ranges = ranges.as<uint2>();
        return t;
    }
    BlendJob job(float* out) const;
};

namespace {

wipes_status check_image(int H, int W) {
    if (H < 1 || W < 1 || H > 16384 || W > 16384)
        return fail(WIPES_ERR_INVALID, "image size must be within 1..16384 (got H=" + std::to_string(H) +
                                           ", W=" + std::to_string(W) + ")");
    return WIPES_OK;
}

// The device error word as last read back into h_total[1]: a set bit is reported once and cleared.
wipes_status take_device_error(wipes_ctx* ctx, cudaStream_t s) {
    if (ctx->h_total[1] == 0) return WIPES_OK;
    const unsigned long long bits = ctx->h_total[1];
    ctx->h_total[1] = 0;
    WIPES_CUDA(cudaMemsetAsync(ctx->d_error, 0, sizeof(unsigned long long), s));
    std::string where = (bits & 1u) ? "radix sort look-back" : "";
    if (bits & 2u) where += std::string(where.empty() ? "" : ", ") + "deformation network pipeline";
    return fail(WIPES_ERR_TIMEOUT, "a bounded device wait ran out (" + where + "); results of the calls since the "
                                   "last check are undefined");
}

// Scan the per-primitive tile counts (in `perm` order when given), read the instance total back,
// size the instance buffers, emit the pairs and sort them by tile (stable).
wipes_status bin_and_sort(wipes_state* st, const uint32_t* perm, cudaStream_t s) {
    const int64_t N = st->N;
    const int nb = (int)std::max<int64_t>(1, ceil_div(N, kScanBlockElems));
    WIPES_TRY(ensure(st->block_sums, sizeof(unsigned long long) * (size_t)nb));
    WIPES_TRY(ensure(st->total, sizeof(unsigned long long)));
    const int n_tiles = st->tiles_x * st->tiles_y;
    WIPES_TRY(ensure(st->ranges, sizeof(uint2) * (size_t)n_tiles));
    unsigned long long* total = st->total.as<unsigned long long>();
    // Emission is enqueued before the host waits for the instance total, into the list buffers as
    // they are, so that the GPU runs it while the host wakes up.  It writes nothing when the total
    // exceeds their capacity (a state's first call, or lists that grew) and is launched again below,
    // once they have grown.
    auto capacity = [&]() {
        return (int64_t)(std::min({st->keys[0].cap, st->vals[0].cap, st->inst_prim.cap}) / sizeof(uint32_t));
    };
    auto emit = [&]() {
        StageTimer t(st->ctx, WIPES_STAGE_EMIT, s);
        launch_emit(st->counts.as<uint32_t>(), perm, N, st->rec.as<float4>(), st->rect.as<PixRect>(),
                    st->block_sums.as<unsigned long long>(), total, capacity(), st->tiles_x,
                    touch_limit(st->opts.cutoff_sigma), st->keys[0].as<uint32_t>(), st->vals[0].as<uint32_t>(),
                    st->inst_prim.as<uint32_t>(), st->offsets.as<uint32_t>(), st->ranges.as<uint2>(), n_tiles, s);
    };
    const int64_t emitted_capacity = capacity();
    if (N > 0) {
        {
            StageTimer t(st->ctx, WIPES_STAGE_SCAN, s);
            launch_block_sums(st->counts.as<uint32_t>(), perm, N, st->block_sums.as<unsigned long long>(), s);
            launch_scan_block_sums(st->block_sums.as<unsigned long long>(), nb, total,
                                   reinterpret_cast<const unsigned long long*>(st->ctx->d_error), st->ctx->d_readback,
                                   s);
            WIPES_CUDA(cudaEventRecord(st->ctx->scan_done, s));
        }
        emit();
        WIPES_CUDA(cudaEventSynchronize(st->ctx->scan_done));
        st->n_inst = (int64_t)st->ctx->h_total[0];
        WIPES_TRY(take_device_error(st->ctx, s));
    } else {
        st->n_inst = 0;
    }
    if (st->n_inst > (int64_t)INT32_MAX)
        return fail(WIPES_ERR_CAPACITY, "tile instance count " + std::to_string(st->n_inst) + " exceeds 2^31-1");
    const int64_t I = st->n_inst;
    for (int k = 0; k < 2; ++k) {
        WIPES_TRY(ensure(st->keys[k], sizeof(uint32_t) * (size_t)std::max<int64_t>(I, 1)));
        WIPES_TRY(ensure(st->vals[k], sizeof(uint32_t) * (size_t)std::max<int64_t>(I, 1)));
    }
    WIPES_TRY(ensure(st->inst_prim, sizeof(uint32_t) * (size_t)std::max<int64_t>(I, 1)));
    WIPES_TRY(ensure(st->sprim, sizeof(uint32_t) * (size_t)std::max<int64_t>(I, 1)));
    WIPES_TRY(ensure(st->hist, sizeof(uint32_t) * (size_t)radix_hist_words(I)));
    if (N > 0 && I > emitted_capacity) emit();  // the first launch wrote nothing
    uint32_t* kb[2] = {st->keys[0].as<uint32_t>(), st->keys[1].as<uint32_t>()};
    uint32_t* vb[2] = {st->vals[0].as<uint32_t>(), st->vals[1].as<uint32_t>()};
    {
        StageTimer t(st->ctx, WIPES_STAGE_TILE_SORT, s);
        st->sorted = radix_sort_pairs(kb, vb, I, ceil_log2(n_tiles), st->hist.as<uint32_t>(), st->ctx->d_error, s,
                                      st->inst_prim.as<uint32_t>(), st->sprim.as<uint32_t>());
    }
    {
        StageTimer t(st->ctx, WIPES_STAGE_RANGES, s);
        launch_tile_ranges(kb[st->sorted], I, st->ranges.as<uint2>(), n_tiles, /*zeroed=*/N > 0, s);
    }
    return WIPES_OK;
}

wipes_status prepare_state(wipes_state* st, int dims, int64_t N, int H, int W, const wipes_opts* opts) {
    st->dims = 0;  // invalid until the forward pass is enqueued
    st->N = N;
    st->H = H;
    st->W = W;
    st->tiles_x = (W + kTile - 1) / kTile;
    st->tiles_y = (H + kTile - 1) / kTile;
    st->opts = *opts;
    const size_t n = (size_t)std::max<int64_t>(N, 1);
    WIPES_TRY(ensure(st->rec, sizeof(float4) * kRecF4 * n));
    WIPES_TRY(ensure(st->rect, sizeof(PixRect) * n));
    WIPES_TRY(ensure(st->counts, sizeof(uint32_t) * n));
    WIPES_TRY(ensure(st->offsets, sizeof(uint32_t) * n));
    (void)dims;
    return WIPES_OK;
}

BlendOpts3 blend_opts(const wipes_opts& o);

}  // namespace

BlendJob wipes_state::job(float* out) const {
    BlendJob j;
    j.rec = rec.as<float4>();
    j.rect = rect.as<PixRect>();
    j.tl = lists();
    j.out = out;
    j.T_final = T_final.as<float>();
    j.last = last.as<uint32_t>();
    j.dims = dims;
    j.W = W;
    j.H = H;
    j.tiles_x = tiles_x;
    j.o = blend_opts(opts);
    return j;
}

namespace {

BlendOpts3 blend_opts(const wipes_opts& o) {
    BlendOpts3 b;
    b.cutoff2 = o.cutoff_sigma * o.cutoff_sigma;
    b.lim = touch_limit(o.cutoff_sigma);
    b.alpha_min = o.alpha_min;
    b.alpha_max = o.alpha_max;
    b.T_min = o.T_min;
    b.bg[0] = o.bg[0];
    b.bg[1] = o.bg[1];
    b.bg[2] = o.bg[2];
    b.damp = o.freq_proj_mode == 2;
    b.cut_scale = cutoff_scale(b.cutoff2);
    return b;
}

wipes_status check_opts(const wipes_opts* o) {
    if (!o) return fail(WIPES_ERR_INVALID, "opts is NULL");
    if (!(o->cutoff_sigma >= 0x1p-10f && o->cutoff_sigma <= 0x1p10f))
        return fail(WIPES_ERR_INVALID, "cutoff_sigma must lie in [2^-10, 2^10]");
    if (!(o->alpha_max > 0.f && o->alpha_max < 1.f))
        return fail(WIPES_ERR_INVALID, "alpha_max must lie in (0, 1)");
    if (!(o->alpha_min >= 0.f) || !(o->T_min >= 0.f) || !(o->dilation >= 0.f))
        return fail(WIPES_ERR_INVALID, "alpha_min, T_min and dilation must be non-negative");
    if (o->freq_proj_mode < 0 || o->freq_proj_mode > 2)
        return fail(WIPES_ERR_INVALID,
                    "freq_proj_mode must be 0 (fronto-parallel phase gradient), 1 (literal J W f) or 2 (integrated "
                    "along the viewing ray)");
    if (o->cov2d != 0 && o->cov2d != 1) return fail(WIPES_ERR_INVALID, "cov2d must be 0 (RS) or 1 (Cholesky)");
    if (o->sh_degree < 0 || o->sh_degree > 3) return fail(WIPES_ERR_INVALID, "sh_degree must lie in 0..3");
    return WIPES_OK;
}

}  // namespace

extern "C" {

void wipes_default_opts(int dims, wipes_opts* out) {
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->cutoff_sigma = 3.0f;
    out->alpha_min = 1.0f / 255.0f;
    out->alpha_max = 0.99f;
    out->T_min = 1e-4f;
    out->dilation = dims == 3 ? 0.3f : 0.0f;
}

wipes_status wipes_create(int device, wipes_ctx** out) {
    if (!out) return fail(WIPES_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int n = 0;
    WIPES_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(WIPES_ERR_INVALID, "no CUDA device " + std::to_string(device));
    DeviceGuard g(device);
    wipes_ctx* c = new wipes_ctx();
    c->device = device;
    cudaError_t e = cudaMallocHost(&c->h_total, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->d_readback, c->h_total, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->scan_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_error, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_error, 0, sizeof(unsigned long long));
    // the loss's block partials and, after them, its block counter (zero between calls)
    if (e == cudaSuccess) e = cudaMalloc(&c->d_loss_partials, sizeof(float) * (kLossBlocks + 1));
    if (e == cudaSuccess) e = cudaMemset(c->d_loss_partials + kLossBlocks, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_batch_counters, sizeof(unsigned int) * kBatchCounterSlots);
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&c->mem.pool, &props);
        // keep freed workspace for reuse instead of returning it to the driver at every sync (a
        // trim of many GB stalls the device); the pool holds at most the largest workspace reached
        uint64_t keep = ~(uint64_t)0;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(c->mem.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        if (c->h_total) cudaFreeHost(c->h_total);
        if (c->scan_done) cudaEventDestroy(c->scan_done);
        if (c->mem.pool) cudaMemPoolDestroy(c->mem.pool);
        delete c;
        return fail(WIPES_ERR_CUDA, std::string("context allocation failed: ") + cudaGetErrorString(e));
    }
    *out = c;
    return WIPES_OK;
}

wipes_status wipes_destroy(wipes_ctx* ctx) {
    if (!ctx) return WIPES_OK;
    if (ctx->live_states.load() != 0)
        return fail(WIPES_ERR_INVALID, "wipes_destroy: " + std::to_string(ctx->live_states.load()) +
                                           " states of this context are still alive");
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& b : ctx->pending) {
        cudaEventDestroy(b.a);
        cudaEventDestroy(b.b);
    }
    for (cudaEvent_t e : ctx->free_events) cudaEventDestroy(e);
    cudaEventDestroy(ctx->scan_done);
    cudaFreeHost(ctx->h_total);
    cudaFree(ctx->d_loss_partials);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_error);
    cudaFree(ctx->d_batch_counters);
    if (ctx->mem.pool) cudaMemPoolDestroy(ctx->mem.pool);
    delete ctx;
    return WIPES_OK;
}

wipes_status wipes_state_create(wipes_ctx* ctx, wipes_state** out) {
    if (!ctx || !out) return fail(WIPES_ERR_INVALID, "ctx or out is NULL");
    wipes_state* st = new wipes_state();
    st->ctx = ctx;
    for (DevBuf* b : st->all) b->acct = &ctx->mem;
    ctx->live_states += 1;
    *out = st;
    return WIPES_OK;
}

wipes_status wipes_state_destroy(wipes_state* st) {
    if (!st) return WIPES_OK;
    wipes_ctx* ctx = st->ctx;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();  // once for all buffers of the state
        for (DevBuf* b : st->all) release(*b, true);
    }
    delete st;
    ctx->live_states -= 1;
    return WIPES_OK;
}

wipes_status wipes_prepare2d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, int H, int W,
                             const wipes_opts* opts, void* stream) {
    if (!ctx || !st || (N > 0 && !params)) return fail(WIPES_ERR_INVALID, "null argument");
    if (N < 0 || N > (int64_t)INT32_MAX) return fail(WIPES_ERR_INVALID, "N out of range");
    WIPES_TRY(check_image(H, W));
    WIPES_TRY(check_opts(opts));
    if (((uintptr_t)params & 15) != 0) return fail(WIPES_ERR_INVALID, "params must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    WIPES_TRY(prepare_state(st, 2, N, H, W, opts));
    {
        StageTimer t(ctx, WIPES_STAGE_FOOTPRINT, s);
        launch_footprint2d(params, N, W, H, opts->cutoff_sigma, opts->cov2d, st->rec.as<float4>(), st->rect.as<PixRect>(),
                           st->counts.as<uint32_t>(), nullptr, s);
    }
    WIPES_TRY(bin_and_sort(st, nullptr, s));
    WIPES_CUDA(cudaGetLastError());
    st->dims = 2;
    return WIPES_OK;
}

wipes_status wipes_render2d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, int H, int W,
                            const wipes_opts* opts, float* out, void* stream) {
    if (!out) return fail(WIPES_ERR_INVALID, "null argument");
    WIPES_TRY(wipes_prepare2d(ctx, st, params, N, H, W, opts, stream));
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    {
        StageTimer t(ctx, WIPES_STAGE_BLEND, s);
        launch_blend2d(st->job(out), st->tiles_y, s);
    }
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_prepare3d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, const wipes_camera* cam,
                             int H, int W, const wipes_opts* opts, void* stream) {
    if (!ctx || !st || !cam || (N > 0 && !params)) return fail(WIPES_ERR_INVALID, "null argument");
    if (N < 0 || N > (int64_t)INT32_MAX) return fail(WIPES_ERR_INVALID, "N out of range");
    WIPES_TRY(check_image(H, W));
    WIPES_TRY(check_opts(opts));
    if (((uintptr_t)params & 15) != 0) return fail(WIPES_ERR_INVALID, "params must be 16-byte aligned");
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !(cam->near_z > 0.f))
        return fail(WIPES_ERR_INVALID, "camera needs fx, fy, near_z > 0");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    WIPES_TRY(prepare_state(st, 3, N, H, W, opts));
    st->cam = *cam;
    const size_t n = (size_t)std::max<int64_t>(N, 1);
    for (int k = 0; k < 2; ++k) {
        WIPES_TRY(ensure(st->dkeys[k], sizeof(uint32_t) * n));
        WIPES_TRY(ensure(st->dvals[k], sizeof(uint32_t) * n));
    }
    WIPES_TRY(ensure(st->hist, sizeof(uint32_t) * (size_t)radix_hist_words(N)));
    const size_t npix = (size_t)H * (size_t)W;
    WIPES_TRY(ensure(st->T_final, sizeof(float) * npix));
    WIPES_TRY(ensure(st->last, sizeof(uint32_t) * npix));
    {
        StageTimer t(ctx, WIPES_STAGE_FOOTPRINT, s);
        launch_footprint3d(params, N, *cam, W, H, opts->cutoff_sigma, opts->dilation, opts->freq_proj_mode,
                           opts->sh_degree, st->rec.as<float4>(),
                           st->rect.as<PixRect>(), st->counts.as<uint32_t>(), st->dkeys[0].as<uint32_t>(), s);
    }
    // front-to-back order: stable sort of the primitives by the bits of their camera depth
    uint32_t* dk[2] = {st->dkeys[0].as<uint32_t>(), st->dkeys[1].as<uint32_t>()};
    uint32_t* dv[2] = {st->dvals[0].as<uint32_t>(), st->dvals[1].as<uint32_t>()};
    int cur = 0;
    {
        StageTimer t(ctx, WIPES_STAGE_DEPTH_SORT, s);
        launch_iota(st->dvals[0].as<uint32_t>(), N, s);
        cur = radix_sort_pairs(dk, dv, N, 32, st->hist.as<uint32_t>(), ctx->d_error, s);
    }
    WIPES_TRY(bin_and_sort(st, dv[cur], s));
    {
        StageTimer t(ctx, WIPES_STAGE_RANGES, s);
        const int n_tiles = st->tiles_x * st->tiles_y;
        WIPES_TRY(ensure(st->order, sizeof(uint32_t) * (size_t)n_tiles));
        // the backward's items: at most one per tile plus one per kBwdChunk instances
        st->max_items = n_tiles + (st->n_inst + kBwdChunk - 1) / kBwdChunk + 1;
        WIPES_TRY(ensure(st->bwd_items, sizeof(uint2) * (size_t)st->max_items));
        WIPES_TRY(ensure(st->item_base, sizeof(uint32_t) * (size_t)n_tiles));
        WIPES_TRY(ensure(st->n_items, 2 * sizeof(uint32_t)));  // item count, work counter
        launch_tile_order(st->ranges.as<uint2>(), n_tiles, st->order.as<uint32_t>(), st->bwd_items.as<uint2>(),
                          st->item_base.as<uint32_t>(), st->n_items.as<uint32_t>(), s);
    }
    WIPES_CUDA(cudaGetLastError());
    st->dims = 3;
    st->bnd_valid = false;  // until a one-frame forward over these lists records them
    return WIPES_OK;
}

wipes_status wipes_render3d(wipes_ctx* ctx, wipes_state* st, const float* params, int64_t N, const wipes_camera* cam,
                            int H, int W, const wipes_opts* opts, float* out, void* stream) {
    if (!out) return fail(WIPES_ERR_INVALID, "null argument");
    WIPES_TRY(wipes_prepare3d(ctx, st, params, N, cam, H, W, opts, stream));
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    WIPES_TRY(ensure(st->bnd, sizeof(float4) * kTilePixels * (size_t)st->max_items));
    WIPES_TRY(ensure(st->cfin, sizeof(float) * 3 * (size_t)H * (size_t)W));
    {
        StageTimer t(ctx, WIPES_STAGE_BLEND, s);
        BlendJob job = st->job(out);
        job.item_base = st->item_base.as<uint32_t>();
        job.bnd = st->bnd.as<float4>();
        job.cfin = st->cfin.as<float>();
        launch_blend3d(job, st->tiles_y, st->order.as<uint32_t>(), s);
    }
    WIPES_CUDA(cudaGetLastError());
    st->bnd_valid = true;
    return WIPES_OK;
}

wipes_status wipes_blend_batch(wipes_ctx* ctx, const wipes_state* const* states, float* const* outs, int n,
                               void* stream) {
    if (!ctx || n < 0 || (n > 0 && (!states || !outs))) return fail(WIPES_ERR_INVALID, "null argument");
    for (int i = 0; i < n; ++i) {
        if (!states[i] || !outs[i]) return fail(WIPES_ERR_INVALID, "null state or output in batch");
        if (states[i]->dims != 2 && states[i]->dims != 3)
            return fail(WIPES_ERR_INVALID, "batch entry " + std::to_string(i) + " holds no prepared frame");
        if (states[i]->ctx != ctx) return fail(WIPES_ERR_INVALID, "batch entry from another context");
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    StageTimer t(ctx, WIPES_STAGE_BLEND, s);
    BlendJob jobs[kMaxBatchJobs];
    int tiles_y[kMaxBatchJobs];
    for (int b0 = 0; b0 < n; b0 += kMaxBatchJobs) {
        const int m = std::min(kMaxBatchJobs, n - b0);
        for (int i = 0; i < m; ++i) {
            jobs[i] = states[b0 + i]->job(outs[b0 + i]);
            tiles_y[i] = states[b0 + i]->tiles_y;
        }
        unsigned int* counter = ctx->d_batch_counters + (ctx->batch_slot++ % kBatchCounterSlots);
        launch_blend_batch(jobs, tiles_y, m, counter, s);
    }
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_render_backward(wipes_ctx* ctx, wipes_state* st, const float* params, const float* dL_dout,
                                   float* dL_dparams, void* stream) {
    if (!ctx || !st || !dL_dout || (st->N > 0 && (!params || !dL_dparams)))
        return fail(WIPES_ERR_INVALID, "null argument");
    if (st->dims != 2 && st->dims != 3) return fail(WIPES_ERR_INVALID, "state holds no forward pass");
    if (st->dims == 3 && !st->bnd_valid)
        return fail(WIPES_ERR_INVALID, "the 3D backward needs a one-frame forward (wipes_render3d) on the state");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    const int64_t N = st->N;
    if (st->dims == 2) {
        WIPES_TRY(ensure(st->partial, sizeof(float) * 12 * (size_t)std::max<int64_t>(st->n_inst, 1)));
        {
            StageTimer t(ctx, WIPES_STAGE_BWD_RASTER, s);
            launch_backward2d(st->rec.as<float4>(), st->rect.as<PixRect>(), st->lists(), st->W, st->H, st->tiles_x,
                              st->tiles_y, st->opts.cutoff_sigma, dL_dout, st->partial.as<float>(), s);
        }
        StageTimer t(ctx, WIPES_STAGE_BWD_CHAIN, s);
        launch_reduce_chain2d(params, N, st->opts.cov2d, st->offsets.as<uint32_t>(), st->counts.as<uint32_t>(),
                              st->partial.as<float>(), dL_dparams, s);
    } else {
        const size_t gstride = (size_t)image_grad_stride3d(st->opts.freq_proj_mode);
        WIPES_TRY(ensure(st->grad_img, sizeof(float) * gstride * (size_t)std::max<int64_t>(N, 1)));
        {
            StageTimer t(ctx, WIPES_STAGE_BWD_RASTER, s);
            if (N > 0) WIPES_CUDA(cudaMemsetAsync(st->grad_img.p, 0, sizeof(float) * gstride * (size_t)N, s));
            const BwdChunks ch{st->bwd_items.as<uint2>(), st->n_items.as<uint32_t>(), st->item_base.as<uint32_t>(),
                               st->bnd.as<float4>(), st->cfin.as<float>(), st->n_items.as<unsigned int>() + 1};
            launch_backward3d(st->rec.as<float4>(), st->rect.as<PixRect>(), st->lists(), st->W, st->H, st->tiles_x,
                              blend_opts(st->opts), st->T_final.as<float>(), st->last.as<uint32_t>(), dL_dout,
                              st->grad_img.as<float>(), ch, st->max_items, s);
        }
        StageTimer t(ctx, WIPES_STAGE_BWD_CHAIN, s);
        launch_chain3d(params, N, st->cam, st->W, st->H, st->opts.dilation, st->opts.freq_proj_mode,
                       st->opts.sh_degree, st->rec.as<float4>(),
                       st->grad_img.as<float>(), dL_dparams, s);
    }
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_sort_pairs(wipes_ctx* ctx, wipes_state* st, uint32_t* keys, uint32_t* vals, int64_t n,
                              int key_bits, void* stream) {
    if (!ctx || !st || st->ctx != ctx) return fail(WIPES_ERR_INVALID, "wipes_sort_pairs: bad context or state");
    if (n < 0 || n > (int64_t)INT32_MAX || key_bits < 1 || key_bits > 32 || (n > 0 && (!keys || !vals)))
        return fail(WIPES_ERR_INVALID, "wipes_sort_pairs: need 0 <= n <= 2^31-1, 1 <= key_bits <= 32 and buffers");
    if (n <= 1) return WIPES_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    WIPES_TRY(ensure(st->sort_k, sizeof(uint32_t) * (size_t)n));
    WIPES_TRY(ensure(st->sort_v, sizeof(uint32_t) * (size_t)n));
    WIPES_TRY(ensure(st->hist, sizeof(uint32_t) * (size_t)radix_hist_words(n)));
    uint32_t* kb[2] = {keys, st->sort_k.as<uint32_t>()};
    uint32_t* vb[2] = {vals, st->sort_v.as<uint32_t>()};
    {
        StageTimer t(ctx, WIPES_STAGE_SORT, s);
        const int cur = radix_sort_pairs(kb, vb, n, key_bits, st->hist.as<uint32_t>(), ctx->d_error, s);
        if (cur == 1) {  // an odd number of passes ends in the second buffers
            WIPES_CUDA(cudaMemcpyAsync(keys, kb[1], sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
            WIPES_CUDA(cudaMemcpyAsync(vals, vb[1], sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        }
    }
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_deform6d(const float* params6, int64_t N, float t, float* params3, void* stream) {
    if (N < 0 || (N > 0 && (!params6 || !params3))) return fail(WIPES_ERR_INVALID, "bad argument");
    launch_deform6d(params6, N, t, params3, (cudaStream_t)stream);
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_deform6d_backward(const float* params6, int64_t N, float t, const float* dL_dparams3,
                                     float* dL_dparams6, int accumulate, void* stream) {
    if (N < 0 || (N > 0 && (!params6 || !dL_dparams3 || !dL_dparams6))) return fail(WIPES_ERR_INVALID, "bad argument");
    launch_deform6d_backward(params6, N, t, dL_dparams3, dL_dparams6, accumulate, (cudaStream_t)stream);
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_l2_loss(wipes_ctx* ctx, const float* img, const float* target, int64_t n, float* loss,
                           float* dL_dimg, void* stream) {
    if (!ctx || n <= 0 || !img || !target || !loss || !dL_dimg) return fail(WIPES_ERR_INVALID, "bad argument");
    DeviceGuard g(ctx->device);
    StageTimer t(ctx, WIPES_STAGE_LOSS, (cudaStream_t)stream);
    launch_l2_loss(img, target, n, loss, dL_dimg, ctx->d_loss_partials, (cudaStream_t)stream);
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_l2_loss_noalloc(const float* img, const float* target, int64_t n, float* loss, float* dL_dimg,
                                   void* stream) {
    if (!img || !target || !loss || !dL_dimg) return fail(WIPES_ERR_INVALID, "null argument");
    const int64_t max_n = l2_loss_noalloc_max_elements();
    if (n < 1 || n > max_n)
        return fail(WIPES_ERR_INVALID, "wipes_l2_loss_noalloc: n = " + std::to_string(n) + " is outside 1.." +
                                           std::to_string(max_n) + " (the fixed scratch holds one partial sum per " +
                                           "4096 elements, 65536 partial sums)");
    cudaError_t e = l2_loss_noalloc(img, target, n, loss, dL_dimg, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(WIPES_ERR_CUDA, std::string("wipes_l2_loss_noalloc: ") + cudaGetErrorString(e));
    return WIPES_OK;
}

wipes_status wipes_state_get_info(const wipes_state* st, wipes_state_info* info) {
    if (!st || !info) return fail(WIPES_ERR_INVALID, "null argument");
    info->dims = st->dims;
    info->H = st->H;
    info->W = st->W;
    info->tiles_x = st->tiles_x;
    info->tiles_y = st->tiles_y;
    info->N = st->N;
    info->n_instances = st->n_inst;
    info->bytes_reserved = (int64_t)st->reserved();
    return WIPES_OK;
}

wipes_status wipes_state_copy_lists(const wipes_state* st, uint32_t* tile_ids, uint32_t* prim_ids,
                                    uint32_t* tile_ranges, void* stream) {
    if (!st) return fail(WIPES_ERR_INVALID, "null state");
    if (st->dims == 0) return fail(WIPES_ERR_INVALID, "state holds no forward pass");
    DeviceGuard g(st->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t I = (size_t)st->n_inst;
    if (tile_ids && I)
        WIPES_CUDA(cudaMemcpyAsync(tile_ids, st->keys[st->sorted].p, I * 4, cudaMemcpyDeviceToDevice, s));
    if (prim_ids && I) WIPES_CUDA(cudaMemcpyAsync(prim_ids, st->sprim.p, I * 4, cudaMemcpyDeviceToDevice, s));
    if (tile_ranges)
        WIPES_CUDA(cudaMemcpyAsync(tile_ranges, st->ranges.p, (size_t)st->tiles_x * st->tiles_y * sizeof(uint2),
                                   cudaMemcpyDeviceToDevice, s));
    return WIPES_OK;
}

wipes_status wipes_state_copy_pixel_state(const wipes_state* st, float* T_final, uint32_t* last_index, void* stream) {
    if (!st) return fail(WIPES_ERR_INVALID, "null state");
    if (st->dims != 3) return fail(WIPES_ERR_INVALID, "state holds no 3D forward pass");
    DeviceGuard g(st->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npix = (size_t)st->H * st->W;
    if (T_final) WIPES_CUDA(cudaMemcpyAsync(T_final, st->T_final.p, npix * 4, cudaMemcpyDeviceToDevice, s));
    if (last_index) WIPES_CUDA(cudaMemcpyAsync(last_index, st->last.p, npix * 4, cudaMemcpyDeviceToDevice, s));
    return WIPES_OK;
}

wipes_status wipes_state_count_pairs(wipes_ctx* ctx, const wipes_state* st, int64_t* visited, int64_t* inside,
                                     void* stream) {
    if (!ctx || !st || !visited || !inside) return fail(WIPES_ERR_INVALID, "null argument");
    if (st->dims == 0) return fail(WIPES_ERR_INVALID, "state holds no forward pass");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    WIPES_CUDA(cudaMemsetAsync(ctx->d_counters, 0, sizeof(unsigned long long) * 2, s));
    launch_count_pairs(st->rec.as<float4>(), st->lists(), st->W, st->H, st->tiles_x, st->tiles_y,
                       st->opts.cutoff_sigma * st->opts.cutoff_sigma,
                       st->dims == 3 ? st->last.as<uint32_t>() : nullptr, ctx->d_counters, s);
    unsigned long long h[2] = {0, 0};
    WIPES_CUDA(cudaMemcpyAsync(h, ctx->d_counters, sizeof(h), cudaMemcpyDeviceToHost, s));
    WIPES_CUDA(cudaStreamSynchronize(s));
    *visited = (int64_t)h[0];
    *inside = (int64_t)h[1];
    return WIPES_OK;
}

wipes_status wipes_set_timing(wipes_ctx* ctx, int enable) {
    if (!ctx) return fail(WIPES_ERR_INVALID, "null ctx");
    ctx->timing = enable != 0;
    return WIPES_OK;
}

wipes_status wipes_get_timing(wipes_ctx* ctx, double* ms, int64_t* brackets, int reset) {
    if (!ctx) return fail(WIPES_ERR_INVALID, "null ctx");
    DeviceGuard g(ctx->device);
    for (auto& b : ctx->pending) {
        WIPES_CUDA(cudaEventSynchronize(b.b));
        float e = 0.f;
        WIPES_CUDA(cudaEventElapsedTime(&e, b.a, b.b));
        ctx->stage_ms[b.stage] += e;
        ctx->stage_n[b.stage] += 1;
        ctx->free_events.push_back(b.a);
        ctx->free_events.push_back(b.b);
    }
    ctx->pending.clear();
    for (int k = 0; k < WIPES_STAGE_COUNT; ++k) {
        if (ms) ms[k] = ctx->stage_ms[k];
        if (brackets) brackets[k] = ctx->stage_n[k];
        if (reset) {
            ctx->stage_ms[k] = 0.0;
            ctx->stage_n[k] = 0;
        }
    }
    return WIPES_OK;
}

int64_t wipes_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

wipes_status wipes_set_memory_limit(wipes_ctx* ctx, int64_t bytes) {
    if (!ctx || bytes < 0) return fail(WIPES_ERR_INVALID, "bad argument");
    ctx->mem.limit = bytes;
    return WIPES_OK;
}

wipes_status wipes_get_memory_reserved(wipes_ctx* ctx, int64_t* bytes) {
    if (!ctx || !bytes) return fail(WIPES_ERR_INVALID, "null argument");
    *bytes = ctx->mem.reserved.load();
    return WIPES_OK;
}

const char* wipes_status_string(wipes_status s) {
    switch (s) {
        case WIPES_OK: return "ok";
        case WIPES_ERR_INVALID: return "invalid argument";
        case WIPES_ERR_CAPACITY: return "capacity exceeded";
        case WIPES_ERR_CUDA: return "CUDA error";
        case WIPES_ERR_TIMEOUT: return "device wait timed out";
        case WIPES_ERR_OOM: return "out of device memory";
    }
    return "unknown status";
}

const char* wipes_last_error(void) { return g_last_error.c_str(); }

wipes_status wipes_sync_status(wipes_ctx* ctx, void* stream) {
    if (!ctx) return fail(WIPES_ERR_INVALID, "null ctx");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    WIPES_CUDA(cudaStreamSynchronize(s));
    WIPES_CUDA(cudaGetLastError());
    WIPES_CUDA(cudaMemcpyAsync(ctx->h_total + 1, ctx->d_error, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    WIPES_CUDA(cudaStreamSynchronize(s));
    return take_device_error(ctx, s);
}

int64_t wipes_deform_mlp_param_count(void) { return mlp_param_count(); }

wipes_status wipes_deform_mlp(wipes_ctx* ctx, wipes_state* st, const float* params3, int64_t N, float t,
                              const float* theta, float* params_out, void* stream) {
    if (!ctx || !st || !theta || (N > 0 && (!params3 || !params_out))) return fail(WIPES_ERR_INVALID, "null argument");
    if (N < 0 || N > (int64_t)INT32_MAX) return fail(WIPES_ERR_INVALID, "N out of range");
    if (!std::isfinite(t)) return fail(WIPES_ERR_INVALID, "t must be finite");
    if (((uintptr_t)params3 & 15) || ((uintptr_t)theta & 15) || ((uintptr_t)params_out & 15))
        return fail(WIPES_ERR_INVALID, "params3, theta and params_out must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    const MlpSizes z = mlp_sizes(std::max<int64_t>(N, 1));
    WIPES_TRY(ensure(st->mlp_act, z.act));
    WIPES_TRY(ensure(st->mlp_d, z.out));
    WIPES_TRY(ensure(st->mlp_theta16, z.theta16));
    st->mlp_N = -1;
    StageTimer tm(ctx, WIPES_STAGE_MLP_FWD, s);
    const std::string e = mlp_forward(params3, N, t, theta, st->mlp_theta16.p, st->mlp_act.p, st->mlp_d.as<float>(),
                                      params_out, ctx->d_error, s);
    if (!e.empty()) return fail(WIPES_ERR_CUDA, e);
    WIPES_CUDA(cudaGetLastError());
    st->mlp_N = N;
    return WIPES_OK;
}

wipes_status wipes_deform_mlp_backward(wipes_ctx* ctx, wipes_state* st, const float* params3, const float* dL_dout,
                                       float* dL_dtheta, float* dL_dparams3, int accumulate, void* stream) {
    if (!ctx || !st || !dL_dtheta) return fail(WIPES_ERR_INVALID, "null argument");
    if (st->mlp_N < 0) return fail(WIPES_ERR_INVALID, "state holds no deformation-network forward pass");
    const int64_t N = st->mlp_N;
    if (N > 0 && (!params3 || !dL_dout || !dL_dparams3)) return fail(WIPES_ERR_INVALID, "null argument");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    AllocStream alloc_stream(s);
    const MlpSizes z = mlp_sizes(std::max<int64_t>(N, 1));
    WIPES_TRY(ensure(st->mlp_scratch, z.scratch));
    if (N == 0) {
        if (!accumulate) WIPES_CUDA(cudaMemsetAsync(dL_dtheta, 0, sizeof(float) * (size_t)mlp_param_count(), s));
        return WIPES_OK;
    }
    StageTimer tm(ctx, WIPES_STAGE_MLP_BWD, s);
    const std::string e = mlp_backward(params3, N, st->mlp_theta16.p, st->mlp_act.p, st->mlp_d.as<float>(),
                                       st->mlp_scratch.p, dL_dout, dL_dtheta, dL_dparams3, accumulate, ctx->d_error, s);
    if (!e.empty()) return fail(WIPES_ERR_CUDA, e);
    WIPES_CUDA(cudaGetLastError());
    return WIPES_OK;
}

wipes_status wipes_selftest_sort_timeout(wipes_ctx* ctx, void* stream) {
    if (!ctx) return fail(WIPES_ERR_INVALID, "null ctx");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // report (and clear) anything latched before, so that the result is this probe's
    WIPES_TRY(wipes_sync_status(ctx, stream));
    void* ws = nullptr;
    WIPES_CUDA(cudaMalloc(&ws, sizeof(uint32_t) * (size_t)sort_timeout_probe_words()));
    sort_timeout_probe(static_cast<uint32_t*>(ws), ctx->d_error, s);
    const wipes_status st = wipes_sync_status(ctx, stream);
    cudaFree(ws);
    return st;
}

}  // extern "C"
