// Binning: scan of per-primitive tile counts, emission of (tile, primitive) pairs, a stable LSD
// radix sort of the pairs, and per-tile ranges of the sorted list (the tile-sorting pipeline of
// 3DGS that the paper follows, Sec. 4.1; the paper cites a GPU sort for this step, Sec. 1).
//
// Order contract: pairs are emitted in scan order (primitive index in 2D, front-to-back depth
// order in 3D), and the sort is stable, so each tile's list is ordered by that scan order.
#include <mutex>

#include "common.cuh"

namespace wipes {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Exclusive scan over a 256-thread block; returns the exclusive prefix and writes the block total.
template <typename T, int NW = kWarps>
__device__ __forceinline__ T block_exclusive_scan(T x, T* total, T* s_warp /* [NW] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    T warp_base = 0, sum = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const T s = s_warp[w];
        if (w < warp) warp_base += s;
        sum += s;
    }
    __syncthreads();
    if (total) *total = sum;
    return warp_base + inc - x;
}

// ---------------------------------------------------------------------------------------------
// scan of tile counts and emission
// ---------------------------------------------------------------------------------------------

constexpr int kScanItems = kScanBlockElems / kThreads;  // 4

__global__ void __launch_bounds__(kThreads) k_block_sums(const uint32_t* __restrict__ counts,
                                                         const uint32_t* __restrict__ perm, int64_t n,
                                                         unsigned long long* __restrict__ block_sums) {
    pdl_enter();
    __shared__ unsigned long long s_warp[kWarps];
    const int64_t base = (int64_t)blockIdx.x * kScanBlockElems + threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t j = base + k;
        if (j < n) s += counts[perm ? perm[j] : (uint32_t)j];
    }
    unsigned long long total;
    block_exclusive_scan<unsigned long long>(s, &total, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_scan_block_sums(unsigned long long* __restrict__ v, int nb,
                                                              unsigned long long* __restrict__ total_out,
                                                              const unsigned long long* __restrict__ error,
                                                              unsigned long long* __restrict__ readback) {
    pdl_enter();
    __shared__ unsigned long long s_warp[kWarps];
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kThreads) {
        const int j = base + threadIdx.x;
        const unsigned long long x = j < nb ? v[j] : 0ull;
        unsigned long long chunk;
        const unsigned long long ex = block_exclusive_scan<unsigned long long>(x, &chunk, s_warp);
        if (j < nb) v[j] = carry + ex;
        carry += chunk;
    }
    if (threadIdx.x == 0) {
        *total_out = carry;
        // the host's pinned readback (device address of mapped host memory): the total and the
        // device error word, read after the stream is synchronised, with no copy
        if (readback) {
            readback[0] = carry;
            readback[1] = *error;
        }
    }
}

// First instance index of every primitive: the block-local exclusive scan of the tile counts of
// its 1024 scan positions plus the block's offset.
__global__ void __launch_bounds__(kThreads) k_scan_offsets(const uint32_t* __restrict__ counts,
                                                           const uint32_t* __restrict__ perm, int64_t n,
                                                           const unsigned long long* __restrict__ block_offsets,
                                                           uint32_t* __restrict__ offsets, uint2* __restrict__ ranges,
                                                           int n_tiles) {
    pdl_enter();
    __shared__ unsigned long long s_warp[kWarps];
    // the tile ranges start empty: k_tile_ranges writes those of the tiles that get pairs
    for (int t = blockIdx.x * kThreads + threadIdx.x; t < n_tiles; t += gridDim.x * kThreads) ranges[t] = make_uint2(0u, 0u);
    const int64_t base = (int64_t)blockIdx.x * kScanBlockElems + threadIdx.x * kScanItems;
    uint32_t prim[kScanItems], cnt[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t j = base + k;
        prim[k] = j < n ? (perm ? perm[j] : (uint32_t)j) : 0u;
        cnt[k] = j < n ? counts[prim[k]] : 0u;
        s += cnt[k];
    }
    unsigned long long off = block_offsets[blockIdx.x] + block_exclusive_scan<unsigned long long>(s, nullptr, s_warp);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) offsets[prim[k]] = (uint32_t)off;
        off += cnt[k];
    }
}

// Emission, one thread per scan position: a primitive writes the tiles of its covered range that
// its cutoff ellipse reaches, in row-major tile order, from its offset on.  The warp's 32 ranges
// are laid end to end (a prefix of their tile counts over the lanes) and visited 32 tiles a round:
// the tile in slot s belongs to the lane whose prefix range holds s (a binary search over the
// lanes' inclusive prefixes); a primitive whose count equals its range's tile count reaches every
// tile and needs no test.  A hit goes to its primitive's next index at the round's start plus the
// primitive's hits in earlier slots of the round's ballot.
__global__ void __launch_bounds__(kThreads) k_emit(const uint32_t* __restrict__ counts,
                                                   const uint32_t* __restrict__ perm, int64_t n,
                                                   const float4* __restrict__ rec, const PixRect* __restrict__ rect,
                                                   const uint32_t* __restrict__ offsets, int tiles_x, float lim,
                                                   const unsigned long long* __restrict__ n_inst, int64_t capacity,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                   uint32_t* __restrict__ inst_prim) {
    pdl_enter();
    if (*n_inst > (unsigned long long)capacity) return;  // the host launches it again into larger buffers
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t p = 0u, run = 0u;  // run: this lane's primitive's next instance index
    PixRect r{1, 1, 0, 0};
    int tx0 = 0, ty0 = 0, nx = 1, nt = 0;
    bool full = true;
    Ellipse e{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (j < n) {
        p = perm ? perm[j] : (uint32_t)j;
        const uint32_t cnt = counts[p];
        if (cnt) {
            r = rect[p];
            run = offsets[p];
            tx0 = r.u0 / kTile;
            ty0 = r.v0 / kTile;
            nx = r.u1 / kTile - tx0 + 1;
            nt = nx * (r.v1 / kTile - ty0 + 1);
            full = (int)cnt == nt;
            if (!full) {
                const float4 A = rec[(size_t)p * kRecF4 + 0];
                e = make_ellipse(A.x, A.y, A.z, A.w, rec[(size_t)p * kRecF4 + 1].x);
            }
        }
    }
    int incl = nt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - nt;
    for (int s0 = 0; s0 < total; s0 += 32) {
        const int s = s0 + lane;
        int k = 0;  // the slot's owner: the number of lanes whose inclusive prefix is at most s
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
            if (__shfl_sync(0xffffffffu, incl, k + step - 1) <= s) k += step;
        const int ek = __shfl_sync(0xffffffffu, excl, k);
        const int nxk = __shfl_sync(0xffffffffu, nx, k);
        const int txk = __shfl_sync(0xffffffffu, tx0, k), tyk = __shfl_sync(0xffffffffu, ty0, k);
        const bool fullk = __shfl_sync(0xffffffffu, full, k);
        const uint32_t pk = __shfl_sync(0xffffffffu, p, k), basek = __shfl_sync(0xffffffffu, run, k);
        PixRect rk;
        rk.u0 = __shfl_sync(0xffffffffu, r.u0, k);
        rk.u1 = __shfl_sync(0xffffffffu, r.u1, k);
        rk.v0 = __shfl_sync(0xffffffffu, r.v0, k);
        rk.v1 = __shfl_sync(0xffffffffu, r.v1, k);
        Ellipse ekk;
        ekk.mx = __shfl_sync(0xffffffffu, e.mx, k);
        ekk.my = __shfl_sync(0xffffffffu, e.my, k);
        ekk.l11 = __shfl_sync(0xffffffffu, e.l11, k);
        ekk.l21 = __shfl_sync(0xffffffffu, e.l21, k);
        ekk.l22 = __shfl_sync(0xffffffffu, e.l22, k);
        ekk.rBA = __shfl_sync(0xffffffffu, e.rBA, k);
        ekk.rBC = __shfl_sync(0xffffffffu, e.rBC, k);
        const int t = s - ek;
        const int row = t / nxk, col = t - row * nxk;
        const int tx = txk + col, ty = tyk + row;
        const bool hit = s < total && (fullk || tile_touched(ekk, rk, tx, ty, lim));
        const uint32_t hits = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int lo = max(ek - s0, 0);  // the owner's first slot of the round
            const uint32_t w = basek + (uint32_t)__popc(hits & ((1u << lane) - 1u) & ~((1u << lo) - 1u));
            keys[w] = (uint32_t)(ty * tiles_x + tx);
            vals[w] = w;
            inst_prim[w] = pk;
        }
        // each primitive's index moves past its hits of the round
        const int lo = max(excl - s0, 0), hi = min(incl - s0, 32);
        if (lo < hi) run += (uint32_t)__popc((hits >> lo) & (0xffffffffu >> (32 - (hi - lo))));
    }
}

__global__ void k_gather_u32(uint32_t* __restrict__ out, const uint32_t* __restrict__ table,
                             const uint32_t* __restrict__ idx, int64_t n) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = table[idx[i]];
}

__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = keys[i];
        if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

__global__ void k_iota(uint32_t* __restrict__ v, int64_t n) {
    pdl_enter();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------------------------
// stable LSD radix sort of 32-bit keys with 32-bit values, up to 8 bits per pass, in one of two
// schemes that rank a tile of keys the same way (radix_sort_pairs picks one per call).
// Onesweep, one kernel per pass: k_sort_histogram counts every pass's digits over all keys once.
// In a pass, blocks take
// tiles of 4096 keys in index order from a counter, rank their keys stably, publish each digit's
// count for their tile and obtain the counts of all earlier tiles by a decoupled look-back over
// the published words (a word holds a tile's count, or the inclusive prefix up to that tile,
// with a flag in its top bits).  Every look-back wait is bounded: when it runs out, the block
// sets bit 0 of the error word and stops looking; the host reports WIPES_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------------------

constexpr int kSortItems = 16;
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = kSortThreads * kSortItems;  // 8192 keys per block (reduce-then-scan)
// Onesweep serves the short sorts of many passes, whose time is the latency of a block's tile:
// half the tile puts twice the blocks to work (300k keys: 74 blocks instead of 37).
constexpr int kPassItems = 8;
constexpr int kPassTile = kSortThreads * kPassItems;  // 4096 keys per block (onesweep)
constexpr int kMaxRadix = 256;
constexpr int kMaxPasses = 4;
constexpr unsigned long long kAggregate = 1ull << 62, kPrefix = 2ull << 62, kCountMask = (1ull << 62) - 1ull;
constexpr int kMaxLookbackPolls = 1 << 21;
constexpr int kLookback = 8;

struct SortPlan {
    int passes;
    int shift[kMaxPasses];
    int nbits[kMaxPasses];
};

// Workspace (32-bit words): digit totals [kMaxPasses][kMaxRadix] | tile counters [kMaxPasses] |
// look-back words [kMaxPasses][tiles][kMaxRadix] (64-bit, 8-byte aligned).
__host__ __device__ inline int64_t sort_status_offset_words() { return (int64_t)kMaxPasses * kMaxRadix + kMaxPasses; }

// A look-back word carries its own value (count and flag in one 64-bit word) and nothing else is
// read on its account, so relaxed gpu-scope accesses suffice; unlike acquire loads they let the
// loads of several predecessors be in flight at once.
__device__ __forceinline__ void store_word(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long load_word(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Digit counts of every pass over all keys.  Each warp counts into its own shared histogram with
// plain shared-memory atomics (equal digits within one instruction are serialised by the hardware,
// different warps never contend); a thread reads four consecutive keys with one 16-byte load when
// the array is 16-byte aligned.
__global__ void __launch_bounds__(kThreads) k_sort_histogram(const uint32_t* __restrict__ keys, int64_t n,
                                                             SortPlan plan, uint32_t* __restrict__ totals) {
    pdl_enter();
    __shared__ uint32_t s_cnt[kWarps][kMaxPasses * kMaxRadix];
    for (int k = threadIdx.x; k < kWarps * kMaxPasses * kMaxRadix; k += kThreads) (&s_cnt[0][0])[k] = 0u;
    __syncthreads();
    uint32_t* my = s_cnt[threadIdx.x >> 5];
    auto count = [&](uint32_t key) {
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p)
            if (p < plan.passes)
                atomicAdd(&my[p * kMaxRadix + ((key >> plan.shift[p]) & ((1u << plan.nbits[p]) - 1u))], 1u);
    };
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    if ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0) {
        const uint4* k4 = reinterpret_cast<const uint4*>(keys);
        const int64_t n4 = n >> 2;
        for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n4; q += stride) {
            const uint4 v = k4[q];
            count(v.x);
            count(v.y);
            count(v.z);
            count(v.w);
        }
        for (int64_t idx = (n4 << 2) + (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < n; idx += stride)
            count(keys[idx]);
    } else {
        for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < n; idx += stride) count(keys[idx]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < plan.passes * kMaxRadix; k += kThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += s_cnt[w][k];
        if (sum) atomicAdd(&totals[k], sum);
    }
}

// Shared memory of k_sort_downsweep (dynamic, 16-byte aligned words): keys and values of the
// tile, the per-warp digit counts, then the small per-digit arrays.  The two peer tables of the
// ranking live in the key area, which is free until the keys are placed.
constexpr int kSortSmemWords = 2 * kSortTile + kSortWarps * kMaxRadix + 3 * kMaxRadix + kSortWarps + 4;
constexpr size_t kSortSmemBytes = sizeof(uint32_t) * kSortSmemWords;
static_assert(2 * kSortWarps * kMaxRadix <= kSortTile, "the peer tables must fit in the key area");
// k_sort_pass: the same arrays for its smaller tile, and the peer tables after them (they do not
// fit in its key area).
constexpr int kPassPeerWords = 2 * kPassTile + kSortWarps * kMaxRadix + 3 * kMaxRadix + kSortWarps + 4;
constexpr size_t kPassSmemBytes = sizeof(uint32_t) * (kPassPeerWords + 2 * kSortWarps * kMaxRadix);
static_assert(kPassPeerWords % 4 == 0, "the peer tables start 16-byte aligned");

struct SortPassArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;
    uint32_t* keys_out;
    uint32_t* vals_out;
    int64_t n;
    int shift, nbits;
    const uint32_t* totals;
    unsigned int* tile_counter;
    unsigned long long* status;
    unsigned int* error;
    const uint32_t* table;  // optional: gathered[g] = table[value] for each placed pair
    uint32_t* gathered;
};

// One tile of a pass.  FULL: the tile holds kPassTile keys (every tile but the last), so no
// element needs a bounds check.  Item i of warp w's run is tile element w * 32 kPassItems + 32 i +
// lane, so that a warp's loads and the element order of its ranking agree.
template <bool FULL>
__device__ __forceinline__ void sort_tile(const SortPassArgs& a, uint32_t tile, int cnt, uint32_t* s_keys,
                                          uint32_t* s_vals, uint32_t (*s_wc)[kMaxRadix], uint32_t* s_cnt,
                                          uint32_t* s_dstart, uint32_t* s_gbase, uint32_t* s_warp) {
    const int radix = 1 << a.nbits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int shift = a.shift;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t blk = (int64_t)tile * kPassTile;
    const int run = warp * (kPassItems * 32) + lane;
    const uint32_t* keys_in = a.keys_in + blk;
    auto valid = [&](int i) { return FULL || run + 32 * i < cnt; };
    // the keys wait in s_vals at their element position until they are placed; the tile's digit
    // counts are taken first so that later tiles can use them as early as possible
    {
        uint32_t k[kPassItems];
#pragma unroll
        for (int i = 0; i < kPassItems; ++i) k[i] = valid(i) ? keys_in[run + 32 * i] : 0u;
#pragma unroll
        for (int i = 0; i < kPassItems; ++i) {
            s_vals[run + 32 * i] = k[i];
            if (valid(i)) atomicAdd(&s_cnt[(k[i] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    unsigned long long* mine = a.status + (size_t)tile * kMaxRadix + threadIdx.x;
    const uint32_t running = (int)threadIdx.x < radix ? s_cnt[threadIdx.x] : 0u;
    if ((int)threadIdx.x < radix) store_word(mine, (tile == 0 ? kPrefix : kAggregate) | running);
    // stable rank within the warp's run, in element order (item i, then lane).  The lanes of an
    // item with the same digit find each other through the warp's peer table: each sets its bit in
    // the digit's word and reads the word back; the last of them then clears it and advances the
    // digit's running count.  Items alternate between two tables, so a table word is cleared a full
    // item before it is used again.
    uint32_t(*s_peer)[kSortWarps][kMaxRadix] = reinterpret_cast<uint32_t(*)[kSortWarps][kMaxRadix]>(s_keys + kPassPeerWords);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t pos[kPassItems];
#pragma unroll
    for (int i = 0; i < kPassItems; ++i) {
        const bool ok = valid(i);
        const uint32_t d = (s_vals[run + 32 * i] >> shift) & mask;
        uint32_t* peer = &s_peer[i & 1][warp][d];
        if (ok) atomicOr(peer, 1u << lane);
        __syncwarp();
        const uint32_t peers = ok ? *peer : 0u;
        const uint32_t before = s_wc[warp][d];
        __syncwarp();
        pos[i] = before + __popc(peers & lt);
        if (ok && lane == 31 - __clz(peers)) {
            *peer = 0u;
            s_wc[warp][d] = before + __popc(peers);
        }
    }
    __syncthreads();
    // per digit: prefix over warps, then the counts of all earlier tiles (look-back)
    if ((int)threadIdx.x < radix) {
        const int d = threadIdx.x;
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = s_wc[w][d];
            s_wc[w][d] = acc;
            acc += t;
        }
        unsigned long long before = 0;
        if (tile != 0) {
            // walk back kLookback tiles per step (their words are loaded together), adding
            // aggregates until an inclusive prefix; a tile that has published nothing yet is polled
            int polls = 0;
            for (int64_t t = (int64_t)tile - 1; t >= 0;) {
                unsigned long long w[kLookback];
#pragma unroll
                for (int j = 0; j < kLookback; ++j)
                    w[j] = t - j >= 0 ? load_word(a.status + (size_t)(t - j) * kMaxRadix + d) : kPrefix;
                bool done = false;
                int used = 0;
#pragma unroll
                for (int j = 0; j < kLookback; ++j) {
                    if (done || used < j) continue;  // stopped at a prefix or at an unpublished tile
                    if (w[j] & kPrefix) {
                        if (t - j >= 0) before += w[j] & kCountMask;
                        done = true;
                    } else if (w[j] & kAggregate) {
                        before += w[j] & kCountMask;
                        used = j + 1;
                    }
                }
                if (done) break;
                t -= used;
                if (used == 0) {
                    if (++polls > kMaxLookbackPolls) {
                        atomicOr(a.error, 1u);
                        break;
                    }
                    if (polls > 64) __nanosleep(128);
                }
            }
            store_word(mine, kPrefix | (before + running));
        }
        s_gbase[d] += (uint32_t)before;
    }
    {
        const uint32_t ex = block_exclusive_scan<uint32_t, kSortWarps>(running, nullptr, s_warp);
        if ((int)threadIdx.x < radix) {
            s_dstart[threadIdx.x] = ex;
            s_gbase[threadIdx.x] -= ex;
        }
    }
    __syncthreads();
    // keys to their place in the tile's digit order, then the values (read only now, so that they
    // occupy no registers during the ranking)
#pragma unroll
    for (int i = 0; i < kPassItems; ++i) {
        if (valid(i)) {
            const uint32_t key = s_vals[run + 32 * i];
            const uint32_t d = (key >> shift) & mask;
            pos[i] += s_dstart[d] + s_wc[warp][d];
            s_keys[pos[i]] = key;
        }
    }
    {
        const uint32_t* vals_in = a.vals_in + blk;
        uint32_t v[kPassItems];
#pragma unroll
        for (int i = 0; i < kPassItems; ++i) v[i] = valid(i) ? vals_in[run + 32 * i] : 0u;
        __syncthreads();  // every key has left s_vals
#pragma unroll
        for (int i = 0; i < kPassItems; ++i)
            if (valid(i)) s_vals[pos[i]] = v[i];
    }
    __syncthreads();
    const int64_t n = a.n;
    for (int t = threadIdx.x; t < (FULL ? kPassTile : cnt); t += kSortThreads) {
        const uint32_t key = s_keys[t];
        const uint32_t g = s_gbase[(key >> shift) & mask] + (uint32_t)t;
        if ((int64_t)g >= n) continue;  // only after a look-back that ran out (error word set)
        const uint32_t val = s_vals[t];
        a.keys_out[g] = key;
        a.vals_out[g] = val;
        if (a.table) a.gathered[g] = a.table[val];
    }
}

__global__ void __launch_bounds__(kSortThreads, 2) k_sort_pass(const __grid_constant__ SortPassArgs a) {
    pdl_enter();
    extern __shared__ uint4 s_sort_raw[];
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_sort_raw);
    uint32_t* s_vals = s_keys + kPassTile;
    uint32_t(*s_wc)[kMaxRadix] = reinterpret_cast<uint32_t(*)[kMaxRadix]>(s_vals + kPassTile);
    uint32_t* s_cnt = s_vals + kPassTile + kSortWarps * kMaxRadix;
    uint32_t* s_dstart = s_cnt + kMaxRadix;
    uint32_t* s_gbase = s_dstart + kMaxRadix;
    uint32_t* s_warp = s_gbase + kMaxRadix;
    uint32_t* s_tile_p = s_warp + kSortWarps;
    const int radix = 1 << a.nbits;
    if (threadIdx.x == 0) *s_tile_p = atomicAdd(a.tile_counter, 1u);
    for (int k = threadIdx.x; k < 2 * kSortWarps * kMaxRadix; k += kSortThreads) s_keys[kPassPeerWords + k] = 0u;
    for (int k = threadIdx.x; k < kSortWarps * kMaxRadix; k += kSortThreads) (&s_wc[0][0])[k] = 0u;
    if ((int)threadIdx.x < kMaxRadix) s_cnt[threadIdx.x] = 0u;
    // global start of each digit = exclusive scan of the digit totals
    {
        const uint32_t x = (int)threadIdx.x < radix ? a.totals[threadIdx.x] : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t, kSortWarps>(x, nullptr, s_warp);
        if ((int)threadIdx.x < radix) s_gbase[threadIdx.x] = ex;
    }
    __syncthreads();
    const uint32_t tile = *s_tile_p;
    const int64_t left = a.n - (int64_t)tile * kPassTile;
    // a pass whose digit is the same for every key (one digit holds all n) is the identity: every
    // block of the pass sees the same totals, so all of them copy their tile and none waits on
    // another's look-back word
    if (__syncthreads_or((int)threadIdx.x < radix && a.totals[threadIdx.x] == (uint32_t)a.n)) {
        const int64_t base = (int64_t)tile * kPassTile;
        const int cnt = left < (int64_t)kPassTile ? (int)left : kPassTile;
        for (int t = threadIdx.x; t < cnt; t += kSortThreads) {
            const uint32_t key = a.keys_in[base + t], val = a.vals_in[base + t];
            a.keys_out[base + t] = key;
            a.vals_out[base + t] = val;
            if (a.table) a.gathered[base + t] = a.table[val];
        }
        return;
    }
    if (left >= kPassTile)
        sort_tile<true>(a, tile, kPassTile, s_keys, s_vals, s_wc, s_cnt, s_dstart, s_gbase, s_warp);
    else
        sort_tile<false>(a, tile, (int)left, s_keys, s_vals, s_wc, s_cnt, s_dstart, s_gbase, s_warp);
}

// Order of the tiles for the blend kernels, longest list first: tiles are bucketed by the bit
// length of their list length and the buckets laid out in decreasing order (the order inside a
// bucket is arbitrary).  The block scheduler starts blocks in index order, so the tiles with the
// most work start first and short tiles fill in at the end.  The same pass lists the 3D backward's
// work items in that order: tile t with a list of len entries has bwd_chunks(len) chunks (none when
// empty), items item_base[t] .. item_base[t] + chunks - 1 = (t, chunk).  One block does all
// tiles.
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 33;
__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const uint2* __restrict__ ranges, int n_tiles,
                                                              uint32_t* __restrict__ order, uint2* __restrict__ items,
                                                              uint32_t* __restrict__ item_base,
                                                              uint32_t* __restrict__ n_items) {
    pdl_enter();
    __shared__ uint32_t s_cnt[kOrderBuckets];
    __shared__ uint32_t s_cur[kOrderBuckets];
    __shared__ uint32_t s_icnt[kOrderBuckets];
    __shared__ uint32_t s_icur[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) s_cnt[threadIdx.x] = 0u, s_icnt[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += kOrderThreads) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x, b = 32 - __clz(len);
        atomicAdd(&s_cnt[b], 1u);
        if (len) atomicAdd(&s_icnt[b], bwd_chunks(len));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0, irun = 0;
        for (int b = kOrderBuckets - 1; b >= 0; --b) {
            s_cur[b] = run;
            run += s_cnt[b];
            s_icur[b] = irun;
            irun += s_icnt[b];
        }
        if (n_items) *n_items = irun;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += kOrderThreads) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x, b = 32 - __clz(len);
        order[atomicAdd(&s_cur[b], 1u)] = (uint32_t)t;
        if (items && len) {
            const uint32_t k_n = bwd_chunks(len);
            const uint32_t base = atomicAdd(&s_icur[b], k_n);
            item_base[t] = base;
            for (uint32_t k = 0; k < k_n; ++k) items[base + k] = make_uint2((uint32_t)t, k);
        }
    }
}

}  // namespace

void launch_block_sums(const uint32_t* counts, const uint32_t* perm, int64_t n, unsigned long long* block_sums,
                       cudaStream_t stream) {
    if (n == 0) return;
    launch_pdl(k_block_sums, ceil_div(n, kScanBlockElems), kThreads, 0, stream, counts, perm, n, block_sums); count_launches(1);
}

void launch_scan_block_sums(unsigned long long* block_sums, int nb, unsigned long long* total,
                            const unsigned long long* error, unsigned long long* readback, cudaStream_t stream) {
    launch_pdl(k_scan_block_sums, 1, kThreads, 0, stream, block_sums, nb, total, error, readback); count_launches(1);
}

void launch_emit(const uint32_t* counts, const uint32_t* perm, int64_t n, const float4* rec, const PixRect* rect,
                 const unsigned long long* block_offsets, const unsigned long long* total, int64_t capacity,
                 int tiles_x, float lim, uint32_t* keys, uint32_t* vals, uint32_t* inst_prim, uint32_t* offsets,
                 uint2* ranges, int n_tiles, cudaStream_t stream) {
    if (n == 0) return;
    launch_pdl(k_scan_offsets, ceil_div(n, kScanBlockElems), kThreads, 0, stream, counts, perm, n, block_offsets, offsets,
               ranges, n_tiles);
    launch_pdl(k_emit, ceil_div(n, kThreads), kThreads, 0, stream, counts, perm, n, rec, rect, offsets, tiles_x, lim,
               total, capacity, keys, vals, inst_prim);
    count_launches(2);
}

void launch_gather_u32(uint32_t* out, const uint32_t* table, const uint32_t* idx, int64_t n, cudaStream_t stream) {
    if (n == 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    launch_pdl(k_gather_u32, grid, 256, 0, stream, out, table, idx, n);
    count_launches(1);
}

void launch_tile_ranges(const uint32_t* sorted_keys, int64_t n, uint2* ranges, int n_tiles, bool zeroed,
                        cudaStream_t stream) {
    if (!zeroed) cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, stream);
    if (n == 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    launch_pdl(k_tile_ranges, grid, 256, 0, stream, sorted_keys, n, ranges); count_launches(1);
}

void launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* order, uint2* items, uint32_t* item_base,
                       uint32_t* n_items, cudaStream_t stream) {
    launch_pdl(k_tile_order, 1, kOrderThreads, 0, stream, ranges, n_tiles, order, items, item_base, n_items);
    count_launches(1);
}

void launch_iota(uint32_t* v, int64_t n, cudaStream_t stream) {
    if (n == 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
    launch_pdl(k_iota, grid, 256, 0, stream, v, n); count_launches(1);
}

// ---------------------------------------------------------------------------------------------
// The same sort by reduce-then-scan, with no wait between blocks.  The input is cut into chunks of
// whole tiles, one chunk per block of the last kernel (two blocks per SM).  Per pass:
//   k_sort_upsweep     block c counts the digits of chunk c;
//   k_sort_chunk_scan  block d scans digit d's counts over the chunks: the digit's count in all
//                      earlier chunks, and its total;
//   k_sort_downsweep   block c walks chunk c tile by tile: it ranks each tile stably in shared
//                      memory and writes each pair to (digits below d overall) + (digit d in
//                      earlier chunks) + (digit d earlier in this chunk) + its rank in the tile.
// ---------------------------------------------------------------------------------------------

constexpr int kChunkBlocksPerSm = 2;
// Below this many keys reduce-then-scan ranks 4096-key tiles, twice the blocks of a short sort.
constexpr int64_t kSmallTileMaxKeys = (int64_t)1 << 20;
int down_tile_keys(int64_t n) { return n < kSmallTileMaxKeys ? kPassTile : kSortTile; }
constexpr int64_t kOnesweepMaxKeys = (int64_t)1 << 22;  // onesweep only below this many keys (and > 2 passes)

// Chunks and whole tiles per chunk for n keys.
int sort_chunks(int64_t n, int tile_keys, int* tiles_per_chunk) {
    const int64_t tiles = ceil_div(std::max<int64_t>(n, 1), (int64_t)tile_keys);
    const int64_t target = std::min<int64_t>(tiles, (int64_t)152 * kChunkBlocksPerSm);
    const int64_t tpc = ceil_div(tiles, target);
    *tiles_per_chunk = (int)tpc;
    return (int)ceil_div(tiles, tpc);
}

// counts: [radix][chunks], or with chunk_major [chunks][kMaxRadix] (read by k_sort_downsweep_fused)
__global__ void __launch_bounds__(kThreads) k_sort_upsweep(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                           int nbits, int64_t chunk_keys, int chunks, int chunk_major,
                                                           uint32_t* __restrict__ counts) {
    pdl_enter();
    __shared__ uint32_t s_cnt[kWarps][kMaxRadix];
    for (int k = threadIdx.x; k < kWarps * kMaxRadix; k += kThreads) (&s_cnt[0][0])[k] = 0u;
    __syncthreads();
    uint32_t* my = s_cnt[threadIdx.x >> 5];
    const uint32_t mask = (1u << nbits) - 1u;
    const int64_t lo = (int64_t)blockIdx.x * chunk_keys, hi = min(n, lo + chunk_keys);
    if ((reinterpret_cast<uintptr_t>(keys + lo) & 15u) == 0) {
        const uint4* k4 = reinterpret_cast<const uint4*>(keys + lo);
        const int64_t q4 = (hi - lo) >> 2;
#pragma unroll 4
        for (int64_t q = threadIdx.x; q < q4; q += kThreads) {
            const uint4 v = k4[q];
            atomicAdd(&my[(v.x >> shift) & mask], 1u);
            atomicAdd(&my[(v.y >> shift) & mask], 1u);
            atomicAdd(&my[(v.z >> shift) & mask], 1u);
            atomicAdd(&my[(v.w >> shift) & mask], 1u);
        }
        for (int64_t i = lo + (q4 << 2) + threadIdx.x; i < hi; i += kThreads) atomicAdd(&my[(keys[i] >> shift) & mask], 1u);
    } else {
        for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) atomicAdd(&my[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < (1 << nbits); d += kThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += s_cnt[w][d];
        counts[chunk_major ? (size_t)blockIdx.x * kMaxRadix + d : (size_t)d * chunks + blockIdx.x] = sum;
    }
}

constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_sort_chunk_scan(const uint32_t* __restrict__ counts, int chunks,
                                                                  uint32_t* __restrict__ bases,
                                                                  uint32_t* __restrict__ totals) {
    pdl_enter();
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int d = blockIdx.x;
    uint32_t run = 0;
    for (int c0 = 0; c0 < chunks; c0 += kScanThreads) {
        const int c = c0 + threadIdx.x;
        const uint32_t x = c < chunks ? counts[(size_t)d * chunks + c] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<uint32_t, kScanThreads / 32>(x, &total, s_warp);
        if (c < chunks) bases[(size_t)d * chunks + c] = run + ex;
        run += total;
    }
    if (threadIdx.x == 0) totals[d] = run;
}

struct SortDownArgs {
    const uint32_t* keys_in;
    const uint32_t* vals_in;
    uint32_t* keys_out;
    uint32_t* vals_out;
    int64_t n;
    int shift, nbits;
    int chunks, tiles_per_chunk;
    const uint32_t* bases;   // [radix][chunks]: the digit's count in earlier chunks (k_sort_downsweep_fused:
                             // the chunk-major counts of k_sort_upsweep)
    const uint32_t* totals;  // [radix]
    const uint32_t* table;   // optional: gathered[g] = table[value] for each placed pair
    uint32_t* gathered;
};

// One tile of a chunk (see sort_tile for the element layout and the ranking).  s_base[d]: where
// the chunk's next digit-d pair goes.
// ITEMS keys per thread: kSortItems (8192-key tiles, the peer tables in the key area) or
// kPassItems (4096-key tiles in the layout of k_sort_pass, the peer tables after the arrays).
template <int ITEMS, bool FULL>
__device__ __forceinline__ void down_tile(const SortDownArgs& a, int64_t tile, int cnt, uint32_t* s_keys,
                                          uint32_t* s_vals, uint32_t (*s_wc)[kMaxRadix], uint32_t* s_dstart,
                                          uint32_t* s_base, uint32_t* s_gofs, uint32_t* s_warp) {
    static_assert(ITEMS == kSortItems || ITEMS == kPassItems, "tile layouts");
    constexpr int kTileKeys = kSortThreads * ITEMS;
    uint32_t* peer_base = ITEMS == kSortItems ? s_keys : s_keys + kPassPeerWords;
    const int radix = 1 << a.nbits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int shift = a.shift;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t blk = tile * kTileKeys;
    const int run = warp * (ITEMS * 32) + lane;
    auto valid = [&](int i) { return FULL || run + 32 * i < cnt; };
    uint32_t(*s_peer)[kSortWarps][kMaxRadix] = reinterpret_cast<uint32_t(*)[kSortWarps][kMaxRadix]>(peer_base);
    for (int k = threadIdx.x; k < kSortWarps * kMaxRadix; k += kSortThreads) (&s_wc[0][0])[k] = 0u;
    for (int k = threadIdx.x; k < 2 * kSortWarps * kMaxRadix; k += kSortThreads) peer_base[k] = 0u;
    {
        const uint32_t* keys_in = a.keys_in + blk;
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) s_vals[run + 32 * i] = valid(i) ? keys_in[run + 32 * i] : 0u;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t pos[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = valid(i);
        const uint32_t d = (s_vals[run + 32 * i] >> shift) & mask;
        uint32_t* peer = &s_peer[i & 1][warp][d];
        if (ok) atomicOr(peer, 1u << lane);
        __syncwarp();
        const uint32_t peers = ok ? *peer : 0u;
        const uint32_t before = s_wc[warp][d];
        __syncwarp();
        pos[i] = before + __popc(peers & lt);
        if (ok && lane == 31 - __clz(peers)) {
            *peer = 0u;
            s_wc[warp][d] = before + __popc(peers);
        }
    }
    __syncthreads();
    uint32_t count = 0;
    if ((int)threadIdx.x < radix) {
        const int d = threadIdx.x;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = s_wc[w][d];
            s_wc[w][d] = count;
            count += t;
        }
    }
    {
        const uint32_t ex = block_exclusive_scan<uint32_t, kSortWarps>(count, nullptr, s_warp);
        if ((int)threadIdx.x < radix) {
            s_dstart[threadIdx.x] = ex;
            s_gofs[threadIdx.x] = s_base[threadIdx.x] - ex;
            s_base[threadIdx.x] += count;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (valid(i)) {
            const uint32_t key = s_vals[run + 32 * i];
            const uint32_t d = (key >> shift) & mask;
            pos[i] += s_dstart[d] + s_wc[warp][d];
            s_keys[pos[i]] = key;
        }
    }
    {
        const uint32_t* vals_in = a.vals_in + blk;
        uint32_t v[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) v[i] = valid(i) ? vals_in[run + 32 * i] : 0u;
        __syncthreads();  // every key has left s_vals
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (valid(i)) s_vals[pos[i]] = v[i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (FULL ? kTileKeys : cnt); t += kSortThreads) {
        const uint32_t key = s_keys[t];
        const uint32_t g = s_gofs[(key >> shift) & mask] + (uint32_t)t;
        const uint32_t val = s_vals[t];
        a.keys_out[g] = key;
        a.vals_out[g] = val;
        if (a.table) a.gathered[g] = a.table[val];
    }
    __syncthreads();  // the tile's buffers are free for the next tile
}

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads, 2) k_sort_downsweep(const __grid_constant__ SortDownArgs a) {
    pdl_enter();
    constexpr int kTileKeys = kSortThreads * ITEMS;
    extern __shared__ uint4 s_sort_raw[];
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_sort_raw);
    uint32_t* s_vals = s_keys + kTileKeys;
    uint32_t(*s_wc)[kMaxRadix] = reinterpret_cast<uint32_t(*)[kMaxRadix]>(s_vals + kTileKeys);
    uint32_t* s_dstart = s_vals + kTileKeys + kSortWarps * kMaxRadix;
    uint32_t* s_base = s_dstart + kMaxRadix;
    uint32_t* s_gofs = s_base + kMaxRadix;
    uint32_t* s_warp = s_gofs + kMaxRadix;
    const int radix = 1 << a.nbits;
    // where this chunk's first pair of each digit goes
    {
        const uint32_t x = (int)threadIdx.x < radix ? a.totals[threadIdx.x] : 0u;
        const uint32_t ex = block_exclusive_scan<uint32_t, kSortWarps>(x, nullptr, s_warp);
        if ((int)threadIdx.x < radix) s_base[threadIdx.x] = ex + a.bases[(size_t)threadIdx.x * a.chunks + blockIdx.x];
    }
    __syncthreads();
    const int64_t tiles = (a.n + kTileKeys - 1) / kTileKeys;
    const int64_t t0 = (int64_t)blockIdx.x * a.tiles_per_chunk, t1 = min(tiles, t0 + a.tiles_per_chunk);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t left = a.n - tile * kTileKeys;
        if (left >= kTileKeys)
            down_tile<ITEMS, true>(a, tile, kTileKeys, s_keys, s_vals, s_wc, s_dstart, s_base, s_gofs, s_warp);
        else
            down_tile<ITEMS, false>(a, tile, (int)left, s_keys, s_vals, s_wc, s_dstart, s_base, s_gofs, s_warp);
    }
}

// k_sort_downsweep without the scan kernel before it, for sorts with few chunks: each block finds
// its chunk's digit offsets from the chunk-major counts itself.  Digit d of chunk c starts after all
// keys of smaller digits and after digit d's keys in the chunks before c; the kSortThreads / radix
// threads of a digit sum its counts over interleaved chunks.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads, 2) k_sort_downsweep_fused(const __grid_constant__ SortDownArgs a) {
    pdl_enter();
    constexpr int kTileKeys = kSortThreads * ITEMS;
    extern __shared__ uint4 s_sort_raw[];
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_sort_raw);
    uint32_t* s_vals = s_keys + kTileKeys;
    uint32_t(*s_wc)[kMaxRadix] = reinterpret_cast<uint32_t(*)[kMaxRadix]>(s_vals + kTileKeys);
    uint32_t* s_dstart = s_vals + kTileKeys + kSortWarps * kMaxRadix;
    uint32_t* s_base = s_dstart + kMaxRadix;
    uint32_t* s_gofs = s_base + kMaxRadix;
    uint32_t* s_warp = s_gofs + kMaxRadix;
    const int radix = 1 << a.nbits;  // 2 .. 256
    {
        const int parts = kSortThreads / radix;
        const int d = (int)threadIdx.x & (radix - 1), part = (int)threadIdx.x / radix;
        uint32_t all = 0, before = 0;
        for (int c = part; c < a.chunks; c += parts) {
            const uint32_t x = a.bases[(size_t)c * kMaxRadix + d];  // chunk-major counts
            all += x;
            before += c < (int)blockIdx.x ? x : 0u;
        }
        s_keys[threadIdx.x] = all;
        s_vals[threadIdx.x] = before;
        __syncthreads();
        uint32_t tot = 0, bef = 0;
        if ((int)threadIdx.x < radix) {
            for (int q = 0; q < parts; ++q) {
                tot += s_keys[q * radix + threadIdx.x];
                bef += s_vals[q * radix + threadIdx.x];
            }
        }
        const uint32_t ex = block_exclusive_scan<uint32_t, kSortWarps>(tot, nullptr, s_warp);
        if ((int)threadIdx.x < radix) s_base[threadIdx.x] = ex + bef;
    }
    __syncthreads();
    const int64_t tiles = (a.n + kTileKeys - 1) / kTileKeys;
    const int64_t t0 = (int64_t)blockIdx.x * a.tiles_per_chunk, t1 = min(tiles, t0 + a.tiles_per_chunk);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t left = a.n - tile * kTileKeys;
        if (left >= kTileKeys)
            down_tile<ITEMS, true>(a, tile, kTileKeys, s_keys, s_vals, s_wc, s_dstart, s_base, s_gofs, s_warp);
        else
            down_tile<ITEMS, false>(a, tile, (int)left, s_keys, s_vals, s_wc, s_dstart, s_base, s_gofs, s_warp);
    }
}
// Sorts whose chunk-major counts hold at most this many words skip the scan kernel.
constexpr int64_t kFusedScanMaxWords = (int64_t)1 << 16;

int64_t radix_hist_words(int64_t n) {
    const int64_t tiles = ceil_div(std::max<int64_t>(n, 1), kPassTile);
    const int64_t onesweep = sort_status_offset_words() + 2 * (int64_t)kMaxPasses * tiles * kMaxRadix;
    int tpc = 0;
    const int64_t chunked = 2 * (int64_t)kMaxRadix * sort_chunks(n, down_tile_keys(n), &tpc) + kMaxRadix;
    return std::max(onesweep, chunked);
}

// The pass kernel's shared memory is above the 48 KB default: raise its limit once per process
// (the attribute is per device; the library uses the device that is current at its first sort).
void sort_pass_attributes() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemBytes);
        cudaFuncSetAttribute(k_sort_downsweep<kSortItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSortSmemBytes);
        cudaFuncSetAttribute(k_sort_downsweep<kPassItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPassSmemBytes);
        cudaFuncSetAttribute(k_sort_downsweep_fused<kSortItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSortSmemBytes);
        cudaFuncSetAttribute(k_sort_downsweep_fused<kPassItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPassSmemBytes);
    });
}

int radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits, uint32_t* hist, unsigned int* error,
                     cudaStream_t stream, const uint32_t* table, uint32_t* gathered) {
    if (n <= 1 || bits <= 0) {
        if (table) launch_gather_u32(gathered, table, vals[0], n, stream);
        return 0;
    }
    SortPlan plan{};
    plan.passes = (bits + 7) / 8;
    for (int p = 0, shift = 0; p < plan.passes; ++p) {
        plan.nbits[p] = (bits - shift + (plan.passes - p) - 1) / (plan.passes - p);  // split the remaining bits evenly
        plan.shift[p] = shift;
        shift += plan.nbits[p];
    }
    sort_pass_attributes();
    // Reduce-then-scan costs three launches per pass, onesweep one (plus one histogram): for a
    // short sort of many passes the launches dominate and onesweep is the faster of the two;
    // otherwise reduce-then-scan, which never waits on another block, is.
    if (plan.passes <= 2 || n >= kOnesweepMaxKeys) {
        int tpc = 0;
        const int tile_keys = down_tile_keys(n);
        const int chunks = sort_chunks(n, tile_keys, &tpc);
        uint32_t* counts = hist;
        uint32_t* bases = hist + (size_t)kMaxRadix * chunks;
        uint32_t* totals = bases + (size_t)kMaxRadix * chunks;
        // few chunks: the downsweep finds its offsets from the counts itself (two launches a pass)
        const bool fused = (int64_t)chunks * kMaxRadix <= kFusedScanMaxWords;
        int cur = 0;
        for (int p = 0; p < plan.passes; ++p) {
            const bool last_pass = p == plan.passes - 1;
            launch_pdl(k_sort_upsweep, (unsigned)chunks, kThreads, 0, stream, (const uint32_t*)keys[cur], n, plan.shift[p],
                       plan.nbits[p], (int64_t)tpc * tile_keys, chunks, (int)fused, counts);
            if (!fused)
                launch_pdl(k_sort_chunk_scan, (unsigned)(1 << plan.nbits[p]), kScanThreads, 0, stream,
                           (const uint32_t*)counts, chunks, bases, totals);
            SortDownArgs da{keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, plan.shift[p], plan.nbits[p], chunks,
                            tpc, fused ? counts : bases, totals, last_pass ? table : nullptr,
                            last_pass ? gathered : nullptr};
            if (fused) {
                if (tile_keys == kPassTile)
                    launch_pdl(k_sort_downsweep_fused<kPassItems>, (unsigned)chunks, kSortThreads, kPassSmemBytes, stream,
                               da);
                else
                    launch_pdl(k_sort_downsweep_fused<kSortItems>, (unsigned)chunks, kSortThreads, kSortSmemBytes, stream,
                               da);
            } else if (tile_keys == kPassTile) {
                launch_pdl(k_sort_downsweep<kPassItems>, (unsigned)chunks, kSortThreads, kPassSmemBytes, stream, da);
            } else {
                launch_pdl(k_sort_downsweep<kSortItems>, (unsigned)chunks, kSortThreads, kSortSmemBytes, stream, da);
            }
            count_launches(fused ? 2 : 3);
            cur ^= 1;
        }
        return cur;
    }
    const int64_t tiles = ceil_div(n, kPassTile);
    uint32_t* totals = hist;
    unsigned int* counters = hist + (int64_t)kMaxPasses * kMaxRadix;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(hist + sort_status_offset_words());
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)sort_status_offset_words() +
                                 sizeof(unsigned long long) * (size_t)(plan.passes * tiles * kMaxRadix), stream);
    const unsigned hgrid = (unsigned)std::min<int64_t>(ceil_div(n, kThreads * 4), 152 * 4);
    launch_pdl(k_sort_histogram, hgrid, kThreads, 0, stream, keys[0], n, plan, totals);
    count_launches(1);
    int cur = 0;
    for (int p = 0; p < plan.passes; ++p) {
        const bool last_pass = p == plan.passes - 1;
        SortPassArgs pa{keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, plan.shift[p], plan.nbits[p],
                        totals + p * kMaxRadix, counters + p, status + (size_t)p * tiles * kMaxRadix, error,
                        last_pass ? table : nullptr, last_pass ? gathered : nullptr};
        launch_pdl(k_sort_pass, (unsigned)tiles, kSortThreads, kPassSmemBytes, stream, pa);
        count_launches(1);
        cur ^= 1;
    }
    return cur;
}

// Scratch words of sort_timeout_probe(): keys and values in and out for two tiles, the digit
// totals, the pass's tile counter and the look-back words of two tiles.
int64_t sort_timeout_probe_words() { return 4 * 2 * kPassTile + sort_status_offset_words() + 2 * 2 * kMaxRadix; }

void sort_timeout_probe(uint32_t* ws, unsigned int* error, cudaStream_t stream) {
    const int64_t n = 2 * kPassTile;
    uint32_t* keys_in = ws;
    uint32_t* vals_in = ws + n;
    uint32_t* keys_out = ws + 2 * n;
    uint32_t* vals_out = ws + 3 * n;
    uint32_t* hist = ws + 4 * n;  // 8-byte aligned: 4 n words from an aligned base
    unsigned int* counter = hist + (int64_t)kMaxPasses * kMaxRadix;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(hist + sort_status_offset_words());
    cudaMemsetAsync(ws, 0, sizeof(uint32_t) * (size_t)sort_timeout_probe_words(), stream);
    // the pass's counter starts at 1: the single block takes tile 1 and tile 0 is never published
    cudaMemsetAsync(counter, 1, 1, stream);
    sort_pass_attributes();
    SortPassArgs pa{keys_in, vals_in, keys_out, vals_out, n, 0, 8, hist, counter, status, error, nullptr, nullptr};
    launch_pdl(k_sort_pass, 1u, kSortThreads, kPassSmemBytes, stream, pa);
    count_launches(1);
}

}  // namespace wipes
