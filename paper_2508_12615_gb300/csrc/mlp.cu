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
// Every product runs on the 5th-generation tensor cores (tcgen05.mma, bfloat16 operands, fp32
// accumulation in tensor memory), in hand-written kernels:
//   k_mlp_encode the positional encoding of every row, written as the tiles the forward loads.
//   k_mlp_fwd   one 128-row tile at a time: the nine layers and the record update.  Each layer's
//               output stays in shared memory as the next layer's A operand (K-major, 128-byte
//               swizzle); the weights, packed once per call into the same layout (k_mlp_pack),
//               stream in by bulk copies, one 64-column K-block at a time, through a ring of
//               stages.  A copy of every layer's A operand goes to global memory for the backward.
//   k_mlp_bwd   one tile at a time: the record update's backward, then dh = dz W through the
//               layers (W transposed), the ReLU mask taken from the stored activations (positive
//               entries), the bias gradients; it writes each layer's dz and dL/dgamma.
//   k_mlp_encode_backward  the encoding's backward to the centre.
//   k_mlp_wgrad the weight gradients dW_l = dz_l^T x_l: a product over all rows (the stored tiles
//               read as MN-major operands), split into row chunks (one partial per chunk), then
//               k_mlp_wsum adds the partials in a fixed order.
// Rounding points: the encoding, weights, hidden activations and upstream gradients are rounded
// to bfloat16 where they become product operands; biases, accumulators, the network outputs and
// the encoding's gradient (both products summed in one accumulator) stay fp32.
// Warp roles in the tile kernels: warps 0 and 10 stream weights (one thread each, half of every
// block), warp 1 issues the MMAs (one thread), warps 2-9 run the epilogue (thread = row; warp w reads TMEM lanes 32 (w % 4) .., warps 2-5 the
// output columns 0-127, warps 6-9 128-255).  Every wait on an mbarrier is bounded (2 s); one that
// runs out sets bit 1 of the context's error word, every role leaves its loop, in-flight copies
// and MMAs are waited for, and the tensor memory is freed before the block exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <utility>
#include <mutex>
#include <string>

#include "common.cuh"
#include "tc.cuh"

namespace wipes {

namespace {

constexpr int kLx = 10, kLt = 6;
constexpr int kInPad = 80;
constexpr int kWidth = 256;
constexpr int kHidden = 8;
constexpr int kSkipLayer = 5;
constexpr int kOut = 13;
constexpr int kOutPad = 16;
constexpr int kX5 = kInPad + kWidth;  // 336

// inputs and outputs of layer l (0 .. 8)
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kInPad : l == kSkipLayer ? kX5 : kWidth; }
__host__ __device__ constexpr int layer_out(int l) { return l == kHidden ? kOut : kWidth; }

__host__ __device__ constexpr int64_t layer_offset(int l) {
    int64_t k = 0;
    for (int i = 0; i < l; ++i) k += (int64_t)layer_out(i) * layer_in(i) + layer_out(i);
    return k;
}

constexpr int kRows = 128;                      // rows per tile: the MMA's M
constexpr int kEpiWarps = 8;                    // two per SM sub-partition, each owning half the columns
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTcThreads = 96 + kEpiThreads;    // warps 0 and 10 stream weights, warp 1 issues MMAs
constexpr int kProducer2 = 2 + kEpiWarps;       // the second weight-streaming warp
constexpr int kWgThreads = 192;                 // weight gradient: 4 epilogue warps
constexpr int kStages = 4;                      // weight stages: a whole 256-wide layer in flight
constexpr uint32_t kABlock = kRows * 128;       // one K-block of a 128-row tile: 16 KB
constexpr uint32_t kWBlock = kWidth * 128;      // one K-block of a 256-row operand: 32 KB
constexpr uint64_t kWaitNs = 2000000000ull;     // a wait on an mbarrier gives up after 2 s
constexpr unsigned kMlpTimeoutBit = 2u;
constexpr int kBiasFloats = kHidden * kWidth + kOutPad;  // 2064: hidden biases, then the head's (padded)
constexpr int kEpiBar = 1;                      // named barrier of the epilogue warps

// Per-tile copies in global memory of the tiles' A operands, as they stand in shared memory
// (K-major along the features, 128-byte swizzle): K-block g holds features 64 g .. 64 g + 63 of
// the 128 rows.  Read back by the weight gradient, where the rows are the contraction (K) axis,
// they are MN-major operands.
constexpr uint32_t kHtLayer = 4 * kABlock;            // a 256-wide layer: 64 KB
constexpr uint32_t kHtTile = kHidden * kHtLayer;      // 8 layers: 512 KB
constexpr uint32_t kGtTile = 2 * kABlock;             // gamma: features 0-63 and 64-79 (+ padding)
constexpr uint32_t kDdTile = kABlock;                 // dL/dd: 16 features (+ padding)
// ReLU masks of a tile's hidden layers, written by the forward for the backward: per layer and row
// 256 bits, 8 words (word w covers columns 32 w .. 32 w + 31: bit j is column 32 w + 2 j, bit
// 16 + j column 32 w + 2 j + 1, set where the ReLU output is positive), the order in which packed
// bfloat16 pairs give up their halves most cheaply
constexpr uint32_t kMkLayer = kRows * 32;             // 4 KB
constexpr uint32_t kMkTile = kHidden * kMkLayer;      // 32 KB

// ---- weight streams ------------------------------------------------------------------------------
// One entry per K-block an MMA group reads: the image's byte offset and size, the A K-block, the K
// steps of 16 in it, the B rows (the MMA's N), the accumulator column, whether its first step
// starts the accumulator (else it adds), whether the group ends with it, and what the issuer waits
// for before it: nothing (its A operand is already in place), the tile's encoding (the bulk copy's
// barrier), or one half of the previous layer's output (the epilogue publishes A K-blocks 0 and 2,
// then 1 and 3, each on its own barrier).
enum : uint8_t { kWaitNone = 0, kWaitGamma = 1, kWaitHalf0 = 2, kWaitHalf1 = 3 };
struct Blk {
    uint32_t off, bytes;
    uint8_t akb, steps, first, last, wait;
    uint16_t n, dcol;
};
constexpr int kMaxBlk = 40;
struct Sched {
    int n;
    Blk b[kMaxBlk];
};

// Forward, per tile: L0 (A = gamma in A K-blocks 4, 5: K 80), L1-L4 (A = h, K-blocks 0-3), L5 (A =
// (h4, gamma), K-blocks 0-5: its image's columns are ordered h4 first), L6, L7, L8 (16 rows).
// Layer l accumulates in tensor-memory columns 256 (l & 1) .., so that layer l + 1's products can
// start while the epilogue still reads layer l's; the h K-blocks go in the order 0, 2, 1, 3, the
// order in which the epilogue publishes them, and the skip layer's encoding part goes first (its A
// operand is in place since the tile started).
__host__ __device__ constexpr uint32_t fwd_image_base(int l) {
    uint32_t base = 2u * kWBlock;  // layer 0: two K-blocks of 256 rows
    for (int i = 1; i < l; ++i) base += (uint32_t)(i == kSkipLayer ? 6 : 4) * kWBlock;
    return l == 0 ? 0u : base;
}
__host__ __device__ constexpr Sched make_fwd() {
    Sched s{};
    auto add = [&](uint32_t off, int akb, int steps, int n, int dcol, bool first, bool last, uint8_t wait) {
        Blk& b = s.b[s.n++];
        b.off = off;
        b.bytes = (uint32_t)n * 128u;
        b.akb = (uint8_t)akb;
        b.steps = (uint8_t)steps;
        b.n = (uint16_t)n;
        b.dcol = (uint16_t)dcol;
        b.first = first;
        b.last = last;
        b.wait = wait;
    };
    add(0u, 4, 4, kWidth, 0, true, false, kWaitGamma);
    add(kWBlock, 5, 1, kWidth, 0, false, true, kWaitNone);
    for (int l = 1; l <= kHidden; ++l) {
        const int n = l == kHidden ? kOutPad : kWidth;
        const uint32_t kbytes = (uint32_t)n * 128u, base = fwd_image_base(l);
        const int dcol = (l & 1) * kWidth;
        bool first = true;
        if (l == kSkipLayer) {
            add(base + 4u * kbytes, 4, 4, n, dcol, true, false, kWaitNone);
            add(base + 5u * kbytes, 5, 1, n, dcol, false, false, kWaitNone);
            first = false;
        }
        const int order[4] = {0, 2, 1, 3};
        for (int i = 0; i < 4; ++i)
            add(base + (uint32_t)order[i] * kbytes, order[i], 4, n, dcol, first && i == 0, i == 3,
                i == 0 ? kWaitHalf0 : i == 2 ? kWaitHalf1 : kWaitNone);
    }
    return s;
}
constexpr uint32_t kFwdImgBytesTotal = fwd_image_base(kHidden) + 4u * kOutPad * 128u;
// Backward data, per tile: head (A = dd, one K step; B = W8^T), L7, L6, L5 (dh4 into columns
// 0-255, then dgamma into columns 256-335), L4 .. L1, L0 (dgamma += dz0 W0).  A group starts once
// the epilogue has published its A operand.
__host__ __device__ constexpr Sched make_bwd() {
    Sched s{};
    uint32_t off = 0;
    bool group_start = true;
    auto add = [&](int akb, int steps, int n, int dcol, bool first, bool last) {
        Blk& b = s.b[s.n++];
        b.off = off;
        b.bytes = (uint32_t)n * 128u;
        b.akb = (uint8_t)akb;
        b.steps = (uint8_t)steps;
        b.n = (uint16_t)n;
        b.dcol = (uint16_t)dcol;
        b.first = first;
        b.last = last;
        b.wait = group_start ? kWaitHalf0 : kWaitNone;
        group_start = last;
        off += b.bytes;
    };
    add(0, 1, kWidth, 0, true, true);
    for (int l = 7; l >= 0; --l) {
        if (l == 0) {
            for (int kb = 0; kb < 4; ++kb) add(kb, 4, kInPad, kWidth, false, kb == 3);
            continue;
        }
        for (int kb = 0; kb < 4; ++kb) add(kb, 4, kWidth, 0, kb == 0, l != kSkipLayer && kb == 3);
        if (l == kSkipLayer)
            for (int kb = 0; kb < 4; ++kb) add(kb, 4, kInPad, kWidth, kb == 0, kb == 3);
    }
    return s;
}
constexpr Sched kFwdSched = make_fwd();
constexpr Sched kBwdSched = make_bwd();
constexpr uint32_t kFwdImgBytes = kFwdImgBytesTotal;
constexpr uint32_t kBwdImgBytes = kBwdSched.b[kBwdSched.n - 1].off + kBwdSched.b[kBwdSched.n - 1].bytes;
__constant__ Sched c_fwd = make_fwd();
__constant__ Sched c_bwd = make_bwd();

// Images of the weights, described for the packing kernel: element (row n, column k) of image i is
// theta[src + n sn + col(k) sk] for n < nvalid and k < kvalid (0 elsewhere), with col(k) = k + klo
// for k < ksplit and k - ksplit + khi beyond (the skip layer's reordered columns).
struct ImgDesc {
    uint32_t dst, rows, nkb;  // byte offset, rows (N), K-blocks
    int64_t src;
    int32_t sn, sk, nvalid, kvalid, ksplit, klo, khi;
};
constexpr int kNumImg = 22;
struct ImgTable {
    ImgDesc d[kNumImg];
    int n;
};
ImgTable make_images() {
    ImgTable t{};
    uint32_t off = 0;
    auto add = [&](int rows, int nkb, int64_t src, int sn, int sk, int nvalid, int kvalid, int ksplit, int klo, int khi) {
        ImgDesc& d = t.d[t.n++];
        d.dst = off;
        d.rows = (uint32_t)rows;
        d.nkb = (uint32_t)nkb;
        d.src = src;
        d.sn = sn;
        d.sk = sk;
        d.nvalid = nvalid;
        d.kvalid = kvalid;
        d.ksplit = ksplit;
        d.klo = klo;
        d.khi = khi;
        off += (uint32_t)rows * 128u * (uint32_t)nkb;
    };
    // forward images (B = W_l: rows = outputs, K = inputs), in the order of kFwdSched
    add(kWidth, 2, layer_offset(0), kInPad, 1, kWidth, kInPad, 1 << 30, 0, 0);
    for (int l = 1; l <= 7; ++l) {
        if (l == kSkipLayer)
            add(kWidth, 6, layer_offset(l), kX5, 1, kWidth, kX5, kWidth, kInPad, 0);
        else
            add(kWidth, 4, layer_offset(l), kWidth, 1, kWidth, kWidth, 1 << 30, 0, 0);
    }
    add(kOutPad, 4, layer_offset(8), kWidth, 1, kOut, kWidth, 1 << 30, 0, 0);
    // backward images (B = W_l^T: rows = inputs, K = outputs), in the order of kBwdSched
    add(kWidth, 1, layer_offset(8), 1, kWidth, kWidth, kOut, 1 << 30, 0, 0);
    for (int l = 7; l >= 0; --l) {
        if (l == 0) {
            add(kInPad, 4, layer_offset(0), 1, kInPad, kInPad, kWidth, 1 << 30, 0, 0);
        } else if (l == kSkipLayer) {
            add(kWidth, 4, layer_offset(l) + kInPad, 1, kX5, kWidth, kWidth, 1 << 30, 0, 0);
            add(kInPad, 4, layer_offset(l), 1, kX5, kInPad, kWidth, 1 << 30, 0, 0);
        } else {
            add(kWidth, 4, layer_offset(l), 1, kWidth, kWidth, kWidth, 1 << 30, 0, 0);
        }
    }
    return t;
}

// ---- small device helpers -------------------------------------------------------------------------
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    const uint32_t a = tc::smem_u32(p);
    return p + ((1024u - (a & 1023u)) & 1023u);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&b);
}
// max(lo, 0) and max(hi, 0) rounded to bfloat16 and packed (one instruction)
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Write 8 packed bfloat16 pairs (16 columns starting at a multiple of 16) of row r into a 128-row
// K-major swizzled tile in shared memory.
__device__ __forceinline__ void store_a16(uint32_t a_base, int r, int k0, const uint32_t* w) {
    const uint32_t kb = (uint32_t)k0 / 64u, c = ((uint32_t)k0 % 64u) / 8u;
    st_shared_v4(a_base + tc::sw128_chunk(kRows, (uint32_t)r, kb, c), w[0], w[1], w[2], w[3]);
    st_shared_v4(a_base + tc::sw128_chunk(kRows, (uint32_t)r, kb, c + 1), w[4], w[5], w[6], w[7]);
}
// Sum 32 per-lane values over the warp by recursive halving: on return lane l holds the warp's
// total of value l (31 shuffles).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = lane & s;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = up ? v[i] : v[i + s];
            const float keep = up ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// Control block of a tile kernel in shared memory.
struct Ctl {
    uint64_t full[kStages], empty[kStages], mma_done, a_ready[2], tmem_free, drain, g_full, mk_full[2], b_full;
    uint32_t tmem;
    volatile int abort;
};

__device__ __forceinline__ void raise_abort(Ctl* ctl, unsigned int* err) {
    ctl->abort = 1;
    atomicOr(err, kMlpTimeoutBit);
}
__device__ __forceinline__ bool wait_or_abort(Ctl* ctl, uint64_t* bar, uint32_t parity, unsigned int* err) {
    if (ctl->abort) return false;
    if (tc::mbar_wait(bar, parity, kWaitNs)) return true;
    raise_abort(ctl, err);
    return false;
}

// Producers (warps 0 and 10, one thread each; `part` 0 or 1): stream the schedule's weight blocks
// for every tile of this block through the stage ring, each producer one half of every block
// (the bulk-copy rate per issuing thread is about half of what the SM's shared memory can take
// in); a stage is full when both halves have landed.  At the end wait for the copies in flight.
__device__ void produce_weights(Ctl* ctl, uint8_t* sW, const uint8_t* img, const Sched* S, int tiles,
                                unsigned int* err, int part) {
    uint32_t it = 0;
    for (int tile = blockIdx.x; tile < tiles && !ctl->abort; tile += gridDim.x) {
        for (int j = 0; j < S->n; ++j, ++it) {
            const uint32_t stage = it % kStages, round = it / kStages;
            if (round > 0 && !wait_or_abort(ctl, &ctl->empty[stage], (round - 1) & 1u, err)) goto drain;
            const uint32_t h0 = S->b[j].bytes / 32u * 16u;  // first half, a multiple of 16 bytes
            const uint32_t off = part ? h0 : 0u, bytes = part ? S->b[j].bytes - h0 : h0;
            tc::mbar_arrive_expect_tx(&ctl->full[stage], bytes);
            if (bytes) tc::bulk_g2s(sW + stage * kWBlock + off, img + S->b[j].off + off, bytes, &ctl->full[stage]);
        }
    }
drain:
    for (uint32_t k = it > (uint32_t)kStages ? it - kStages : 0u; k < it; ++k)
        tc::mbar_wait(&ctl->full[k % kStages], (k / kStages) & 1u, kWaitNs);
}

// MMA issuer (warp 1, one thread): for every tile, the schedule's groups, each after the
// epilogue has its A operand ready; a stage is released when its MMAs complete, a group's end is
// signalled on mma_done.  At the end, the MMAs in flight are waited for.  The schedule is expanded
// at compile time (every block's A K-block, steps, N, accumulator column and flags are constants):
// a tcgen05.mma takes about as long to issue as to run, so the issuing thread keeps nothing but
// the MMAs, the commits and one test of each stage's barrier between them.
// The issuer's barrier counters: stage ring position, a_ready[0], a_ready[1] and g_full phases.
struct IssueCount {
    uint32_t it, ar0, ar1, gr;
};
template <bool BWD, int J>
__device__ __forceinline__ bool issue_block(Ctl* ctl, IssueCount& n, uint64_t adesc0, uint64_t wdesc0, uint32_t tmem,
                                            unsigned int* err) {
    constexpr Blk b = (BWD ? make_bwd() : make_fwd()).b[J];
    constexpr uint32_t idesc = tc::idesc_bf16(kRows, b.n);
    if constexpr (b.wait != kWaitNone) {  // the A operand comes from the epilogue or the encoding's copy
        uint64_t* bar = b.wait == kWaitGamma ? &ctl->g_full : b.wait == kWaitHalf0 ? &ctl->a_ready[0] : &ctl->a_ready[1];
        uint32_t& ph = b.wait == kWaitGamma ? n.gr : b.wait == kWaitHalf0 ? n.ar0 : n.ar1;
        if (!wait_or_abort(ctl, bar, ph & 1u, err)) return false;
        ++ph;
        tc::fence_after_sync();
    }
    const uint32_t stage = n.it % kStages;
    if (!tc::mbar_try_wait(&ctl->full[stage], (n.it / kStages) & 1u) &&
        !wait_or_abort(ctl, &ctl->full[stage], (n.it / kStages) & 1u, err))
        return false;
    tc::fence_after_sync();
    // descriptor start addresses are in 16-byte units
    const uint64_t ad = adesc0 + (uint64_t)((b.akb * kABlock) >> 4);
    const uint64_t bd = wdesc0 + (uint64_t)((stage * kWBlock) >> 4);
#pragma unroll
    for (int k = 0; k < b.steps; ++k)
        tc::mma_bf16(tmem + b.dcol, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (b.first && k == 0) ? 0u : 1u);
    tc::mma_commit(&ctl->empty[stage]);
    if (b.last) tc::mma_commit(&ctl->mma_done);
    ++n.it;
    return true;
}
template <bool BWD, int... J>
__device__ __forceinline__ bool issue_tile(Ctl* ctl, IssueCount& n, uint64_t adesc0, uint64_t wdesc0, uint32_t tmem,
                                           unsigned int* err, std::integer_sequence<int, J...>) {
    return (issue_block<BWD, J>(ctl, n, adesc0, wdesc0, tmem, err) && ...);
}
template <bool BWD>
__device__ void issue_mmas(Ctl* ctl, uint8_t* sA, uint8_t* sW, int tiles, uint32_t tmem, unsigned int* err) {
    constexpr int nblk = (BWD ? make_bwd() : make_fwd()).n;
    IssueCount n{0u, 0u, 0u, 0u};
    const uint64_t adesc0 = tc::desc_sw128(tc::smem_u32(sA)), wdesc0 = tc::desc_sw128(tc::smem_u32(sW));
    for (int tile = blockIdx.x; tile < tiles && !ctl->abort; tile += gridDim.x)
        if (!issue_tile<BWD>(ctl, n, adesc0, wdesc0, tmem, err, std::make_integer_sequence<int, nblk>{})) break;
    tc::mma_commit(&ctl->drain);
    tc::mbar_wait(&ctl->drain, 0, kWaitNs);
}

// ---- forward ----------------------------------------------------------------------------------
struct FwdArgs {
    const float* params3;
    int64_t N;
    float t;
    const uint8_t* wimg;   // forward weight images (kFwdSched order)
    const float* bias;     // kBiasFloats
    float* d;              // [N, 16] network outputs including the head's bias
    float* params_out;     // [N, 20]
    uint8_t* ht;           // [tiles][8 layers][4 K-blocks of 16 KB] hidden activations
    const uint8_t* gt;     // [tiles][2 K-blocks of 16 KB] encoding (written by k_mlp_encode)
    uint8_t* mk;           // [tiles][8 layers][128 rows][8 words] ReLU masks
    unsigned int* err;
    int tiles;
    int vec;               // params3 / params_out rows 16-byte aligned
};

constexpr uint32_t kFwdSmem = 1024 + 6 * kABlock + kStages * kWBlock + kWidth * 4 + sizeof(Ctl);

// The epilogue warps' hand-off around an A operand that they rewrite: the copy of its previous
// contents to global memory (issued by one thread) must have read them first.
__device__ __forceinline__ void await_a_free(bool lead) {
    if (lead) tc::bulk_wait_read();
    tc::named_sync(kEpiBar, kEpiThreads);
}
// After writing A: make it visible to the tensor core, copy `nkb` K-blocks from A K-block `kb0`
// to global `dst` (one thread), and tell the MMA issuer.
__device__ __forceinline__ void publish_a(Ctl* ctl, bool lead, uint8_t* sA, int kb0, int nkb, uint8_t* dst) {
    tc::fence_proxy_async();
    tc::named_sync(kEpiBar, kEpiThreads);
    if (lead) {
        for (int k = 0; k < nkb; ++k) tc::bulk_s2g(dst + (size_t)k * kABlock, sA + (size_t)(kb0 + k) * kABlock, kABlock);
        tc::bulk_commit();
    }
    tc::fence_before_sync();
    tc::mbar_arrive(&ctl->a_ready[0]);
}
// Wait for the MMA group; every epilogue thread learns whether any of them (or another role) gave up.
__device__ __forceinline__ bool await_mma(Ctl* ctl, uint32_t parity, unsigned int* err) {
    const bool ok = wait_or_abort(ctl, &ctl->mma_done, parity, err);
    const bool stop = tc::named_sync_or(kEpiBar, kEpiThreads, !ok || ctl->abort);
    tc::fence_after_sync();
    return !stop;
}

// The encoding of every row, as the forward's gamma tiles (K-major, 128-byte swizzle: K-block 0
// features 0-63, K-block 1 features 64-79 in its first two chunks): one thread per row, one
// sincosf per coordinate and octave (Sec. 4.3: gamma(p) = (p, sin 2^k p, cos 2^k p)).
__global__ void __launch_bounds__(256) k_mlp_encode(const float* __restrict__ params3, int64_t N, float t, int tiles,
                                                    uint8_t* __restrict__ gt) {
    pdl_enter();
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (int64_t)tiles * kRows) return;
    float g[kInPad];
#pragma unroll
    for (int c = 0; c < kInPad; ++c) g[c] = 0.f;
    if (row < N) {
        float mu[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) mu[j] = g[j] = params3[row * WIPES_P3D + j];
#pragma unroll
        for (int k = 0; k < kLx; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) sincosf(mu[j] * (float)(1 << k), &g[3 + 6 * k + j], &g[6 + 6 * k + j]);
        g[3 + 6 * kLx] = t;
#pragma unroll
        for (int k = 0; k < kLt; ++k) sincosf(t * (float)(1 << k), &g[4 + 6 * kLx + 2 * k], &g[5 + 6 * kLx + 2 * k]);
    }
    uint8_t* base = gt + (size_t)(row / kRows) * kGtTile;
    const uint32_t r = (uint32_t)(row % kRows);
#pragma unroll
    for (int c = 0; c < kInPad / 8; ++c)
        *reinterpret_cast<uint4*>(base + tc::sw128_chunk(kRows, r, (uint32_t)c / 8u, (uint32_t)c % 8u)) =
            make_uint4(pack_bf16(g[8 * c], g[8 * c + 1]), pack_bf16(g[8 * c + 2], g[8 * c + 3]),
                       pack_bf16(g[8 * c + 4], g[8 * c + 5]), pack_bf16(g[8 * c + 6], g[8 * c + 7]));
}

// dL/dmu += the encoding's backward: d/dx (x, sin(2^k x), cos(2^k x)) = (1, 2^k cos, -2^k sin), from
// dgamma [N, 80] (fp32, the skip layer's and layer 0's products summed)
__global__ void __launch_bounds__(256) k_mlp_encode_backward(const float* __restrict__ params3, int64_t N,
                                                             const float* __restrict__ dgam,
                                                             float* __restrict__ g_params3) {
    pdl_enter();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float dg[64];
    const float4* src = reinterpret_cast<const float4*>(dgam + i * kInPad);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 v = src[q];
        dg[4 * q] = v.x;
        dg[4 * q + 1] = v.y;
        dg[4 * q + 2] = v.z;
        dg[4 * q + 3] = v.w;
    }
    float gm[3] = {dg[0], dg[1], dg[2]};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float x = params3[i * WIPES_P3D + j];
#pragma unroll
        for (int k = 0; k < kLx; ++k) {
            const float f = (float)(1 << k);
            float sn, cs;
            sincosf(f * x, &sn, &cs);
            gm[j] += f * (dg[3 + 6 * k + j] * cs - dg[6 + 6 * k + j] * sn);
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) g_params3[i * WIPES_P3D + j] += gm[j];
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_fwd(const __grid_constant__ FwdArgs P) {
    pdl_enter();  // inputs written by the previous kernel on the stream
    extern __shared__ uint8_t smem_raw[];
    __shared__ Sched s_sched;
    if (threadIdx.x < kMaxBlk) s_sched.b[threadIdx.x] = c_fwd.b[threadIdx.x];
    if (threadIdx.x == 0) s_sched.n = c_fwd.n;
    uint8_t* sA = align1024(smem_raw);        // 6 K-blocks: h (0-3), gamma (4-5)
    uint8_t* sW = sA + 6 * kABlock;           // stage ring
    float* s_bias = reinterpret_cast<float*>(sW + kStages * kWBlock);  // the current hidden layer's bias
    Ctl* ctl = reinterpret_cast<Ctl*>(s_bias + kWidth);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&ctl->full[s], 2);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        tc::mbar_init(&ctl->mma_done, 1);
        tc::mbar_init(&ctl->a_ready[0], 1);
        tc::mbar_init(&ctl->a_ready[1], 1);
        tc::mbar_init(&ctl->tmem_free, 1);
        tc::mbar_init(&ctl->drain, 1);
        tc::mbar_init(&ctl->g_full, 1);
        tc::mbar_init(&ctl->b_full, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&ctl->tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 || warp == kProducer2) {
        if (lane == 0) produce_weights(ctl, sW, P.wimg, &s_sched, P.tiles, P.err, warp == kProducer2);
    } else if (warp == 1) {
        if (lane == 0) issue_mmas<false>(ctl, sA, sW, P.tiles, tmem, P.err);
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; warps 2-5 own columns 0-127, 6-9 128-255
        const int ew = warp - 2, q = warp & 3, half = ew >> 2, r = q * 32 + lane;
        const bool lead = ew == 0 && lane == 0;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t a0 = tc::smem_u32(sA);
        uint32_t md = 0, ng = 0;
        // the bias copies are issued by another thread than the lead, whose bulk copies queue behind
        // the activation stores it issues
        const bool blead = ew == 1 && lane == 0;
        uint32_t bfills = 0, bused = 0;  // bias copies issued (blead) and waited for (every thread)
        auto fetch_bias = [&](int l) {
            tc::fence_proxy_async();  // the previous layer's bias was read by the generic proxy
            tc::mbar_arrive_expect_tx(&ctl->b_full, kWidth * 4);
            tc::bulk_g2s(s_bias, P.bias + (size_t)l * kWidth, kWidth * 4, &ctl->b_full);
            ++bfills;
        };
        for (int tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
            const int64_t row = (int64_t)tile * kRows + r;
            const bool valid = row < P.N;
            // the tile's encoding (written by k_mlp_encode) into A K-blocks 4 and 5, and layer 0's
            // bias into s_bias (each hidden layer's bias is copied there once the previous layer's
            // epilogue has read its own, so it lands while the layer's MMAs run)
            // (the MMA issuer waits for the encoding's copy itself; every tensor-memory load of the
            // previous tile precedes await_a_free's barrier, after which the copy is issued)
            tc::fence_before_sync();
            await_a_free(lead);
            if (lead) {
                tc::mbar_arrive_expect_tx(&ctl->g_full, kGtTile);
                tc::bulk_g2s(sA + 4 * kABlock, P.gt + (size_t)tile * kGtTile, kGtTile, &ctl->g_full);
                ++ng;
            }
            if (blead) fetch_bias(0);
            for (int l = 0; l <= kHidden; ++l) {
                if (!await_mma(ctl, md & 1u, P.err)) goto done;
                ++md;
                if (l == kHidden) {
                    // the head: 16 fp32 outputs (13 used) plus the bias, and the deformed record
                    if (half == 0) {
                        uint32_t v[16];
                        tc::tmem_ld16(tl, v);
                        tc::tmem_wait_ld();
                        float e[kOutPad];
#pragma unroll
                        for (int j = 0; j < kOutPad; ++j) e[j] = __uint_as_float(v[j]) + __ldg(&P.bias[kHidden * kWidth + j]);
                        if (valid) {
                            float4* dr = reinterpret_cast<float4*>(P.d + row * kOutPad);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                dr[j] = make_float4(e[4 * j], e[4 * j + 1], e[4 * j + 2], e[4 * j + 3]);
                            float p[WIPES_P3D], o[WIPES_P3D];
                            if (P.vec) load_row<true, WIPES_P3D>(p, P.params3 + row * WIPES_P3D);
                            else load_row<false, WIPES_P3D>(p, P.params3 + row * WIPES_P3D);
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
                            if (P.vec) store_row<true, WIPES_P3D>(P.params_out + row * WIPES_P3D, o);
                            else store_row<false, WIPES_P3D>(P.params_out + row * WIPES_P3D, o);
                        }
                    }
                    tc::fence_before_sync();
                    break;
                }
                // this layer's bias in s_bias (a wait that runs out raises the abort flag, and the
                // next await_mma takes every epilogue thread out together)
                (void)wait_or_abort(ctl, &ctl->b_full, bused & 1u, P.err);
                ++bused;
                await_a_free(lead);
                // bias (packed f32x2 add), ReLU and bfloat16 rounding (one instruction per pair), 64
                // columns at a time: both tensor-memory loads are in flight before the one wait
                const float4* b4 = reinterpret_cast<const float4*>(s_bias + half * 128);
                const uint32_t tacc = tl + (uint32_t)(l & 1) * (uint32_t)kWidth;  // layer l's accumulator
                uint8_t* hdst = P.ht + (size_t)tile * kHtTile + (size_t)l * kHtLayer;
#pragma unroll 1
                for (int cp = 0; cp < 2; ++cp) {
                    // pass cp writes A K-block cp (warps 2-5) and K-block cp + 2 (warps 6-9)
                    const int c = half * 4 + 2 * cp;
                    uint32_t v0[32], v1[32];
                    tc::tmem_ld32(tacc + 32u * c, v0);
                    tc::tmem_ld32(tacc + 32u * (c + 1), v1);
                    float4 b[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) b[j] = b4[cp * 16 + j];
                    tc::tmem_wait_ld();
                    uint32_t w[32];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const uint32_t* v = j < 8 ? v0 + 4 * j : v1 + 4 * (j - 8);
                        const f2 z0 = f2_add(f2_pack(__uint_as_float(v[0]), __uint_as_float(v[1])), f2_pack(b[j].x, b[j].y));
                        const f2 z1 = f2_add(f2_pack(__uint_as_float(v[2]), __uint_as_float(v[3])), f2_pack(b[j].z, b[j].w));
                        w[2 * j] = pack_bf16_relu(f2_lo(z0), f2_hi(z0));
                        w[2 * j + 1] = pack_bf16_relu(f2_lo(z1), f2_hi(z1));
                    }
                    store_a16(a0, r, 32 * c, w);
                    store_a16(a0, r, 32 * c + 16, w + 8);
                    store_a16(a0, r, 32 * c + 32, w + 16);
                    store_a16(a0, r, 32 * c + 48, w + 24);
                    // the ReLU masks of these 64 columns for the backward (the ReLU output is +0 or
                    // positive, so a nonzero half is a positive one)
                    uint32_t m0 = 0u, m1 = 0u;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        m0 |= __vcmpne2(w[j], 0u) & (0x00010001u << j);
                        m1 |= __vcmpne2(w[16 + j], 0u) & (0x00010001u << j);
                    }
                    *reinterpret_cast<uint2*>(P.mk + ((size_t)tile * kHidden + l) * kMkLayer + (size_t)r * 32u +
                                              (size_t)c * 4u) = make_uint2(m0, m1);
                    // publish this half of the next layer's A operand: the next layer's products on
                    // it start while the other half is computed
                    tc::fence_proxy_async();
                    tc::fence_before_sync();
                    tc::named_sync(kEpiBar, kEpiThreads);
                    if (lead) {
                        tc::bulk_s2g(hdst + (size_t)cp * kABlock, sA + (size_t)cp * kABlock, kABlock);
                        tc::bulk_s2g(hdst + (size_t)(cp + 2) * kABlock, sA + (size_t)(cp + 2) * kABlock, kABlock);
                        tc::bulk_commit();
                        tc::mbar_arrive(&ctl->a_ready[cp]);
                    }
                }
                // every thread has read s_bias (the second publish's barrier): the next layer's bias
                if (blead && l + 1 < kHidden) fetch_bias(l + 1);
            }
        }
    done:
        if (blead)
            for (; bused < bfills; ++bused) tc::mbar_wait(&ctl->b_full, bused & 1u, kWaitNs);  // copies still in flight
        if (lead) {
            if (ng > 0) tc::mbar_wait(&ctl->g_full, (ng - 1u) & 1u, kWaitNs);  // the last encoding copy
            tc::bulk_wait_all();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// ---- backward (data) ---------------------------------------------------------------------------
struct BwdArgs {
    const float* params3;
    int64_t N;
    const uint8_t* wimg;   // backward weight images (kBwdSched order)
    const float* d;        // [N, 16]
    const float* g_out;    // [N, 20]
    float* g_params3;      // [N, 20]
    int accumulate;
    const uint8_t* mk;     // the forward's ReLU masks (kMkTile per tile)
    uint8_t* dzt;          // [tiles][8 layers][4 K-blocks of 16 KB] dz
    uint8_t* ddt;          // [tiles][1 K-block of 16 KB] dL/dd
    float* dgam;           // [N, 80] dL/dgamma (fp32), for k_mlp_encode_backward
    float* g_theta;        // bias gradients are added here (atomics, one per entry and block)
    unsigned int* err;
    int tiles;
    int vec;
};

constexpr uint32_t kBwdSmem = 1024 + 4 * kABlock + kStages * kWBlock + 2 * kMkLayer + kBiasFloats * 4 + sizeof(Ctl);

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_bwd(const __grid_constant__ BwdArgs P) {
    pdl_enter();  // inputs written by the previous kernel on the stream
    extern __shared__ uint8_t smem_raw[];
    __shared__ Sched s_sched;
    if (threadIdx.x < kMaxBlk) s_sched.b[threadIdx.x] = c_bwd.b[threadIdx.x];
    if (threadIdx.x == 0) s_sched.n = c_bwd.n;
    uint8_t* sA = align1024(smem_raw);        // 4 K-blocks: dd (K-block 0, 16 columns) or dz
    uint8_t* sW = sA + 4 * kABlock;
    uint8_t* sMk = sW + kStages * kWBlock;     // two slots of a layer's ReLU masks (layer l in slot l & 1)
    float* s_db = reinterpret_cast<float*>(sMk + 2 * kMkLayer);  // bias gradients of this block
    Ctl* ctl = reinterpret_cast<Ctl*>(s_db + kBiasFloats);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&ctl->full[s], 2);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        tc::mbar_init(&ctl->mma_done, 1);
        tc::mbar_init(&ctl->a_ready[0], kEpiThreads);
        tc::mbar_init(&ctl->a_ready[1], 1);
        tc::mbar_init(&ctl->tmem_free, kEpiThreads);
        tc::mbar_init(&ctl->drain, 1);
        tc::mbar_init(&ctl->mk_full[0], 1);
        tc::mbar_init(&ctl->mk_full[1], 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < kBiasFloats; i += blockDim.x) s_db[i] = 0.f;
    if (warp == 1) {
        tc::tmem_alloc(&ctl->tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0 || warp == kProducer2) {
        if (lane == 0) produce_weights(ctl, sW, P.wimg, &s_sched, P.tiles, P.err, warp == kProducer2);
    } else if (warp == 1) {
        if (lane == 0) issue_mmas<true>(ctl, sA, sW, P.tiles, tmem, P.err);
    } else {
        const int ew = warp - 2, q = warp & 3, half = ew >> 2, r = q * 32 + lane;
        const bool lead = ew == 0 && lane == 0;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t a0 = tc::smem_u32(sA);
        uint32_t md = 0;
        // one thread (not the lead, whose bulk copies queue behind the dz stores it issues) copies
        // each layer's masks into slot l & 1 one layer ahead: fills[s] counts the copies issued into
        // slot s (by mlead), used[s] those waited for (by every thread)
        const bool mlead = ew == 1 && lane == 0;
        uint32_t fills[2] = {0u, 0u}, used[2] = {0u, 0u};
        auto fetch_masks = [&](int tile, int l) {
            const int slot = l & 1;
            tc::fence_proxy_async();  // the slot's previous masks were read by the generic proxy
            tc::mbar_arrive_expect_tx(&ctl->mk_full[slot], kMkLayer);
            tc::bulk_g2s(sMk + (size_t)slot * kMkLayer, P.mk + ((size_t)tile * kHidden + l) * kMkLayer, kMkLayer,
                         &ctl->mk_full[slot]);
            ++fills[slot];
        };
        for (int tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
            const int64_t row = (int64_t)tile * kRows + r;
            const bool valid = row < P.N;
            if (mlead) fetch_masks(tile, kHidden - 1);
            await_a_free(lead);
            if (half == 0) {
                // the record update's backward: dL/dd (rounded: the head's product operand) and the
                // direct part of dL/dparams3
                float gd[kOutPad];
#pragma unroll
                for (int k = 0; k < kOutPad; ++k) gd[k] = 0.f;
                if (valid) {
                    float p[WIPES_P3D], e[kOutPad], g[WIPES_P3D], gp[WIPES_P3D];
                    if (P.vec) {
                        load_row<true, WIPES_P3D>(p, P.params3 + row * WIPES_P3D);
                        load_row<true, WIPES_P3D>(g, P.g_out + row * WIPES_P3D);
                    } else {
                        load_row<false, WIPES_P3D>(p, P.params3 + row * WIPES_P3D);
                        load_row<false, WIPES_P3D>(g, P.g_out + row * WIPES_P3D);
                    }
                    load_row<true, kOutPad>(e, P.d + row * kOutPad);
#pragma unroll
                    for (int k = 0; k < WIPES_P3D; ++k) gp[k] = g[k];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float es = expf(e[7 + k]);
                        gd[k] = g[k];
                        gd[7 + k] = g[3 + k] * p[3 + k] * es;
                        gd[10 + k] = g[10 + k];
                        gp[3 + k] = g[3 + k] * es;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) gd[3 + k] = g[6 + k];
                    float* go = P.g_params3 + row * WIPES_P3D;
                    if (P.accumulate) {
                        float prev[WIPES_P3D];
                        if (P.vec) load_row<true, WIPES_P3D>(prev, go);
                        else load_row<false, WIPES_P3D>(prev, go);
#pragma unroll
                        for (int k = 0; k < WIPES_P3D; ++k) gp[k] = prev[k] + gp[k];
                    }
                    if (P.vec) store_row<true, WIPES_P3D>(go, gp);
                    else store_row<false, WIPES_P3D>(go, gp);
                }
                uint32_t w[8];
                float s32[32];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    w[j] = pack_bf16(gd[2 * j], gd[2 * j + 1]);
                    s32[2 * j] = bf16_lo(w[j]);
                    s32[2 * j + 1] = bf16_hi(w[j]);
                }
#pragma unroll
                for (int j = 16; j < 32; ++j) s32[j] = 0.f;
                store_a16(a0, r, 0, w);
                const float tot = warp_reduce_scatter32(s32);
                if (lane < kOutPad) atomicAdd(&s_db[kHidden * kWidth + lane], tot);
            }
            publish_a(ctl, lead, sA, 0, 1, P.ddt + (size_t)tile * kDdTile);
            // dz_l = dh_l (rounded) where h_l > 0, for l = 7 .. 0; then dgamma
            for (int l = kHidden - 1; l >= -1; --l) {
                if (!await_mma(ctl, md & 1u, P.err)) goto done;
                ++md;
                if (l < 0) {
                    // dgamma (columns 256 .. 335: the skip layer's part plus layer 0's), written out for
                    // k_mlp_encode_backward
                    if (half == 0) {
                        float4* dst = reinterpret_cast<float4*>(P.dgam + row * kInPad);
#pragma unroll 1
                        for (int c0 = 0; c0 < kInPad; c0 += 16) {
                            uint32_t v[16];
                            tc::tmem_ld16(tl + 256u + (uint32_t)c0, v);
                            tc::tmem_wait_ld();
                            if (valid)
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    dst[c0 / 4 + j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                                  __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                        }
                    }
                    tc::fence_before_sync();
                    break;
                }
                // the ReLU mask of h_l for this row (the forward wrote it, the lead copied it into
                // slot l & 1 a layer ago): every thread waits for the copy, the lead then fetches the
                // next layer's into the other slot (read by every thread before this layer's
                // await_mma barrier)
                {
                    const int slot = l & 1;
                    const bool ok = wait_or_abort(ctl, &ctl->mk_full[slot], used[slot] & 1u, P.err);
                    ++used[slot];
                    if (mlead && ok && l > 0) fetch_masks(tile, l - 1);
                }
                await_a_free(lead);
                const uint4 mw4 = *reinterpret_cast<const uint4*>(sMk + (size_t)(l & 1) * kMkLayer + (size_t)r * 32u +
                                                                 (size_t)half * 16u);
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {
                    const int c = half * 4 + cc;
                    const uint32_t mword = cc == 0 ? mw4.x : cc == 1 ? mw4.y : cc == 2 ? mw4.z : mw4.w;
                    uint32_t v[32];
                    tc::tmem_ld32(tl + 32u * c, v);
                    tc::tmem_wait_ld();
                    uint32_t w[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const uint32_t keep = ((mword >> j) & 0x00010001u) * 0xFFFFu;
                        w[j] = pack_bf16(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1])) & keep;
                    }
                    store_a16(a0, r, 32 * c, w);
                    store_a16(a0, r, 32 * c + 16, w + 8);
                }
                publish_a(ctl, lead, sA, 0, 4, P.dzt + (size_t)tile * kHtTile + (size_t)l * kHtLayer);
                // the bias gradient of layer l: the column sums of dz over the tile's rows, read back
                // from the A operand just published while the next product runs (thread t sums
                // columns 2 (t % 128), + 1 over rows 64 (t / 128) .. + 63; the A operand is next
                // rewritten only after the await_mma barrier that every thread reaches)
                {
                    const uint32_t t = (uint32_t)(ew * 32 + lane), col = 2u * (t & 127u), rh = t >> 7;
                    const uint32_t kb = col / 64u, cch = (col % 64u) / 8u, e = col % 8u;
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
                    for (uint32_t i = 0; i < 64u; ++i) {
                        const uint32_t v2 = *reinterpret_cast<const uint32_t*>(
                            sA + tc::sw128_chunk(kRows, rh * 64u + i, kb, cch) + e * 2u);
                        s0 += bf16_lo(v2);
                        s1 += bf16_hi(v2);
                    }
                    atomicAdd(&s_db[l * kWidth + (int)col], s0);
                    atomicAdd(&s_db[l * kWidth + (int)col + 1], s1);
                }
            }
        }
    done:
        if (mlead)  // masks copied into a slot but not waited for (a role gave up): let the copies land
            for (int sl = 0; sl < 2; ++sl)
                for (; used[sl] < fills[sl]; ++used[sl]) tc::mbar_wait(&ctl->mk_full[sl], used[sl] & 1u, kWaitNs);
        if (lead) tc::bulk_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
    // the block's bias gradients (hidden layers: [l][256]; head: 13 of 16)
    for (int i = threadIdx.x; i < kBiasFloats; i += blockDim.x) {
        const int l = i / kWidth, j = i % kWidth;
        if (l < kHidden) atomicAdd(&P.g_theta[layer_offset(l) + (int64_t)layer_out(l) * layer_in(l) + j], s_db[i]);
        else if (j < kOut) atomicAdd(&P.g_theta[layer_offset(kHidden) + (int64_t)kOut * kWidth + j], s_db[i]);
    }
}

// ---- weight gradients ----------------------------------------------------------------------------
// Ten products over the rows: part 0 dW_0 = dz_0^T gamma; 1-4 dW_l = dz_l^T h_{l-1}; 5 the skip
// layer's h4 columns (dz_5^T h_4), 6 its gamma columns (dz_5^T gamma); 7, 8 dW_6, dW_7; 9 the head,
// taken transposed (h_7^T dd: M = the 256 inputs, N = the 16 padded outputs).  Each part is split
// into `chunks` ranges of tiles; an item = (part, chunk) accumulates its range in tensor memory
// (two 128-row halves of M, at columns 0 and 256) and writes its 256 x N partial.  Both operands
// are the tile copies written by the tile kernels, read MN-major: a stage holds 64 rows (K) of
// every 64-feature group (8 KB each; A: 4 groups, B: N / 64 rounded up).
constexpr int kParts = 10;
struct WgArgs {
    const uint8_t* ht;
    const uint8_t* gt;
    const uint8_t* dzt;
    const uint8_t* ddt;
    float* partial;  // [parts * chunks][256][256]
    int tiles, chunks;
    unsigned int* err;
};
struct WgPart {
    const uint8_t* a;  // tile 0 of A's tensor
    const uint8_t* b;
    uint32_t a_tile, b_tile, n, nb;  // tile strides, N, B's 64-feature groups
};
__device__ __forceinline__ WgPart wg_part(const WgArgs& P, int p) {
    WgPart w;
    w.a_tile = kHtTile;
    if (p == kParts - 1) {
        w.a = P.ht + 7u * kHtLayer;
        w.b = P.ddt;
        w.b_tile = kDdTile;
        w.n = kOutPad;
        w.nb = 1;
        return w;
    }
    const int la = p == 0 ? 0 : p <= 4 ? p : p <= 6 ? 5 : p - 1;  // dz layer of parts 0-8
    w.a = P.dzt + (size_t)la * kHtLayer;
    if (p == 0 || p == 6) {
        w.b = P.gt;
        w.b_tile = kGtTile;
        w.n = kInPad;
        w.nb = 2;
    } else {
        w.b = P.ht + (size_t)(la - 1) * kHtLayer;  // h_{l-1}; part 5 reads h_4
        w.b_tile = kHtTile;
        w.n = kWidth;
        w.nb = 4;
    }
    return w;
}

constexpr uint32_t kGroupRows = 64;                  // K rows per stage
constexpr uint32_t kGroupBytes = kGroupRows * 128;   // one 64-feature group of them: 8 KB
constexpr uint32_t kWgStage = 8 * kGroupBytes;       // A (4 groups) and B (up to 4 groups): 64 KB
constexpr int kWgStages = 3;
constexpr uint32_t kWgSmem = 1024 + kWgStages * kWgStage + sizeof(Ctl);

__global__ void __launch_bounds__(kWgThreads, 1) k_mlp_wgrad(const __grid_constant__ WgArgs P) {
    pdl_enter();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sW = align1024(smem_raw);
    Ctl* ctl = reinterpret_cast<Ctl*>(sW + kWgStages * kWgStage);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = kParts * P.chunks;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        tc::mbar_init(&ctl->mma_done, 1);
        tc::mbar_init(&ctl->a_ready[0], 1);
        tc::mbar_init(&ctl->a_ready[1], 1);
        tc::mbar_init(&ctl->tmem_free, 128);
        tc::mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&ctl->tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = ctl->tmem;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int item = blockIdx.x; item < items && !ctl->abort; item += gridDim.x) {
                const WgPart w = wg_part(P, item / P.chunks);
                const int c = item % P.chunks;
                const int t0 = (int)((int64_t)c * P.tiles / P.chunks), t1 = (int)((int64_t)(c + 1) * P.tiles / P.chunks);
                for (int t = t0; t < t1; ++t)
                    for (uint32_t kc = 0; kc < kRows / kGroupRows; ++kc, ++it) {
                        const uint32_t stage = it % kWgStages, round = it / kWgStages;
                        if (round > 0 && !wait_or_abort(ctl, &ctl->empty[stage], (round - 1) & 1u, P.err)) goto pdrain;
                        tc::mbar_arrive_expect_tx(&ctl->full[stage], (4 + w.nb) * kGroupBytes);
                        uint8_t* dst = sW + stage * kWgStage;
                        const uint8_t* a = w.a + (size_t)t * w.a_tile + kc * kGroupBytes;
                        const uint8_t* b = w.b + (size_t)t * w.b_tile + kc * kGroupBytes;
                        for (int g = 0; g < 4; ++g)
                            tc::bulk_g2s(dst + g * kGroupBytes, a + (size_t)g * kABlock, kGroupBytes, &ctl->full[stage]);
                        for (uint32_t g = 0; g < w.nb; ++g)
                            tc::bulk_g2s(dst + (4 + g) * kGroupBytes, b + (size_t)g * kABlock, kGroupBytes,
                                         &ctl->full[stage]);
                    }
            }
        pdrain:
            for (uint32_t k = it > (uint32_t)kWgStages ? it - kWgStages : 0u; k < it; ++k)
                tc::mbar_wait(&ctl->full[k % kWgStages], (k / kWgStages) & 1u, kWaitNs);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, nitem = 0;
            const uint32_t w0 = tc::smem_u32(sW);
            for (int item = blockIdx.x; item < items && !ctl->abort; item += gridDim.x, ++nitem) {
                const WgPart w = wg_part(P, item / P.chunks);
                const int c = item % P.chunks;
                const int t0 = (int)((int64_t)c * P.tiles / P.chunks), t1 = (int)((int64_t)(c + 1) * P.tiles / P.chunks);
                // the accumulator is free once the epilogue has read the previous item's
                if (nitem > 0) {
                    if (!wait_or_abort(ctl, &ctl->tmem_free, (nitem - 1) & 1u, P.err)) goto mdrain;
                    tc::fence_after_sync();
                }
                const uint32_t idesc = tc::idesc_bf16(kRows, (int)w.n, true, true);
                bool first = true;
                for (int t = t0; t < t1; ++t)
                    for (uint32_t kc = 0; kc < kRows / kGroupRows; ++kc, ++it) {
                        const uint32_t stage = it % kWgStages;
                        if (!wait_or_abort(ctl, &ctl->full[stage], (it / kWgStages) & 1u, P.err)) goto mdrain;
                        tc::fence_after_sync();
                        const uint32_t sa = w0 + stage * kWgStage, sb = sa + 4 * kGroupBytes;
                        for (int h = 0; h < 2; ++h)
                            for (int k = 0; k < 4; ++k)  // 16 rows (two 8-row groups) per step
                                tc::mma_bf16(tmem + (uint32_t)h * 256u,
                                             tc::desc_sw128_mn(sa + (uint32_t)h * 2 * kGroupBytes + 2048u * k,
                                                               kGroupBytes, 1024),
                                             tc::desc_sw128_mn(sb + 2048u * k, kGroupBytes, 1024), idesc,
                                             (first && k == 0) ? 0u : 1u);
                        first = false;
                        tc::mma_commit(&ctl->empty[stage]);
                    }
                // an empty range leaves the accumulator unwritten: the epilogue writes zeros then
                tc::mma_commit(&ctl->mma_done);
            }
        mdrain:
            tc::mma_commit(&ctl->drain);
            tc::mbar_wait(&ctl->drain, 0, kWaitNs);
        }
    } else {
        const int q = warp & 3, m = q * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t nitem = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++nitem) {
            const WgPart w = wg_part(P, item / P.chunks);
            const int c = item % P.chunks;
            const bool empty_range = (int64_t)c * P.tiles / P.chunks == (int64_t)(c + 1) * P.tiles / P.chunks;
            if (!wait_or_abort(ctl, &ctl->mma_done, nitem & 1u, P.err)) break;
            tc::fence_after_sync();
            float* out = P.partial + (size_t)item * kWidth * kWidth;
            for (int h = 0; h < 2; ++h) {
                float* orow = out + (size_t)(h * kRows + m) * kWidth;
                for (uint32_t c0 = 0; c0 < w.n; c0 += 16) {
                    uint32_t v[16];
                    tc::tmem_ld16(tl + (uint32_t)h * 256u + c0, v);
                    tc::tmem_wait_ld();
                    float4* o4 = reinterpret_cast<float4*>(orow + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o4[j] = empty_range ? make_float4(0.f, 0.f, 0.f, 0.f)
                                            : make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                          __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&ctl->tmem_free);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// g_theta (weights) += the sum of the chunks' partials, in chunk order; one thread per weight.
__global__ void __launch_bounds__(256) k_mlp_wsum(const float* __restrict__ partial, int chunks,
                                                  float* __restrict__ g_theta) {
    pdl_enter();
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // weights in theta order: layer l, output o, input i
    int l = 0;
    int64_t rem = idx;
    while (l <= kHidden && rem >= (int64_t)layer_out(l) * layer_in(l)) {
        rem -= (int64_t)layer_out(l) * layer_in(l);
        ++l;
    }
    if (l > kHidden) return;
    const int o = (int)(rem / layer_in(l)), i = (int)(rem % layer_in(l));
    int part, row, col;
    if (l == kHidden) {
        part = kParts - 1, row = i, col = o;  // the head's product is transposed
    } else if (l == kSkipLayer) {
        if (i < kInPad) part = 6, row = o, col = i;
        else part = 5, row = o, col = i - kInPad;
    } else {
        part = l <= 4 ? l : l + 1;
        row = o, col = i;
    }
    float s = 0.f;
    for (int c = 0; c < chunks; ++c)
        s += partial[((size_t)(part * chunks + c) * kWidth + row) * kWidth + col];
    g_theta[layer_offset(l) + (int64_t)o * layer_in(l) + i] += s;
}

// Pack theta (fp32) into the weight images (bfloat16, K-major, 128-byte swizzle) and the fp32
// bias vector: one thread per 16-byte chunk of an image.
__global__ void __launch_bounds__(256) k_mlp_pack(const float* __restrict__ theta, const ImgTable tab,
                                                  uint8_t* __restrict__ img, float* __restrict__ bias) {
    pdl_enter();
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kBiasFloats) {
        const int l = (int)(idx / kWidth), j = (int)(idx % kWidth);
        float b = 0.f;
        if (l < kHidden) b = theta[layer_offset(l) + (int64_t)layer_out(l) * layer_in(l) + j];
        else if (j < kOut) b = theta[layer_offset(kHidden) + (int64_t)kOut * kWidth + j];
        bias[idx] = b;
    }
    for (int i = 0; i < tab.n; ++i) {
        const ImgDesc& d = tab.d[i];
        const int64_t chunks = (int64_t)d.rows * d.nkb * 8;
        if (idx >= chunks) {
            idx -= chunks;
            continue;
        }
        const uint32_t kb = (uint32_t)(idx / ((int64_t)d.rows * 8)), rem = (uint32_t)(idx % ((int64_t)d.rows * 8));
        const uint32_t n = rem / 8, c = rem % 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = (int)(kb * 64 + c * 8 + e);
            v[e] = 0.f;
            if ((int)n < d.nvalid && k < d.kvalid) {
                const int col = k < d.ksplit ? k + d.klo : k - d.ksplit + d.khi;
                v[e] = theta[d.src + (int64_t)n * d.sn + (int64_t)col * d.sk];
            }
        }
        uint4 w;
        w.x = pack_bf16(v[0], v[1]);
        w.y = pack_bf16(v[2], v[3]);
        w.z = pack_bf16(v[4], v[5]);
        w.w = pack_bf16(v[6], v[7]);
        *reinterpret_cast<uint4*>(img + d.dst + tc::sw128_chunk(d.rows, n, kb, c)) = w;
        return;
    }
}

int tiles_of(int64_t N) { return (int)((N + kRows - 1) / kRows); }
int chunks_of(int tiles) { return std::max(1, std::min(tiles, 30)); }

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;
void set_smem_attributes() {
    std::call_once(g_attr_once, [] {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
        g_attr_err = e;
    });
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Layout of the state buffers (mlp_sizes): theta16 = forward images, backward images, bias;
// act = h^T tiles, gamma^T tiles, ReLU mask tiles; scratch = dz^T tiles, dd^T tiles, partials.
struct ActLayout {
    size_t ht, gt, mk, total;
};
ActLayout act_layout(int64_t N) {
    const size_t tiles = (size_t)tiles_of(std::max<int64_t>(N, 1));
    ActLayout a;
    a.ht = 0;
    a.gt = tiles * kHtTile;
    a.mk = a.gt + tiles * kGtTile;
    a.total = a.mk + tiles * kMkTile;
    return a;
}
struct ScratchLayout {
    size_t dzt, ddt, partial, dgam, total;
};
ScratchLayout scratch_layout(int64_t N) {
    const int tiles = tiles_of(std::max<int64_t>(N, 1));
    ScratchLayout s;
    s.dzt = 0;
    s.ddt = (size_t)tiles * kHtTile;
    s.partial = s.ddt + (size_t)tiles * kDdTile;
    s.dgam = s.partial + (size_t)kParts * chunks_of(tiles) * kWidth * kWidth * sizeof(float);
    s.total = s.dgam + (size_t)tiles * kRows * kInPad * sizeof(float);
    return s;
}

}  // namespace

int64_t mlp_param_count() { return layer_offset(kHidden + 1); }

MlpSizes mlp_sizes(int64_t N) {
    MlpSizes z;
    z.act = act_layout(N).total;
    z.scratch = scratch_layout(N).total;
    z.out = (size_t)std::max<int64_t>(N, 1) * kOutPad * sizeof(float);
    z.theta16 = (size_t)kFwdImgBytes + kBwdImgBytes + kBiasFloats * sizeof(float);
    return z;
}

std::string mlp_forward(const float* params3, int64_t N, float t, const float* theta, void* theta16_buf, void* act,
                        float* d, float* params_out, unsigned int* err, cudaStream_t s) {
    if (N == 0) return "";
    set_smem_attributes();
    if (g_attr_err != cudaSuccess) return std::string("deformation network: ") + cudaGetErrorString(g_attr_err);
    static const ImgTable tab = make_images();
    uint8_t* img = static_cast<uint8_t*>(theta16_buf);
    float* bias = reinterpret_cast<float*>(img + kFwdImgBytes + kBwdImgBytes);
    int64_t chunks = 0;
    for (int i = 0; i < tab.n; ++i) chunks += (int64_t)tab.d[i].rows * tab.d[i].nkb * 8;
    launch_pdl(k_mlp_pack, ceil_div(std::max<int64_t>(chunks, kBiasFloats), 256), 256, 0, s, theta, tab, img, bias);
    const ActLayout a = act_layout(N);
    uint8_t* ab = static_cast<uint8_t*>(act);
    FwdArgs P;
    P.params3 = params3;
    P.N = N;
    P.t = t;
    P.wimg = img;
    P.bias = bias;
    P.d = d;
    P.params_out = params_out;
    P.ht = ab + a.ht;
    P.gt = ab + a.gt;
    P.mk = ab + a.mk;
    P.err = err;
    P.tiles = tiles_of(N);
    P.vec = ((reinterpret_cast<uintptr_t>(params3) | reinterpret_cast<uintptr_t>(params_out)) & 15u) == 0;
    launch_pdl(k_mlp_encode, ceil_div((int64_t)P.tiles * kRows, 256), 256, 0, s, params3, N, t, P.tiles, ab + a.gt);
    const int grid = std::min(P.tiles, sm_count());
    launch_pdl(k_mlp_fwd, grid, kTcThreads, kFwdSmem, s, P);
    count_launches(3);
    return "";
}

std::string mlp_backward(const float* params3, int64_t N, const void* theta16_buf, const void* act, const float* d,
                         void* scratch, const float* g_out, float* g_theta, float* g_params3, int accumulate,
                         unsigned int* err, cudaStream_t s) {
    if (N == 0) return "";
    set_smem_attributes();
    if (g_attr_err != cudaSuccess) return std::string("deformation network: ") + cudaGetErrorString(g_attr_err);
    const uint8_t* img = static_cast<const uint8_t*>(theta16_buf);
    const ActLayout a = act_layout(N);
    const ScratchLayout sl = scratch_layout(N);
    const uint8_t* ab = static_cast<const uint8_t*>(act);
    uint8_t* sb = static_cast<uint8_t*>(scratch);
    const int tiles = tiles_of(N);
    if (!accumulate) cudaMemsetAsync(g_theta, 0, sizeof(float) * (size_t)mlp_param_count(), s);
    BwdArgs B;
    B.params3 = params3;
    B.N = N;
    B.wimg = img + kFwdImgBytes;
    B.d = d;
    B.g_out = g_out;
    B.g_params3 = g_params3;
    B.accumulate = accumulate;
    B.mk = ab + a.mk;
    B.dzt = sb + sl.dzt;
    B.ddt = sb + sl.ddt;
    B.dgam = reinterpret_cast<float*>(sb + sl.dgam);
    B.g_theta = g_theta;
    B.err = err;
    B.tiles = tiles;
    B.vec = ((reinterpret_cast<uintptr_t>(params3) | reinterpret_cast<uintptr_t>(g_out) |
              reinterpret_cast<uintptr_t>(g_params3)) & 15u) == 0;
    const int n_sm = sm_count();
    launch_pdl(k_mlp_bwd, std::min(tiles, n_sm), kTcThreads, kBwdSmem, s, B);
    launch_pdl(k_mlp_encode_backward, ceil_div(N, 256), 256, 0, s, params3, N, (const float*)B.dgam, g_params3);
    WgArgs W;
    W.ht = ab + a.ht;
    W.gt = ab + a.gt;
    W.dzt = B.dzt;
    W.ddt = B.ddt;
    W.partial = reinterpret_cast<float*>(sb + sl.partial);
    W.tiles = tiles;
    W.chunks = chunks_of(tiles);
    W.err = err;
    launch_pdl(k_mlp_wgrad, std::min(kParts * W.chunks, n_sm), kWgThreads, kWgSmem, s, W);
    const int64_t nw = mlp_param_count() - (int64_t)kHidden * kWidth - kOut;  // weights (no biases)
    launch_pdl(k_mlp_wsum, ceil_div(nw, 256), 256, 0, s, (const float*)W.partial, W.chunks, g_theta);
    count_launches(4);
    return "";
}

}  // namespace wipes
