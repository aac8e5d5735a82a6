// k_field_tc.cu - the field on the 5th-generation tensor cores (FP16 or BF16
// operands, FP32 accumulation in tensor memory): hash encoding, density MLP
// (sigma = exp(h_0)), SH view encoding and colour MLP forward (steps a3-a6), and the
// recomputing backward pass with the weight gradients accumulated in tensor memory
// across a persistent block's tiles (steps a10-a11).
//
// A block owns a tile of 128 samples at a time; thread r of the block owns sample
// row r, which is TMEM lane r of every 128-row accumulator.  Each layer is one
// chain of tcgen05.mma instructions issued by thread 0 on shared-memory operands
// (layout in tc_ptx.cuh), committed to an mbarrier; the block then reads the
// accumulator rows back with tcgen05.ld, applies the activation in FP32, rounds to
// the MLP type and writes the next operand tile.  Weight gradients are M=64
// products over the tile's samples (MN-major operands of the same tiles) that keep
// accumulating in TMEM until the block has no tiles left.
//
// Gradient tiles are scaled by powers of two before rounding to the MLP type: the
// colour branch (dL/dz through the colour MLP down to its input, weights W3-W5) by
// S_c, which brings the step's largest colour seed |dL/dc| to about 2^8, and the
// density branch (from dL/dh on, weights W1-W2 and the tables) by S_d, which does the
// same for the larger of the density seeds |dL/dsigma * sigma| and the colour seeds.
// The depth term's seeds are usually far larger than the colour ones, so one shared
// scale would push the colour gradients into FP16's subnormal range.  2^8 leaves a
// factor 2^8 of headroom below FP16's largest value for the growth of the gradient
// through the layers (fan-in 64) and keeps seeds down to 2^-22 of the largest one
// normal; with 2^13 the deepest colour-branch tiles saturated in trained fields.
// FP16 encodings enter the MLP scaled by 2^8 (table values start near 1e-4, below
// FP16's normal range).  Both scales are exact and are removed in FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "encoding.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace nm {

using namespace tc;

namespace {

constexpr float kGradTarget = 256.f;  // largest scaled gradient seed (see above)

// Two values rounded to the MLP type, a in the low half: one cvt to a packed pair
// (the pair's first source operand fills the upper half).  FP16 saturates at the
// largest finite value (+-65504) instead of overflowing; RELU also maps negative
// values to zero.
template <bool BF16, bool RELU = false>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    uint32_t d;
    if constexpr (BF16) {
        if constexpr (RELU) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
        else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    } else {
        if constexpr (RELU) asm("cvt.rn.relu.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
        else asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    }
    return d;
}

template <bool BF16>
__device__ __forceinline__ uint16_t pack1(float a) {
    if constexpr (BF16) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(a));
    } else {
        return __half_as_ushort(__float2half_rn(fminf(fmaxf(a, -65504.f), 65504.f)));
    }
}

// Row r (of 128) of a tile with C columns, from C floats.
template <bool BF16, int C>
__device__ __forceinline__ void store_row(uint8_t* tile, int r, const float* v) {
#pragma unroll
    for (int g = 0; g < C / 8; ++g) {
        uint4 q;
        q.x = pack2<BF16>(v[8 * g + 0], v[8 * g + 1]);
        q.y = pack2<BF16>(v[8 * g + 2], v[8 * g + 3]);
        q.z = pack2<BF16>(v[8 * g + 4], v[8 * g + 5]);
        q.w = pack2<BF16>(v[8 * g + 6], v[8 * g + 7]);
        *reinterpret_cast<uint4*>(tile + tile_offset(r, 8 * g, 128)) = q;
    }
}

// C columns of row r of a 128-row tile from C floats, starting at column c0
// (RELU: max(v, 0) is stored).
template <bool BF16, int C, bool RELU = false>
__device__ __forceinline__ void store_row_at(uint8_t* tile, int r, int c0, const float* v) {
#pragma unroll
    for (int g = 0; g < C / 8; ++g) {
        uint4 q;
        q.x = pack2<BF16, RELU>(v[8 * g + 0], v[8 * g + 1]);
        q.y = pack2<BF16, RELU>(v[8 * g + 2], v[8 * g + 3]);
        q.z = pack2<BF16, RELU>(v[8 * g + 4], v[8 * g + 5]);
        q.w = pack2<BF16, RELU>(v[8 * g + 6], v[8 * g + 7]);
        *reinterpret_cast<uint4*>(tile + tile_offset(r, c0 + 8 * g, 128)) = q;
    }
}

// N consecutive accumulator columns of this thread's lane.
template <int N>
__device__ __forceinline__ void ld_cols(uint32_t trow, uint32_t col, float* v) {
#pragma unroll
    for (int c = 0; c < N; c += 16) tmem_ld16(trow + col + c, v + c);
    tmem_wait_ld();
}

struct Op {
    uint32_t addr, lbo, sbo, kstep;
};
// Tile with R rows used as a K-major operand (rows = M or N, columns = K).
__device__ __forceinline__ Op kmaj(const void* t, int R) {
    return Op{smem_u32(t), (uint32_t)(R / 8) * 128u, 128u, (uint32_t)(R / 8) * 256u};
}
// Tile with R rows used as an MN-major operand (rows = K, columns = M or N).
__device__ __forceinline__ Op mnmaj(const void* t, int R) {
    return Op{smem_u32(t), 128u, (uint32_t)(R / 8) * 128u, 256u};
}

__device__ __forceinline__ void gemm(uint32_t d, Op a, Op b, int ksteps, uint32_t idesc, bool acc) {
    for (int k = 0; k < ksteps; ++k)
        mma_f16(d, smem_desc(a.addr + k * a.kstep, a.lbo, a.sbo), smem_desc(b.addr + k * b.kstep, b.lbo, b.sbo),
                idesc, (acc || k > 0) ? 1u : 0u);
}

// Makes this thread's operand writes visible to the tensor core and orders its
// earlier TMEM reads before the next MMA; block-wide.
__device__ __forceinline__ void to_tensor() {
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Waits for the MMAs committed to `bar` (at most `polls` polls; 0 makes the wait
// expire at once).  After a timeout the thread stops waiting, the rest of its work is
// garbage, and the block drains its MMAs before it frees tensor memory (drain_mma).
__device__ __forceinline__ void wait_mma(uint64_t* bar, uint32_t& phase, bool& timed_out, uint32_t polls) {
    if (!timed_out) timed_out = !mbar_wait(bar, phase, polls);
    phase ^= 1u;
    fence_after_sync();
}

// After a timeout: the MMA-issuing thread commits once more, to a barrier that has
// seen no other commit, and waits for it (bounded by the default limit).  The commit
// arrives when every MMA that thread has issued has completed, so the tensor memory
// can be freed afterwards; the phases of the main barrier are not trusted (several
// of its phases may have completed while nobody waited).
__device__ __forceinline__ void drain_mma(uint64_t* drain_bar) {
    mma_commit(drain_bar);
    mbar_wait(drain_bar, 0u, kWaitPollsDefault);
    fence_after_sync();
}

// Weight tiles (MLP type) from the FP32 master weights: W1 64x32, W2 16x64,
// W3 64x32, W4 64x64, W5 padded to 16x64 (rows 3..15 zero).
template <bool BF16>
__device__ void load_weight_tiles(const float* __restrict__ mlp, uint8_t* sW1, uint8_t* sW2, uint8_t* sW3,
                                  uint8_t* sW4, uint8_t* sW5) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const float w = mlp[i];
        uint8_t* dst;
        if (i < kOffW2) {
            dst = sW1 + tile_offset(i / 32, i % 32, 64);
        } else if (i < kOffW3) {
            const int j = i - kOffW2;
            dst = sW2 + tile_offset(j / 64, j % 64, 16);
        } else if (i < kOffW4) {
            const int j = i - kOffW3;
            dst = sW3 + tile_offset(j / 32, j % 32, 64);
        } else if (i < kOffW5) {
            const int j = i - kOffW4;
            dst = sW4 + tile_offset(j / 64, j % 64, 64);
        } else {
            const int j = i - kOffW5;
            dst = sW5 + tile_offset(j / 64, j % 64, 16);
        }
        *reinterpret_cast<uint16_t*>(dst) = pack1<BF16>(w);
    }
    for (int j = 192 + threadIdx.x; j < 16 * 64; j += blockDim.x)
        *reinterpret_cast<uint16_t*>(sW5 + tile_offset(j / 64, j % 64, 16)) = 0;
}

__device__ __forceinline__ float3 sample_pos_tc(const DevCfg& c, const float* __restrict__ rays, uint32_t cap,
                                                uint32_t r, float t, float3& d) {
    const float3 o = make_float3(rays[kOx * cap + r], rays[kOy * cap + r], rays[kOz * cap + r]);
    d = make_float3(rays[kDx * cap + r], rays[kDy * cap + r], rays[kDz * cap + r]);
    return grid_pos(c, o, d, t);
}

constexpr int kW1B = 64 * 32 * 2, kW2B = 16 * 64 * 2, kW3B = 64 * 32 * 2, kW4B = 64 * 64 * 2, kW5B = 16 * 64 * 2;
constexpr int kWB = kW1B + kW2B + kW3B + kW4B + kW5B;  // 20480
constexpr int kT32 = 128 * 32 * 2, kT64 = 128 * 64 * 2, kT16 = 128 * 16 * 2;

}  // namespace

constexpr int kFwdSmem = kWB + kT32 + kT64;                            // 45056

// ------------------------------------------------------------------ forward
// One tile of the forward: samples i0 .. min(i0 + 128, i_end) - 1; thread r of the
// block owns sample row r.  smem: the weight tiles, then tA (128 x 32: X0, X3) and
// tB (128 x 64: H1, H3, H4; a layer's MMAs have completed before its output
// overwrites its input).  Returns after the tile's last MMA wait.
// kSel: row r evaluates sample sel[i0 + r] of the batch instead of i0 + r (a render's
// passes over a subset of the samples).
template <bool BF16, bool kSel = false>
__device__ __forceinline__ void fwd_tile(const DevCfg& c, const float2* __restrict__ tables,
                                         const float* __restrict__ rays, uint32_t cap,
                                         const uint32_t* __restrict__ ray_id, const float* __restrict__ ts,
                                         float4* __restrict__ sig_rgb, uint4* __restrict__ feat_out,
                                         float feat_scale, uint32_t i0, uint32_t i_end, uint8_t* smem,
                                         uint32_t tmem, uint64_t* bar, uint32_t& phase, bool& timed_out,
                                         const uint32_t* __restrict__ sel = nullptr) {
    uint8_t* sW1 = smem;
    uint8_t* sW2 = sW1 + kW1B;
    uint8_t* sW3 = sW2 + kW2B;
    uint8_t* sW4 = sW3 + kW3B;
    uint8_t* sW5 = sW4 + kW4B;
    uint8_t* tA = smem + kWB;
    uint8_t* tB = tA + kT32;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const float inv_fs = 1.f / feat_scale;
    const bool valid = i0 + tid < i_end;
    const uint32_t i = kSel ? (valid ? sel[i0 + tid] : 0u) : i0 + tid;
    float v[32];
    float3 d = make_float3(0.f, 0.f, 0.f);
    float3 x = make_float3(0.f, 0.f, 0.f);
    if (valid) x = sample_pos_tc(c, rays, cap, ray_id[i], ts[i], d);
    // one group of kGatherGroup = 4 levels = 8 features = one 16-byte chunk of the row
#pragma unroll 1
    for (int g = 0; g < kEnc / 8; ++g) {
        if (valid) {
            encode_group(c, tables, x, kGatherGroup * g, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] *= feat_scale;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = 0.f;
        }
        uint4 q;
        q.x = pack2<BF16>(v[0], v[1]);
        q.y = pack2<BF16>(v[2], v[3]);
        q.z = pack2<BF16>(v[4], v[5]);
        q.w = pack2<BF16>(v[6], v[7]);
        *reinterpret_cast<uint4*>(tA + tile_offset(tid, 8 * g, 128)) = q;
        if (!kSel && feat_out && valid) feat_out[(size_t)i * 4 + g] = q;
    }
    // layer 1: D = X0 W1^T (128 x 64)
    to_tensor();
    if (tid == 0) {
        gemm(tmem, kmaj(tA, 128), kmaj(sW1, 64), 2, idesc_f16(128, 64, BF16, false, false), false);
        mma_commit(bar);
    }
    wait_mma(bar, phase, timed_out, c.wait_polls);
#pragma unroll
    for (int h = 0; h < 64; h += 32) {  // 32-column halves keep fewer values live
        ld_cols<32>(trow, h, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] *= inv_fs;
        store_row_at<BF16, 32, true>(tB, tid, h, v);
    }
    // layer 2: y = H1 W2^T (128 x 16)
    to_tensor();
    if (tid == 0) {
        gemm(tmem, kmaj(tB, 128), kmaj(sW2, 16), 4, idesc_f16(128, 16, BF16, false, false), false);
        mma_commit(bar);
    }
    wait_mma(bar, phase, timed_out, c.wait_polls);
    ld_cols<16>(trow, 0, v);
    const float sigma = expf(fminf(v[0], kSigmaHMax));
    if (valid) sh16(d.x, d.y, d.z, v + kGeo);
    else {
#pragma unroll
        for (int k = kGeo; k < 32; ++k) v[k] = 0.f;
    }
    store_row<BF16, 32>(tA, tid, v);
    // layer 3: H3 = relu(X3 W3^T)
    to_tensor();
    if (tid == 0) {
        gemm(tmem, kmaj(tA, 128), kmaj(sW3, 64), 2, idesc_f16(128, 64, BF16, false, false), false);
        mma_commit(bar);
    }
    wait_mma(bar, phase, timed_out, c.wait_polls);
#pragma unroll
    for (int h = 0; h < 64; h += 32) {
        ld_cols<32>(trow, h, v);
        store_row_at<BF16, 32, true>(tB, tid, h, v);
    }
    // layer 4: H4 = relu(H3 W4^T)
    to_tensor();
    if (tid == 0) {
        gemm(tmem, kmaj(tB, 128), kmaj(sW4, 64), 4, idesc_f16(128, 64, BF16, false, false), false);
        mma_commit(bar);
    }
    wait_mma(bar, phase, timed_out, c.wait_polls);
#pragma unroll
    for (int h = 0; h < 64; h += 32) {
        ld_cols<32>(trow, h, v);
        store_row_at<BF16, 32, true>(tB, tid, h, v);
    }
    // layer 5: z = H4 W5^T (3 of 16 columns used)
    to_tensor();
    if (tid == 0) {
        gemm(tmem, kmaj(tB, 128), kmaj(sW5, 16), 4, idesc_f16(128, 16, BF16, false, false), false);
        mma_commit(bar);
    }
    wait_mma(bar, phase, timed_out, c.wait_polls);
    ld_cols<16>(trow, 0, v);
    if (valid) sig_rgb[i] = make_float4(sigma, sigmoidf_(v[0]), sigmoidf_(v[1]), sigmoidf_(v[2]));
}

// Tensor memory and barriers of a forward block: 64 TMEM columns (one 128 x 64 FP32
// accumulator), the MMA barrier and the drain barrier.
__device__ __forceinline__ uint32_t fwd_block_setup(uint32_t* tslot, uint64_t* bar, uint64_t* drain_bar) {
    if ((threadIdx.x >> 5) == 0) tmem_alloc(tslot, 64);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(drain_bar, 1);
        mbar_fence_init();
    }
    to_tensor();
    return *tslot;
}

// End of a forward block: after a timeout, drain the issued MMAs; free the TMEM.
__device__ __forceinline__ void fwd_block_finish(uint32_t tmem, uint64_t* drain_bar, bool timed_out) {
    fence_before_sync();
    const bool any_timeout = __syncthreads_or(timed_out) != 0;
    fence_after_sync();
    if (any_timeout) {
        if (threadIdx.x == 0) drain_mma(drain_bar);
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    }
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 64);
}

template <bool BF16, bool kSel = false>
__global__ void __launch_bounds__(128, 4) k_field_fwd_tc(DevCfg c, const float* __restrict__ params,
                                                      const float* __restrict__ rays, uint32_t cap,
                                                      const uint32_t* __restrict__ n_total,
                                                      const uint32_t* __restrict__ ray_id,
                                                      const float* __restrict__ ts, float4* __restrict__ sig_rgb,
                                                      uint4* __restrict__ feat_out, float feat_scale,
                                                      uint32_t* __restrict__ err,
                                                      const uint32_t* __restrict__ sel = nullptr) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar, drain_bar;
    __shared__ uint32_t tslot;
    load_weight_tiles<BF16>(params + (size_t)c.L * c.T * 2, smem, smem + kW1B, smem + kW1B + kW2B,
                            smem + kW1B + kW2B + kW3B, smem + kW1B + kW2B + kW3B + kW4B);
    const uint32_t tmem = fwd_block_setup(&tslot, &bar, &drain_bar);
    const uint32_t n = *n_total;
    const uint32_t n_tiles = (n + 127) / 128;
    const float2* tables = reinterpret_cast<const float2*>(params);
    uint32_t phase = 0;
    bool timed_out = false;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t i0 = tile * 128;
        fwd_tile<BF16, kSel>(c, tables, rays, cap, ray_id, ts, sig_rgb, feat_out, feat_scale, i0, n, smem, tmem, &bar,
                             phase, timed_out, sel);
        fence_before_sync();
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
            break;
        }
    }
    fwd_block_finish(tmem, &drain_bar, timed_out);
}

// Grouped forward (render of several views of several scenes): the batch's tiles
// are those of its pieces in order (a tile never mixes two pieces); a persistent
// block takes tiles i, i + grid, ...; where a tile belongs to another piece than the
// block's previous one, the block copies that piece's configuration into shared
// memory and, if the scene differs, rounds that scene's weights into the operand
// tiles.  Each tile is then exactly the single-view forward's tile.
// kSel: the pieces' runs s0 .. s0 + n_s - 1 index the selection sel (a render pass).
template <bool BF16, bool kSel = false>
__global__ void __launch_bounds__(128, 4) k_group_fwd_tc(const GroupItem* __restrict__ items, uint32_t n_items,
                                                      const uint32_t* __restrict__ n_tiles_total,
                                                      const float* __restrict__ rays, uint32_t cap,
                                                      const uint32_t* __restrict__ ray_id,
                                                      const float* __restrict__ ts, float4* __restrict__ sig_rgb,
                                                      float feat_scale, uint32_t* __restrict__ err,
                                                      const uint32_t* __restrict__ sel = nullptr) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar, drain_bar;
    __shared__ uint32_t tslot;
    __shared__ DevCfg cfg_s;
    __shared__ uint32_t tile0_s[kGroupMaxItems + 1];
    const uint32_t tmem = fwd_block_setup(&tslot, &bar, &drain_bar);
    const uint32_t total = *n_tiles_total;
    if (threadIdx.x < n_items) tile0_s[threadIdx.x] = items[threadIdx.x].tile0;
    if (threadIdx.x == 0) tile0_s[n_items] = total;
    __syncthreads();
    const float* cur_params = nullptr;
    uint32_t cur = n_items;  // no piece yet
    uint32_t phase = 0;
    bool timed_out = false;
    for (uint32_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        uint32_t j = 0;
        while (j + 1 < n_items && tile0_s[j + 1] <= tile) ++j;
        const GroupItem& it = items[j];
        if (j != cur) {
            __syncthreads();  // every thread is done with the previous tile's configuration
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&it.c);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&cfg_s);
            for (uint32_t w = threadIdx.x; w < sizeof(DevCfg) / 4; w += blockDim.x) dst[w] = src[w];
            if (it.params != cur_params)
                load_weight_tiles<BF16>(it.params + (size_t)it.c.L * it.c.T * 2, smem, smem + kW1B,
                                        smem + kW1B + kW2B, smem + kW1B + kW2B + kW3B,
                                        smem + kW1B + kW2B + kW3B + kW4B);
            cur_params = it.params;
            cur = j;
            to_tensor();      // the weights to the tensor core, the configuration to every thread
        }
        const uint32_t k = (tile - tile0_s[j]) * 128;
        fwd_tile<BF16, kSel>(cfg_s, reinterpret_cast<const float2*>(it.params), rays, cap, ray_id, ts, sig_rgb,
                             nullptr, feat_scale, it.s0 + k, it.s0 + it.n_s, smem, tmem, &bar, phase, timed_out, sel);
        fence_before_sync();
        if (__syncthreads_or(timed_out)) {
            if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
            break;
        }
    }
    fwd_block_finish(tmem, &drain_bar, timed_out);
}

// ------------------------------------------------------------------ backward
// Warp-specialised in three warpgroups: warps 0-3 (the "MLP" group, thread r =
// sample row r = TMEM lane r) run the layer chain on the tensor cores; warps 4-7
// (the "IO" group, thread 128 + r serves row r) load each tile's inputs one tile
// ahead and scatter the even levels of each finished tile's encoding gradient into
// the tables; warps 8-11 (the "SC" group, thread 256 + r) scatter its odd levels.
// Both scatter groups work on tile k while the MLP group runs tile k + 1: the
// scatter is the longer path (its reductions and warp shuffles load the L1 data
// pipe), so it gets two warpgroups.  Registers are split with setmaxnreg: the
// block is launched with 80 per thread (two blocks of 384 threads per SM), the
// MLP group takes 136, the IO group 64 (its prefetched inputs are dead while it
// scatters), the SC group 40 (the scatter alone needs no more without spilling):
// 128 x 136 + 128 x 64 + 128 x 40 = 384 x 80.  The groups hand tiles over through
// named barriers:
//   kBarIn      IO -> MLP        the tile's encodings (X0) and row data are in place
//   kBarDfReady MLP -> IO, SC    the chain is done (X0 free) and dL/dfeat is in smem
//   kBarDfFree  IO, SC -> MLP    both scatters of the tile are done (dL/dfeat read)
// All groups walk the same tile list and meet every barrier, whatever happens to
// an MMA wait (a timed-out wait only skips waiting), so no barrier can block.
//
// TMEM columns: [0,64) layer chain, [64,128) dW4, [128,160) dW3, [160,192) dW1,
// [192,208) dW2^T, [208,224) dW5^T.  The weight gradients are M=64 products: row m
// of such an accumulator is TMEM lane 32*(m/16) + m%16.
constexpr uint32_t kColW4 = 64, kColW3 = 128, kColW1 = 160, kColW2T = 192, kColW5T = 208;
constexpr int kBarMlp = 1, kBarIn = 2, kBarDfReady = 3, kBarDfFree = 4;
constexpr int kBwdThreads = 384;            // MLP, IO and SC warpgroups
constexpr uint32_t kRegMlp = 136, kRegIo = 64, kRegSc = 40;
static_assert(128 * (kRegMlp + kRegIo + kRegSc) == kBwdThreads * 80,
              "the setmaxnreg split must add up to the launch allocation (80 registers per thread)");
constexpr uint32_t kLevelsIo = 0x5555u, kLevelsSc = 0xAAAAu;  // even / odd levels
constexpr int kDfBytes = 128 * 32 * 4;      // dL/dfeat, [level][row] float2
constexpr int kRowBytes = 128 * 32;         // row data: {d.xyz, valid}, {dz0, dz1, dz2, dL/dsigma}
constexpr int kXBytes = 2 * 128 * 16;       // sample positions (x, valid) of the tiles, by parity
constexpr int kBwdSmem = kWB + kT32 + kT64 + kT32 + kT64 + kT64 + kT16 + kDfBytes + kRowBytes + kXBytes;  // 114688

namespace {

__device__ __forceinline__ void nb_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

// to_tensor() for the 128 threads of the MLP group only.
__device__ __forceinline__ void to_tensor_mlp() {
    fence_proxy_async();
    fence_before_sync();
    nb_sync(kBarMlp, 128);
    fence_after_sync();
}

// 64 accumulator columns -> relu(scale * a) into a 64-column tile; the ReLU branch
// of each column is returned as two 32-bit masks.
template <bool BF16>
__device__ __forceinline__ void relu_epilogue(uint32_t trow, uint8_t* tile, int r, float scale, uint32_t& ma,
                                              uint32_t& mb) {
    float v[32];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ld_cols<32>(trow, 32 * h, v);
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            v[k] *= scale;
            if (v[k] > 0.f) m |= 1u << k;
        }
        store_row_at<BF16, 32, true>(tile, r, 32 * h, v);
        if (h == 0) ma = m;
        else mb = m;
    }
}

// 64 accumulator columns masked by the ReLU branches into a 64-column tile.
template <bool BF16>
__device__ __forceinline__ void mask_epilogue(uint32_t trow, uint8_t* tile, int r, uint32_t ma, uint32_t mb) {
    float v[32];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ld_cols<32>(trow, 32 * h, v);
        const uint32_t m = h == 0 ? ma : mb;
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = ((m >> k) & 1u) ? v[k] : 0.f;
        store_row_at<BF16, 32>(tile, r, 32 * h, v);
    }
}

}  // namespace

// kPose: also writes, per sample, dL/dp (world position; IO group) and the
// view-direction gradient through the SH encoding (MLP group) into pose_s[2 i],
// pose_s[2 i + 1].
template <bool BF16, bool kPose>
__global__ void __launch_bounds__(kBwdThreads, 2) k_field_bwd_tc(DevCfg c, const float* __restrict__ params,
                                                         float* __restrict__ grads, const float* __restrict__ rays,
                                                         uint32_t cap, const uint32_t* __restrict__ n_total,
                                                         const uint32_t* __restrict__ ray_id,
                                                         const float* __restrict__ ts, const uint4* __restrict__ feat,
                                                         const float4* __restrict__ sig_rgb,
                                                         const float4* __restrict__ dsig_rgb, float feat_scale,
                                                         const float* __restrict__ seed_max,
                                                         float4* __restrict__ pose_s, uint32_t* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar, drain_bar;
    __shared__ uint32_t tslot;
    uint8_t* sW1 = smem;
    uint8_t* sW2 = sW1 + kW1B;
    uint8_t* sW3 = sW2 + kW2B;
    uint8_t* sW4 = sW3 + kW3B;
    uint8_t* sW5 = sW4 + kW4B;
    uint8_t* tX0 = smem + kWB;   // 128 x 32, written by the IO group
    uint8_t* tH1 = tX0 + kT32;   // 128 x 64  (later G1)
    uint8_t* tX3 = tH1 + kT64;   // 128 x 32  (later G2 in columns 0..15)
    uint8_t* tH3 = tX3 + kT32;   // 128 x 64  (later G3)
    uint8_t* tH4 = tH3 + kT64;   // 128 x 64  (later G4)
    uint8_t* tG5 = tH4 + kT64;   // 128 x 16
    uint8_t* sDf = tG5 + kT16;   // dL/dfeat: [16 levels][128 rows] float2
    float4* sRow = reinterpret_cast<float4*>(sDf + kDfBytes);  // [128][2]
    float4* sX = sRow + 2 * 128;                                // [2][128]: (x, valid) of tile k at k & 1
    const float2* sDf2 = reinterpret_cast<const float2*>(sDf);

    const int tid = threadIdx.x, warp = tid >> 5, r = tid & 127;
    load_weight_tiles<BF16>(params + (size_t)c.L * c.T * 2, sW1, sW2, sW3, sW4, sW5);
    if (warp == 0) tmem_alloc(&tslot, 256);
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init(&drain_bar, 1);
        mbar_fence_init();
    }
    to_tensor();
    const uint32_t tmem = tslot;
    const uint32_t n = *n_total;
    const uint32_t n_tiles = (n + 127) / 128;
    const uint32_t n_mine = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const float gm_d = seed_max[1], gm_c = seed_max[2];
    const float gm_dc = fmaxf(gm_d, gm_c);
    const float S = gm_dc > 0.f ? exp2f(fminf(fmaxf(floorf(log2f(kGradTarget / gm_dc)), -100.f), 100.f)) : 1.f;
    const float Sc = gm_c > 0.f ? exp2f(fminf(fmaxf(floorf(log2f(kGradTarget / gm_c)), -100.f), 100.f)) : S;
    const float inv_S = 1.f / S, inv_Sc = 1.f / Sc;
    const float c_to_d = S * inv_Sc;  // power of two: exact
    bool timed_out = false;

    if (warp < 4) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kRegMlp));
        // ======================= MLP group: the layer chain on the tensor cores
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const float inv_fs = 1.f / feat_scale;
        uint32_t phase = 0;
        constexpr uint32_t kM128N64 = idesc_f16(128, 64, BF16, false, false);
        constexpr uint32_t kM128N16 = idesc_f16(128, 16, BF16, false, false);
        for (uint32_t k = 0; k < n_mine; ++k) {
            nb_sync(kBarIn, 256);
            const float4 rd = sRow[2 * r], rz = sRow[2 * r + 1];
            const bool valid = rd.w != 0.f;
            float v[32];
            uint32_t m1a, m1b, m3a, m3b, m4a, m4b;
            // ---- forward recompute (same arithmetic as the forward kernel)
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem, kmaj(tX0, 128), kmaj(sW1, 64), 2, kM128N64, false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            relu_epilogue<BF16>(trow, tH1, r, inv_fs, m1a, m1b);
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem, kmaj(tH1, 128), kmaj(sW2, 16), 4, kM128N16, false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            float y[32];
            ld_cols<16>(trow, 0, y);
            const float sigma = expf(fminf(y[0], kSigmaHMax));
            const float sig_grad = y[0] < kSigmaHMax ? sigma : 0.f;
            if (valid) sh16(rd.x, rd.y, rd.z, y + kGeo);
            else {
#pragma unroll
                for (int q = kGeo; q < 32; ++q) y[q] = 0.f;
            }
            store_row_at<BF16, 32>(tX3, r, 0, y);
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem, kmaj(tX3, 128), kmaj(sW3, 64), 2, kM128N64, false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            relu_epilogue<BF16>(trow, tH3, r, 1.f, m3a, m3b);
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem, kmaj(tH3, 128), kmaj(sW4, 64), 4, kM128N64, false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            relu_epilogue<BF16>(trow, tH4, r, 1.f, m4a, m4b);
            // the colours' gradient seed dz (FP32, scaled by S) comes from the IO group
            v[0] = rz.x;
            v[1] = rz.y;
            v[2] = rz.z;
#pragma unroll
            for (int q = 3; q < 16; ++q) v[q] = 0.f;
            store_row_at<BF16, 16>(tG5, r, 0, v);
            // ---- backward: dW5^T += H4^T G5 ; dH4 = G5 W5
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem + kColW5T, mnmaj(tH4, 128), mnmaj(tG5, 128), 8, idesc_f16(64, 16, BF16, true, true), k > 0);
                gemm(tmem, kmaj(tG5, 128), mnmaj(sW5, 16), 1, idesc_f16(128, 64, BF16, false, true), false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            mask_epilogue<BF16>(trow, tH4, r, m4a, m4b);                 // G4
            // dW4 += G4^T H3 ; dH3 = G4 W4
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem + kColW4, mnmaj(tH4, 128), mnmaj(tH3, 128), 8, idesc_f16(64, 64, BF16, true, true), k > 0);
                gemm(tmem, kmaj(tH4, 128), mnmaj(sW4, 64), 4, idesc_f16(128, 64, BF16, false, true), false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            mask_epilogue<BF16>(trow, tH3, r, m3a, m3b);                 // G3
            // dW3 += G3^T X3 ; dX3 = G3 W3
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem + kColW3, mnmaj(tH3, 128), mnmaj(tX3, 128), 8, idesc_f16(64, 32, BF16, true, true), k > 0);
                gemm(tmem, kmaj(tH3, 128), mnmaj(sW3, 64), 4, idesc_f16(128, 32, BF16, false, true), false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            if (kPose) {
                // the SH inputs' gradient (columns 16..31, colour scale) -> view direction
                ld_cols<16>(trow, 16, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] *= inv_Sc;
                const float3 gd = sh16_vjp(rd.x, rd.y, rd.z, v);
                const uint32_t i = (blockIdx.x + k * gridDim.x) * 128 + r;
                if (valid) pose_s[2 * (size_t)i + 1] = make_float4(gd.x, gd.y, gd.z, 0.f);
            }
            ld_cols<16>(trow, 0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] *= c_to_d;                // colour scale -> density scale
            v[0] += S * rz.w * sig_grad;                                 // dL/dh_0 += dL/dsigma * dsigma/dh_0
            store_row_at<BF16, 16>(tX3, r, 0, v);                        // G2 (columns 0..15)
            // dW2^T += H1^T G2 ; dH1 = G2 W2
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem + kColW2T, mnmaj(tH1, 128), mnmaj(tX3, 128), 8, idesc_f16(64, 16, BF16, true, true),
                     k > 0);
                gemm(tmem, kmaj(tX3, 128), mnmaj(sW2, 16), 1, idesc_f16(128, 64, BF16, false, true), false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            mask_epilogue<BF16>(trow, tH1, r, m1a, m1b);                 // G1
            // dW1 += G1^T X0 ; dF = G1 W1
            to_tensor_mlp();
            if (r == 0) {
                gemm(tmem + kColW1, mnmaj(tH1, 128), mnmaj(tX0, 128), 8, idesc_f16(64, 32, BF16, true, true), k > 0);
                gemm(tmem, kmaj(tH1, 128), mnmaj(sW1, 64), 4, idesc_f16(128, 32, BF16, false, true), false);
                mma_commit(&bar);
            }
            wait_mma(&bar, phase, timed_out, c.wait_polls);
            ld_cols<32>(trow, 0, v);
            fence_before_sync();
            if (k > 0) nb_sync(kBarDfFree, kBwdThreads);  // both scatters of the previous tile are done
#pragma unroll
            for (int q = 0; q < 16; ++q)
                reinterpret_cast<float2*>(sDf)[q * 128 + r] = make_float2(v[2 * q] * inv_S, v[2 * q + 1] * inv_S);
            nb_arrive(kBarDfReady, kBwdThreads);          // also: X0 and the row data are free
        }
        // ---- flush the weight gradients (lane 32*(m/16) + m%16 holds row m)
        const bool any_timeout = __syncthreads_or(timed_out) != 0;  // all three groups take part
        fence_after_sync();
        if (any_timeout && r == 0) drain_mma(&drain_bar);          // r == 0 issued every MMA
        if (n_mine > 0 && !any_timeout) {
            float* gm_ = grads + (size_t)c.L * c.T * 2;
            const int lane = tid & 31;
            const int m = warp * 16 + lane;
            const bool has = lane < 16;
            float w[32];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                ld_cols<32>(trow, kColW4 + 32 * h, w);
                if (has)
                    for (int q = 0; q < 32; ++q) atomicAdd(gm_ + kOffW4 + m * 64 + 32 * h + q, w[q] * inv_Sc);
            }
            ld_cols<32>(trow, kColW3, w);
            if (has)
                for (int q = 0; q < 32; ++q) atomicAdd(gm_ + kOffW3 + m * 32 + q, w[q] * inv_Sc);
            ld_cols<32>(trow, kColW1, w);
            if (has)
                for (int q = 0; q < 32; ++q) atomicAdd(gm_ + kOffW1 + m * 32 + q, w[q] * inv_S * inv_fs);
            ld_cols<16>(trow, kColW2T, w);
            if (has)
                for (int q = 0; q < 16; ++q) atomicAdd(gm_ + kOffW2 + q * 64 + m, w[q] * inv_S);
            ld_cols<16>(trow, kColW5T, w);
            if (has)
                for (int q = 0; q < 3; ++q) atomicAdd(gm_ + kOffW5 + q * 64 + m, w[q] * inv_Sc);
        }
        if (any_timeout && tid == 0) atomicOr(err, kErrTimeout);
    } else if (warp >= 8) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kRegSc));
        // ======================= SC group: the odd levels' gradient scatter
        float2* gtables = reinterpret_cast<float2*>(grads);
        for (uint32_t k = 0; k < n_mine; ++k) {
            nb_sync(kBarDfReady, kBwdThreads);
            const float4 xq = sX[(k & 1u) * 128 + r];
            hash_scatter_warp<true>(c, gtables, make_float3(xq.x, xq.y, xq.z),
                                    [&](int l) { return sDf2[l * 128 + r]; }, xq.w != 0.f, kLevelsSc);
            if (k + 1 < n_mine) nb_arrive(kBarDfFree, kBwdThreads);
        }
        __syncthreads_or(false);                      // pairs with the MLP group's flush barrier
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kRegIo));
        // ======================= IO group: tile inputs one tile ahead, the even levels' scatter
        float2* gtables = reinterpret_cast<float2*>(grads);
        float3 x_cur = make_float3(0.f, 0.f, 0.f), x_next = x_cur;
        bool valid_cur = false, valid_next = false;
        uint32_t i_cur = 0, i_next = 0;
        uint4 f_next[4];
        float4 rd_next, rz_next;
        // inputs of this block's k-th tile for row r, into registers
        auto load = [&](uint32_t k) {
            const uint32_t i = (blockIdx.x + k * gridDim.x) * 128 + r;
            i_next = i;
            valid_next = i < n;
            float3 d = make_float3(0.f, 0.f, 0.f);
            x_next = make_float3(0.f, 0.f, 0.f);
            rd_next = make_float4(0.f, 0.f, 0.f, 0.f);
            rz_next = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) f_next[q] = make_uint4(0u, 0u, 0u, 0u);
            if (valid_next) {
                x_next = sample_pos_tc(c, rays, cap, ray_id[i], ts[i], d);
                const float4 g = dsig_rgb[i], col = sig_rgb[i];
#pragma unroll
                for (int q = 0; q < 4; ++q) f_next[q] = feat[(size_t)i * 4 + q];
                rd_next = make_float4(d.x, d.y, d.z, 1.f);
                rz_next = make_float4(Sc * g.y * col.y * (1.f - col.y), Sc * g.z * col.z * (1.f - col.z),
                                      Sc * g.w * col.w * (1.f - col.w), g.x);
            }
        };
        // the inputs of tile kk into the operand tile and the row data (and its sample
        // positions for the SC group)
        auto publish = [&](uint32_t kk) {
            sX[(kk & 1u) * 128 + r] = make_float4(x_next.x, x_next.y, x_next.z, valid_next ? 1.f : 0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(tX0 + tile_offset(r, 8 * q, 128)) = f_next[q];
            sRow[2 * r] = rd_next;
            sRow[2 * r + 1] = rz_next;
            x_cur = x_next;
            valid_cur = valid_next;
            i_cur = i_next;
            fence_proxy_async();                      // X0 is read by the tensor core
            nb_arrive(kBarIn, 256);
        };
        if (n_mine > 0) {
            load(0);
            publish(0);
        }
        for (uint32_t k = 0; k < n_mine; ++k) {
            if (k + 1 < n_mine) load(k + 1);          // global loads in flight during the chain
            nb_sync(kBarDfReady, kBwdThreads);
            const float3 x_done = x_cur;
            const bool valid_done = valid_cur;
            const uint32_t i_done = i_cur;
            if (k + 1 < n_mine) publish(k + 1);       // next tile's inputs; the MLP group starts on it
            hash_scatter_warp<true>(c, gtables, x_done, [&](int l) { return sDf2[l * 128 + r]; }, valid_done,
                                    kLevelsIo);
            if (kPose && valid_done) {
                float v[32];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float2 a = sDf2[q * 128 + r];
                    v[2 * q] = a.x;
                    v[2 * q + 1] = a.y;
                }
                const float3 gx = hash_grad_x(c, reinterpret_cast<const float2*>(params), x_done, v);
                pose_s[2 * (size_t)i_done] =
                    make_float4(gx.x * c.inv_size, gx.y * c.inv_size, gx.z * c.inv_size, 0.f);
            }
            if (k + 1 < n_mine) nb_arrive(kBarDfFree, kBwdThreads);  // dL/dfeat read: the MLP group may overwrite it
        }
        __syncthreads_or(false);                      // pairs with the MLP group's flush barrier
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// ------------------------------------------------------------------ launchers

template <bool BF16>
static void fwd_tc(const DevCfg& c, const float* params, uint32_t n_rays, const StepBufs& b, bool store_feat,
                   int n_sm, cudaStream_t s) {
    // per call: the attribute belongs to the current device (cheap next to the kernel)
    cudaFuncSetAttribute(k_field_fwd_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    const float fs = BF16 ? 1.f : 256.f;
    k_field_fwd_tc<BF16><<<n_sm * 4, 128, kFwdSmem, s>>>(c, params, b.rays, b.cap_rays, b.offsets + n_rays,
                                                          b.ray_id, b.t, b.sig_rgb,
                                                          store_feat ? reinterpret_cast<uint4*>(b.feat) : nullptr,
                                                          fs, b.err);
}

template <bool BF16, bool kPose>
static void bwd_tc(const DevCfg& c, const float* params, float* grads, uint32_t n_rays, const StepBufs& b, int n_sm,
                   cudaStream_t s) {
    // per call: the attribute belongs to the current device (cheap next to the kernel)
    cudaFuncSetAttribute(k_field_bwd_tc<BF16, kPose>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
    const float fs = BF16 ? 1.f : 256.f;
    k_field_bwd_tc<BF16, kPose><<<n_sm * 2, kBwdThreads, kBwdSmem, s>>>(
        c, params, grads, b.rays, b.cap_rays, b.offsets + n_rays, b.ray_id, b.t, reinterpret_cast<const uint4*>(b.feat),
        b.sig_rgb, b.dsig_rgb, fs, b.loss, kPose ? b.pose_s : nullptr, b.err);
}

template <bool BF16>
static void fwd_tc_sel(const DevCfg& c, const float* params, const uint32_t* sel, const uint32_t* n_sel,
                       const StepBufs& b, int n_sm, cudaStream_t s) {
    cudaFuncSetAttribute(k_field_fwd_tc<BF16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    const float fs = BF16 ? 1.f : 256.f;
    k_field_fwd_tc<BF16, true><<<n_sm * 4, 128, kFwdSmem, s>>>(c, params, b.rays, b.cap_rays, n_sel, b.ray_id, b.t,
                                                                b.sig_rgb, nullptr, fs, b.err, sel);
}

void launch_field_fwd_tc_sel(const DevCfg& c, const float* params, const uint32_t* sel, const uint32_t* n_sel,
                             const StepBufs& b, bool bf16, int n_sm, cudaStream_t s) {
    if (bf16) fwd_tc_sel<true>(c, params, sel, n_sel, b, n_sm, s);
    else fwd_tc_sel<false>(c, params, sel, n_sel, b, n_sm, s);
}

void launch_field_fwd_tc(const DevCfg& c, const float* params, uint32_t n_rays, const StepBufs& b, bool store_feat,
                         bool bf16, int n_sm, cudaStream_t s) {
    if (bf16) fwd_tc<true>(c, params, n_rays, b, store_feat, n_sm, s);
    else fwd_tc<false>(c, params, n_rays, b, store_feat, n_sm, s);
}

template <bool BF16, bool kSel>
static void group_fwd(const GroupItem* items, uint32_t n_items, const uint32_t* n_tiles, const StepBufs& b,
                      const uint32_t* sel, int n_sm, cudaStream_t s) {
    cudaFuncSetAttribute(k_group_fwd_tc<BF16, kSel>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    k_group_fwd_tc<BF16, kSel><<<n_sm * 4, 128, kFwdSmem, s>>>(items, n_items, n_tiles, b.rays, b.cap_rays, b.ray_id,
                                                                b.t, b.sig_rgb, BF16 ? 1.f : 256.f, b.err, sel);
}

void launch_group_fwd_tc(const GroupItem* items, uint32_t n_items, const uint32_t* n_tiles, const StepBufs& b,
                         bool bf16, int n_sm, cudaStream_t s, const uint32_t* sel) {
    if (sel) {
        if (bf16) group_fwd<true, true>(items, n_items, n_tiles, b, sel, n_sm, s);
        else group_fwd<false, true>(items, n_items, n_tiles, b, sel, n_sm, s);
    } else {
        if (bf16) group_fwd<true, false>(items, n_items, n_tiles, b, sel, n_sm, s);
        else group_fwd<false, false>(items, n_items, n_tiles, b, sel, n_sm, s);
    }
}

void launch_field_bwd_tc(const DevCfg& c, const float* params, float* grads, uint32_t n_rays, const StepBufs& b,
                         bool bf16, int n_sm, cudaStream_t s, bool pose) {
    if (pose) {
        if (bf16) bwd_tc<true, true>(c, params, grads, n_rays, b, n_sm, s);
        else bwd_tc<false, true>(c, params, grads, n_rays, b, n_sm, s);
    } else {
        if (bf16) bwd_tc<true, false>(c, params, grads, n_rays, b, n_sm, s);
        else bwd_tc<false, false>(c, params, grads, n_rays, b, n_sm, s);
    }
}

}  // namespace nm
