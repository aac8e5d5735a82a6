// encoding.cuh - multiresolution hash-grid encoding and its gradient scatter
// (step a3 / a11).  The grid is the Instant-NGP encoding the paper uses as its map
// (Sec. 3.4): per level l, the sample's cell at resolution N_l, the 8 corner slots
// (dense index or spatial hash), and trilinear interpolation of 2 FP32 features.
#pragma once

#include "common.cuh"

namespace nm {

// Trilinear corner weight of corner k = bx + 2 by + 4 bz.
__device__ __forceinline__ float corner_weight(int k, float wx, float wy, float wz) {
    return ((k & 1) ? wx : 1.f - wx) * ((k & 2) ? wy : 1.f - wy) * ((k & 4) ? wz : 1.f - wz);
}

// Corners k and k + 1 (k even) differ only in x.  Their slots s and s' share one
// aligned 16-byte chunk (two float2 entries) exactly when s' = s ^ 1: in a hashed
// level that holds whenever cx is even (the x coordinate enters the hash by xor with
// prime 1), in a dense level whenever s is even.  The encoding reads such a pair
// with one 16-byte load.  (The gradient scatter keeps one 8-byte reduction per
// corner: 16-byte reductions of the shared pairs made the backward slower.)
__device__ __forceinline__ bool x_pair_shared(uint32_t s0, uint32_t s1) { return (s0 ^ s1) == 1u; }

// Features of levels l0 .. l0 + kGatherGroup - 1 of grid position x into
// f[0 .. 2 kGatherGroup) (zero for levels >= L).  tables: [L][T] float2.  Level by
// level, the level's 4 x-pair loads are issued before any is used.  An x-pair of
// corners in one chunk is read with one 16-byte load (halves swapped when corner k is
// the upper one), any other pair with two 8-byte loads.  (Issuing the loads of 4 or 2
// levels before using any kept more loads in flight but spilled registers in the
// tensor-core forward: 3.18 and 3.08 ms against 3.03 ms for one level at a time.)
constexpr int kGatherGroup = 4;

__device__ __forceinline__ void encode_level(const DevCfg& c, const float2* __restrict__ tables, float3 x, int l,
                                             float* f) {
    const uint32_t Tmask = c.T - 1;
    float4 q[4];   // (corner 2j, corner 2j + 1), halves swapped if bit j of swp
    uint32_t swp = 0u;
    float w[3];
    const uint32_t N = c.res[l];
    const bool dense = (c.dense_mask >> l) & 1u;
    uint32_t cx, cy, cz;
    level_cell(x.x, N, cx, w[0]);
    level_cell(x.y, N, cy, w[1]);
    level_cell(x.z, N, cz, w[2]);
    const float2* tab = tables + (size_t)l * c.T;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t yy = cy + (j & 1), zz = cz + (j >> 1);
        const uint32_t s0 = vertex_slot(cx, yy, zz, N, dense, Tmask);
        const uint32_t s1 = vertex_slot(cx + 1, yy, zz, N, dense, Tmask);
        if (x_pair_shared(s0, s1)) {
            q[j] = __ldg(reinterpret_cast<const float4*>(tab + (s0 & ~1u)));
            swp |= (s0 & 1u) << j;
        } else {
            const float2 a = __ldg(tab + s0), b = __ldg(tab + s1);
            q[j] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool hi = (swp >> j) & 1u;
        const float4 v = q[j];
        const float w0 = corner_weight(2 * j, w[0], w[1], w[2]);
        const float w1 = corner_weight(2 * j + 1, w[0], w[1], w[2]);
        a0 += w0 * (hi ? v.z : v.x);
        a1 += w0 * (hi ? v.w : v.y);
        a0 += w1 * (hi ? v.x : v.z);
        a1 += w1 * (hi ? v.y : v.w);
    }
    f[0] = a0;
    f[1] = a1;
}

__device__ __forceinline__ void encode_group(const DevCfg& c, const float2* __restrict__ tables, float3 x,
                                             int l0, float* f) {
#pragma unroll
    for (int g = 0; g < kGatherGroup; ++g) {
        if (l0 + g < (int)c.L) {
            encode_level(c, tables, x, l0 + g, f + 2 * g);
        } else {
            f[2 * g] = 0.f;
            f[2 * g + 1] = 0.f;
        }
    }
}

// Encodes grid position x into f[0 .. 2L) (f[2L .. 32) set to zero).
__device__ __forceinline__ void hash_encode(const DevCfg& c, const float2* __restrict__ tables,
                                            float3 x, float* f) {
#pragma unroll
    for (int l0 = 0; l0 < kEnc / 2; l0 += kGatherGroup) encode_group(c, tables, x, l0, f + 2 * l0);
}

// dL/dtable[l][slot_k] += w_k * dL/df_l for every corner and for the levels whose
// bit is set in `levels` (FP32 vector reductions of 8 bytes, one per corner),
// warp-cooperative: called by all 32 lanes (lanes with valid = false contribute
// nothing).  df(l) returns this lane's (dL/df_{l,0}, dL/df_{l,1}) as a float2.  Consecutive samples of a ray fall into the
// same cell of the coarse levels, so per level the lanes with equal cells (runs of
// consecutive lanes) first sum their 8 corner contributions with a segmented
// shuffle reduction, and only the first lane of each run issues the 8 atomics.
// A level whose 32 cells are all different skips the reduction.  A level whose 32
// samples share one cell (one run, all lanes valid: the common case of the coarse
// levels) sums, with kButterfly, by a butterfly that halves the corners held per
// lane at each step (18 shuffles instead of the segmented form's 80); lane 4k then
// holds corner k's sum and 8 lanes issue the 8 reductions together (the tensor-core
// backward: -2 % time; the FP32 backward keeps the segmented form, +7 % with it).
// The level loop is unrolled by two only (two levels' shuffles in flight): the fully
// unrolled form's code did not fit the instruction cache next to the tensor-core
// layer chain of the backward kernel.  Runs are not cut short to save reduction
// rounds: every extra head costs 8 reductions, which the large map's HBM-resident
// tables pay dearly (cutting runs every 8 lanes: -1 % on a 64 MB table, +20 % on a
// 512 MB one).
template <bool kButterfly, class DF>
__device__ __forceinline__ void hash_scatter_warp(const DevCfg& c, float2* __restrict__ gtables,
                                                  float3 x, DF df, bool valid, uint32_t levels = 0xFFFFu) {
    const uint32_t Tmask = c.T - 1;
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 2
    for (int l = 0; l < kEnc / 2; ++l) {
        if (l >= (int)c.L) break;
        if (!((levels >> l) & 1u)) continue;
        const uint32_t N = c.res[l];
        const bool dense = (c.dense_mask >> l) & 1u;
        uint32_t cx, cy, cz;
        float wx, wy, wz;
        level_cell(x.x, N, cx, wx);
        level_cell(x.y, N, cy, wy);
        level_cell(x.z, N, cz, wz);
        float2* gtab = gtables + (size_t)l * c.T;
        const float2 gl = df(l);
        const float g0 = valid ? gl.x : 0.f, g1 = valid ? gl.y : 0.f;
        const uint64_t key = valid ? (((uint64_t)cz << 42) | ((uint64_t)cy << 21) | cx) : ~(uint64_t)lane;
        const uint64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool head = lane == 0 || prev != key;
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        float v[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float wk = corner_weight(k, wx, wy, wz);
            v[2 * k] = wk * g0;
            v[2 * k + 1] = wk * g1;
        }
        if (kButterfly && heads == 1u) {
            // one run: after the exchanges across lane bits 4, 3 and 2 a lane holds
            // the partial sums of corner (lane >> 2), completed across bits 1 and 0
            const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
            float2 a[4], h[2];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 lo = make_float2(v[2 * j], v[2 * j + 1]);
                const float2 hi = make_float2(v[2 * j + 8], v[2 * j + 9]);
                const float2 snd = b4 ? lo : hi, kp = b4 ? hi : lo;
                a[j] = make_float2(kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 16),
                                   kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 16));
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float2 snd = b3 ? a[j] : a[j + 2], kp = b3 ? a[j + 2] : a[j];
                h[j] = make_float2(kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 8),
                                   kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 8));
            }
            const float2 snd = b2 ? h[0] : h[1], kp = b2 ? h[1] : h[0];
            float2 d = make_float2(kp.x + __shfl_xor_sync(0xffffffffu, snd.x, 4),
                                   kp.y + __shfl_xor_sync(0xffffffffu, snd.y, 4));
            d.x += __shfl_xor_sync(0xffffffffu, d.x, 2);
            d.y += __shfl_xor_sync(0xffffffffu, d.y, 2);
            d.x += __shfl_xor_sync(0xffffffffu, d.x, 1);
            d.y += __shfl_xor_sync(0xffffffffu, d.y, 1);
            if ((lane & 3u) == 0u) {
                const uint32_t k = lane >> 2;
                const uint32_t slot = vertex_slot(cx + (k & 1u), cy + ((k >> 1) & 1u), cz + (k >> 2), N, dense, Tmask);
                atomicAdd(gtab + slot, d);
            }
            continue;
        }
        if (heads != 0xffffffffu) {
            // lanes lane .. run_end form this lane's run; the head ends up with the sum
            const uint32_t above = (lane == 31u) ? 0u : (heads & ~((2u << lane) - 1u));
            const uint32_t run_end = above ? (uint32_t)(__ffs(above) - 2) : 31u;
            const uint32_t max_len = __reduce_max_sync(0xffffffffu, head ? run_end - lane + 1u : 1u);
            for (uint32_t off = 1; off < max_len; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float o = __shfl_down_sync(0xffffffffu, v[q], off);
                    if (lane + off <= run_end) v[q] += o;
                }
            }
        }
        if (head && valid) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t slot = vertex_slot(cx + (k & 1), cy + ((k >> 1) & 1), cz + ((k >> 2) & 1), N,
                                                  dense, Tmask);
                atomicAdd(gtab + slot, make_float2(v[2 * k], v[2 * k + 1]));
            }
        }
    }
}

// dL/dx = sum_l (d f_l / dx) . dL/df_l at grid position x, for the pose gradient:
// inside a cell of level l (resolution N) the trilinear weight of corner k is
// w_k = prod_a (b_a ? w_a : 1 - w_a) with w_a = x_a N - c_a, so
// dw_k/dx_a = N (b_a ? 1 : -1) prod_{a' != a} (b_a' ? w_a' : 1 - w_a'); the table
// values of the 8 corners are read again.  df: dL/df [kEnc].
__device__ __forceinline__ float3 hash_grad_x(const DevCfg& c, const float2* __restrict__ tables, float3 x,
                                              const float* df) {
    const uint32_t Tmask = c.T - 1;
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 1
    for (int l = 0; l < kEnc / 2; ++l) {
        if (l >= (int)c.L) break;
        const uint32_t N = c.res[l];
        const bool dense = (c.dense_mask >> l) & 1u;
        uint32_t cx, cy, cz;
        float wx, wy, wz;
        level_cell(x.x, N, cx, wx);
        level_cell(x.y, N, cy, wy);
        level_cell(x.z, N, cz, wz);
        const float2* tab = tables + (size_t)l * c.T;
        const float g0 = df[2 * l], g1 = df[2 * l + 1];
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int bx = k & 1, by = (k >> 1) & 1, bz = (k >> 2) & 1;
            const uint32_t slot = vertex_slot(cx + bx, cy + by, cz + bz, N, dense, Tmask);
            const float2 v = __ldg(tab + slot);
            const float e = v.x * g0 + v.y * g1;                    // corner value . dL/df_l
            const float fx = bx ? wx : 1.f - wx, fy = by ? wy : 1.f - wy, fz = bz ? wz : 1.f - wz;
            ax += (bx ? e : -e) * fy * fz;
            ay += (by ? e : -e) * fx * fz;
            az += (bz ? e : -e) * fx * fy;
        }
        gx += (float)N * ax;
        gy += (float)N * ay;
        gz += (float)N * az;
    }
    return make_float3(gx, gy, gz);
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

}  // namespace nm
