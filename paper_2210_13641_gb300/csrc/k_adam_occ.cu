// k_adam_occ.cu - Adam over all parameters (step a12), parameter initialisation,
// and the occupancy-grid refresh (step a13).
#include <cmath>

#include "encoding.cuh"
#include "internal.h"

namespace nm {

// Adam with bias correction (c1 = 1/(1-b1^t), c2 = 1/(1-b2^t) precomputed), dense
// over every parameter; the gradient is cleared after it is read.  float4 lanes.
__global__ void k_adam(float4* __restrict__ p, float4* __restrict__ g, float4* __restrict__ m,
                       float4* __restrict__ v, size_t n4, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const float ob1 = 1.f - b1, ob2 = 1.f - b2;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
         i += (size_t)gridDim.x * blockDim.x) {
        float4 gg = g[i], mm = m[i], vv = v[i], pp = p[i];
#define NM_ADAM_LANE(q)                                                  \
    mm.q = b1 * mm.q + ob1 * gg.q;                                       \
    vv.q = b2 * vv.q + ob2 * gg.q * gg.q;                                \
    pp.q -= lr * (mm.q * c1) / (sqrtf(vv.q * c2) + eps);
        NM_ADAM_LANE(x) NM_ADAM_LANE(y) NM_ADAM_LANE(z) NM_ADAM_LANE(w)
#undef NM_ADAM_LANE
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
        g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

void launch_adam(float* p, float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                 float eps, float c1, float c2, cudaStream_t s) {
    const size_t n4 = n / 4;
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    size_t blocks = (n4 + 255) / 256;
    const size_t cap = (size_t)n_sm * 8;
    if (blocks > cap) blocks = cap;
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(g),
                                            reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v),
                                            n4, lr, b1, b2, eps, c1, c2);
}

// Initial parameters: tables ~ U(-1e-4, 1e-4), MLP weights ~ N(0, 0.05) (Box-Muller
// on two 24-bit uniforms).  Counter stream 3 << 30 keyed by the parameter index.
__global__ void k_init_params(float* __restrict__ p, size_t n_table, size_t n, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t r = counter_rand(seed, 3ull << 30, i, 0);
        const float u1 = ((float)(r >> 40) + 0.5f) * (1.f / 16777216.f);
        const float u2 = ((float)((r >> 16) & 0xFFFFFF) + 0.5f) * (1.f / 16777216.f);
        if (i < n_table) {
            p[i] = (2.f * u1 - 1.f) * 1e-4f;
        } else {
            p[i] = 0.05f * sqrtf(-2.f * logf(u1)) * cosf(6.283185307179586f * u2);
        }
    }
}

void launch_init_params(float* p, size_t n_table, uint64_t seed, cudaStream_t s) {
    const size_t n = n_table + kMlpParams;
    k_init_params<<<1024, 256, 0, s>>>(p, n_table, n, seed);
}

// Occupancy refresh: one seeded point x = (c + u) / R per cell (u: three 21-bit
// fields of one counter draw, stream kOccStream + refresh index), its density
// sigma = exp(min((W2 relu(W1 enc(x)))_0, 15)) on FP32 cores, EMA d <- max(decay d, sigma),
// bit = d > thresh (32 cells per ballot word).
__global__ void __launch_bounds__(256) k_occ_refresh(DevCfg c, const float* __restrict__ params,
                                                     float* __restrict__ density,
                                                     uint32_t* __restrict__ bits, uint64_t seed,
                                                     uint64_t refresh_idx, float decay, float thresh) {
    __shared__ float W1[kW1];
    __shared__ float W2r0[kHid];  // only the first output row of W2 feeds sigma
    const float* mlp = params + (size_t)c.L * c.T * 2;
    for (int i = threadIdx.x; i < kW1; i += blockDim.x) W1[i] = mlp[kOffW1 + i];
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) W2r0[i] = mlp[kOffW2 + i];
    __syncthreads();
    const uint32_t R = c.occ_res;
    const uint32_t n = R * R * R;
    const float2* tables = reinterpret_cast<const float2*>(params);
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t cell = base + threadIdx.x;  // n is a multiple of 512: no tail
        const uint64_t r = counter_rand(seed, kOccStream + refresh_idx, cell, 0);
        const float ux = (float)(r & 0x1FFFFFu) * (1.f / 2097152.f);
        const float uy = (float)((r >> 21) & 0x1FFFFFu) * (1.f / 2097152.f);
        const float uz = (float)((r >> 42) & 0x1FFFFFu) * (1.f / 2097152.f);
        const uint32_t cx = cell % R, cy = (cell / R) % R, cz = cell / (R * R);
        float3 x;
        x.x = fdiv(fadd((float)cx, ux), (float)R);
        x.y = fdiv(fadd((float)cy, uy), (float)R);
        x.z = fdiv(fadd((float)cz, uz), (float)R);
        float f[kEnc];
        hash_encode(c, tables, x, f);
        float h0 = 0.f;
#pragma unroll 4
        for (int j = 0; j < kHid; ++j) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < kEnc; ++k) a += W1[j * kEnc + k] * f[k];
            h0 += W2r0[j] * fmaxf(a, 0.f);
        }
        const float sigma = expf(fminf(h0, kSigmaHMax));
        const float d = fmaxf(decay * density[cell], sigma);
        density[cell] = d;
        const uint32_t word = __ballot_sync(0xffffffffu, d > thresh);
        if ((threadIdx.x & 31) == 0) bits[cell >> 5] = word;
    }
}

void launch_occ_refresh(const DevCfg& c, const float* params, float* density, uint32_t* bits,
                        uint64_t seed, uint64_t refresh_idx, float decay, float thresh,
                        cudaStream_t s) {
    const uint32_t n = c.occ_res * c.occ_res * c.occ_res;
    uint32_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_occ_refresh<<<blocks, 256, 0, s>>>(c, params, density, bits, seed, refresh_idx, decay, thresh);
}

__global__ void k_occ_from_bits(const uint32_t* __restrict__ bits, float* __restrict__ density,
                                uint32_t n_cells) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cells) density[i] = ((bits[i >> 5] >> (i & 31)) & 1u) ? 1.f : 0.f;
}

void launch_occ_from_bits(const uint32_t* bits, float* density, uint32_t n_cells, cudaStream_t s) {
    k_occ_from_bits<<<(n_cells + 255) / 256, 256, 0, s>>>(bits, density, n_cells);
}

}  // namespace nm
