// k_field_fp32.cu - the field on FP32 CUDA cores (the plain form): hash encoding,
// density MLP (sigma = exp(h_0)), SH view encoding and colour MLP (sigmoid) forward
// (steps a3-a6), and the recomputing backward pass (steps a10-a11).
//
// Forward: one thread per sample, weights in shared memory.  Backward: tiles of
// 128 samples per 128-thread block; each thread recomputes its sample's activations
// into a shared-memory row, the block then forms the weight-gradient tile products
// (sum over the tile's samples), and every thread scatters its encoding gradient into
// the tables with FP32 atomics.  Weight gradients stay in shared memory across the
// tiles a persistent block visits and are flushed with one atomic per weight.
#include "encoding.cuh"
#include "internal.h"

namespace nm {

// Weights in shared memory, with the transposes the per-thread loops read along.
struct SmemW {
    float W1[kHid * kEnc];        // [j][k]
    float W2T[kHid * kGeo];       // [j][m] = W2[m][j]
    float W3[kHid * 32];          // [j][k]
    float W4T[kHid * kHid];       // [j][i] = W4[i][j]
    float W5[3 * kHid];           // [c][i]
};

__device__ void load_weights(SmemW& s, const float* __restrict__ mlp) {
    for (int i = threadIdx.x; i < kW1; i += blockDim.x) s.W1[i] = mlp[kOffW1 + i];
    for (int i = threadIdx.x; i < kW2; i += blockDim.x) {
        const int m = i / kHid, j = i % kHid;
        s.W2T[j * kGeo + m] = mlp[kOffW2 + i];
    }
    for (int i = threadIdx.x; i < kW3; i += blockDim.x) s.W3[i] = mlp[kOffW3 + i];
    for (int i = threadIdx.x; i < kW4; i += blockDim.x) {
        const int r = i / kHid, j = i % kHid;
        s.W4T[j * kHid + r] = mlp[kOffW4 + i];
    }
    for (int i = threadIdx.x; i < kW5; i += blockDim.x) s.W5[i] = mlp[kOffW5 + i];
}

__device__ __forceinline__ float3 sample_pos(const DevCfg& c, const float* __restrict__ rays,
                                             uint32_t cap, uint32_t r, float t, float3& d) {
    const float3 o = make_float3(rays[kOx * cap + r], rays[kOy * cap + r], rays[kOz * cap + r]);
    d = make_float3(rays[kDx * cap + r], rays[kDy * cap + r], rays[kDz * cap + r]);
    return grid_pos(c, o, d, t);
}

// Density MLP: y = W2 relu(W1 f).
__device__ __forceinline__ void density_mlp(const SmemW& s, const float* f, float* y) {
#pragma unroll
    for (int m = 0; m < kGeo; ++m) y[m] = 0.f;
#pragma unroll 2
    for (int j = 0; j < kHid; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < kEnc; ++k) a += s.W1[j * kEnc + k] * f[k];
        a = fmaxf(a, 0.f);
#pragma unroll
        for (int m = 0; m < kGeo; ++m) y[m] += s.W2T[j * kGeo + m] * a;
    }
}

// Colour MLP: rgb = sigmoid(W5 relu(W4 relu(W3 x3))).
__device__ __forceinline__ float3 color_mlp(const SmemW& s, const float* x3) {
    float h4[kHid];
#pragma unroll
    for (int i = 0; i < kHid; ++i) h4[i] = 0.f;
#pragma unroll 1
    for (int j = 0; j < kHid; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) a += s.W3[j * 32 + k] * x3[k];
        a = fmaxf(a, 0.f);
#pragma unroll
        for (int i = 0; i < kHid; ++i) h4[i] += s.W4T[j * kHid + i] * a;
    }
    float z0 = 0.f, z1 = 0.f, z2 = 0.f;
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
        const float h = fmaxf(h4[i], 0.f);
        z0 += s.W5[i] * h;
        z1 += s.W5[kHid + i] * h;
        z2 += s.W5[2 * kHid + i] * h;
    }
    return make_float3(sigmoidf_(z0), sigmoidf_(z1), sigmoidf_(z2));
}

// kSel: the samples sel[0 .. *n_total) of the batch instead of 0 .. *n_total (a
// render's passes); the encodings are not stored then.
template <bool kSel>
__global__ void __launch_bounds__(128) k_field_fwd_fp32(DevCfg c, const float* __restrict__ params,
                                                        const float* __restrict__ rays, uint32_t cap,
                                                        const uint32_t* __restrict__ n_total,
                                                        const uint32_t* __restrict__ ray_id,
                                                        const float* __restrict__ ts,
                                                        float4* __restrict__ sig_rgb,
                                                        float* __restrict__ feat_out,
                                                        const uint32_t* __restrict__ sel) {
    extern __shared__ float smem_raw[];
    SmemW& s = *reinterpret_cast<SmemW*>(smem_raw);
    const float* mlp = params + (size_t)c.L * c.T * 2;
    load_weights(s, mlp);
    __syncthreads();
    const uint32_t n = *n_total;
    const float2* tables = reinterpret_cast<const float2*>(params);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const uint32_t i = kSel ? sel[j] : j;
        const uint32_t r = ray_id[i];
        float3 d;
        const float3 x = sample_pos(c, rays, cap, r, ts[i], d);
        float f[kEnc];
        hash_encode(c, tables, x, f);
        if (!kSel && feat_out) {
            float4* fo = reinterpret_cast<float4*>(feat_out + (size_t)i * kEnc);
#pragma unroll
            for (int k = 0; k < kEnc / 4; ++k) fo[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
        }
        float x3[32];
        density_mlp(s, f, x3);
        sh16(d.x, d.y, d.z, x3 + kGeo);
        const float sigma = expf(fminf(x3[0], kSigmaHMax));
        const float3 rgb = color_mlp(s, x3);
        sig_rgb[i] = make_float4(sigma, rgb.x, rgb.y, rgb.z);
    }
}

void launch_field_fwd_fp32(const DevCfg& c, const float* params, uint32_t n_rays, const StepBufs& b,
                           bool store_feat, int n_sm, cudaStream_t st) {
    const size_t smem = sizeof(SmemW);
    // per call: the attribute belongs to the current device (cheap next to the kernel)
    cudaFuncSetAttribute(k_field_fwd_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    (void)n_rays;
    k_field_fwd_fp32<false><<<n_sm * 8, 128, smem, st>>>(c, params, b.rays, b.cap_rays, b.offsets + n_rays,
                                                        b.ray_id, b.t, b.sig_rgb, store_feat ? b.feat : nullptr,
                                                        nullptr);
}

void launch_field_fwd_fp32_sel(const DevCfg& c, const float* params, const uint32_t* sel, const uint32_t* n_sel,
                               const StepBufs& b, int n_sm, cudaStream_t st) {
    const size_t smem = sizeof(SmemW);
    cudaFuncSetAttribute(k_field_fwd_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_field_fwd_fp32<true><<<n_sm * 8, 128, smem, st>>>(c, params, b.rays, b.cap_rays, n_sel, b.ray_id, b.t,
                                                       b.sig_rgb, nullptr, sel);
}

// ------------------------------------------------------------------ backward
constexpr int kTile = 128;
constexpr int kRow = 261;  // per-sample activation row (odd stride: conflict-free per-thread access)
// Row layout: f[0,32) h1[32,96) x3[96,128) h3[128,192) h4[192,256) dz[256,259)
constexpr int kRf = 0, kRh1 = 32, kRx3 = 96, kRh3 = 128, kRh4 = 192, kRdz = 256;

struct SmemBwd {
    float W[kMlpParams];          // plain (out, in) layout as in the parameter buffer
    float dW[kMlpParams];         // gradient accumulators
    float act[kTile * kRow];
};

// dW[n][k] += sum_s A[s][a_off + n] * B[s][b_off + k] for an (NO x NI) weight,
// 4x4 register blocks distributed over the block's threads.
__device__ __forceinline__ void tile_outer(const float* __restrict__ act, int a_off, int b_off,
                                           int NO, int NI, float* __restrict__ dW) {
    const int nb_i = NI / 4;
    const int n_blocks = (NO / 4) * nb_i;
    for (int blk = threadIdx.x; blk < n_blocks; blk += blockDim.x) {
        const int n0 = (blk / nb_i) * 4, k0 = (blk % nb_i) * 4;
        float acc[4][4] = {};
        for (int sidx = 0; sidx < kTile; ++sidx) {
            const float* row = act + sidx * kRow;
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = row[a_off + n0 + q];
                b[q] = row[b_off + k0 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) dW[(n0 + p) * NI + k0 + q] += acc[p][q];
    }
}

// kPose: also writes, per sample, dL/dp (world position) and the view-direction
// gradient through the SH encoding into pose_s[2 i], pose_s[2 i + 1].
template <bool kPose>
__global__ void __launch_bounds__(kTile) k_field_bwd_fp32(DevCfg c, const float* __restrict__ params,
                                                          float* __restrict__ grads,
                                                          const float* __restrict__ rays, uint32_t cap,
                                                          const uint32_t* __restrict__ n_total,
                                                          const uint32_t* __restrict__ ray_id,
                                                          const float* __restrict__ ts,
                                                          const float* __restrict__ feat,
                                                          const float4* __restrict__ dsig_rgb,
                                                          float4* __restrict__ pose_s) {
    extern __shared__ float smem_raw[];
    SmemBwd& s = *reinterpret_cast<SmemBwd*>(smem_raw);
    const float* mlp = params + (size_t)c.L * c.T * 2;
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        s.W[i] = mlp[i];
        s.dW[i] = 0.f;
    }
    __syncthreads();
    const float* W1 = s.W + kOffW1;
    const float* W2 = s.W + kOffW2;
    const float* W3 = s.W + kOffW3;
    const float* W4 = s.W + kOffW4;
    const float* W5 = s.W + kOffW5;
    const uint32_t n = *n_total;
    float2* gtables = reinterpret_cast<float2*>(grads);
    float* row = s.act + threadIdx.x * kRow;
    const uint32_t n_tiles = (n + kTile - 1) / kTile;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t i = tile * kTile + threadIdx.x;
        const bool valid = i < n;
        float3 x = make_float3(0.f, 0.f, 0.f);
        float3 d = make_float3(0.f, 0.f, 0.f);
        float dsig = 0.f, sigma = 0.f;
        bool sig_grad_off = false;
        if (valid) {
            // ---- recompute the forward pass into this sample's row
            x = sample_pos(c, rays, cap, ray_id[i], ts[i], d);
            float f[kEnc];
            const float4* fi = reinterpret_cast<const float4*>(feat + (size_t)i * kEnc);
#pragma unroll
            for (int k = 0; k < kEnc / 4; ++k) {
                const float4 v = fi[k];
                f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < kEnc; ++k) row[kRf + k] = f[k];
            float y[kGeo];
#pragma unroll
            for (int m = 0; m < kGeo; ++m) y[m] = 0.f;
#pragma unroll 2
            for (int j = 0; j < kHid; ++j) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < kEnc; ++k) a += W1[j * kEnc + k] * f[k];
                a = fmaxf(a, 0.f);
                row[kRh1 + j] = a;
#pragma unroll
                for (int m = 0; m < kGeo; ++m) y[m] += W2[m * kHid + j] * a;
            }
            float x3[32];
#pragma unroll
            for (int m = 0; m < kGeo; ++m) x3[m] = y[m];
            sh16(d.x, d.y, d.z, x3 + kGeo);
#pragma unroll
            for (int k = 0; k < 32; ++k) row[kRx3 + k] = x3[k];
            sigma = expf(fminf(x3[0], kSigmaHMax));
            if (!(x3[0] < kSigmaHMax)) sig_grad_off = true;
            float h4[kHid];
#pragma unroll
            for (int q = 0; q < kHid; ++q) h4[q] = 0.f;
#pragma unroll 1
            for (int j = 0; j < kHid; ++j) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < 32; ++k) a += W3[j * 32 + k] * x3[k];
                a = fmaxf(a, 0.f);
                row[kRh3 + j] = a;
#pragma unroll
                for (int q = 0; q < kHid; ++q) h4[q] += W4[q * kHid + j] * a;
            }
            float z0 = 0.f, z1 = 0.f, z2 = 0.f;
#pragma unroll
            for (int q = 0; q < kHid; ++q) {
                const float h = fmaxf(h4[q], 0.f);
                row[kRh4 + q] = h;
                z0 += W5[q] * h;
                z1 += W5[kHid + q] * h;
                z2 += W5[2 * kHid + q] * h;
            }
            const float4 g = dsig_rgb[i];
            dsig = g.x;
            const float c0 = sigmoidf_(z0), c1 = sigmoidf_(z1), c2 = sigmoidf_(z2);
            row[kRdz + 0] = g.y * c0 * (1.f - c0);
            row[kRdz + 1] = g.z * c1 * (1.f - c1);
            row[kRdz + 2] = g.w * c2 * (1.f - c2);
        } else {
            for (int k = 0; k < kRow; ++k) row[k] = 0.f;
        }
        __syncthreads();
        // dW5[c][q] += sum_s dz[s][c] h4[s][q]
        for (int e = threadIdx.x; e < 3 * kHid; e += blockDim.x) {
            const int cc = e / kHid, q = e % kHid;
            float acc = 0.f;
            for (int sidx = 0; sidx < kTile; ++sidx)
                acc += s.act[sidx * kRow + kRdz + cc] * s.act[sidx * kRow + kRh4 + q];
            s.dW[kOffW5 + e] += acc;
        }
        __syncthreads();
        // dA4 = (W5^T dz) * [h4 > 0]  (overwrites h4)
        {
            const float dz0 = row[kRdz], dz1 = row[kRdz + 1], dz2 = row[kRdz + 2];
#pragma unroll 8
            for (int q = 0; q < kHid; ++q) {
                const float dh = W5[q] * dz0 + W5[kHid + q] * dz1 + W5[2 * kHid + q] * dz2;
                row[kRh4 + q] = row[kRh4 + q] > 0.f ? dh : 0.f;
            }
        }
        __syncthreads();
        tile_outer(s.act, kRh4, kRh3, kHid, kHid, s.dW + kOffW4);   // dW4 = dA4^T h3
        __syncthreads();
        // dA3 = (W4^T dA4) * [h3 > 0]  (overwrites h3)
        {
            float dh[kHid];
#pragma unroll
            for (int q = 0; q < kHid; ++q) dh[q] = 0.f;
#pragma unroll 1
            for (int nn = 0; nn < kHid; ++nn) {
                const float a = row[kRh4 + nn];
#pragma unroll
                for (int q = 0; q < kHid; ++q) dh[q] += W4[nn * kHid + q] * a;
            }
#pragma unroll
            for (int q = 0; q < kHid; ++q) row[kRh3 + q] = row[kRh3 + q] > 0.f ? dh[q] : 0.f;
        }
        __syncthreads();
        tile_outer(s.act, kRh3, kRx3, kHid, 32, s.dW + kOffW3);     // dW3 = dA3^T x3
        __syncthreads();
        // dy = (W3^T dA3)[0:16], dy_0 += dL/dsigma * sigma  (overwrites x3[0:16])
        {
            float dy[kGeo];
#pragma unroll
            for (int m = 0; m < kGeo; ++m) dy[m] = 0.f;
#pragma unroll 4
            for (int nn = 0; nn < kHid; ++nn) {
                const float a = row[kRh3 + nn];
#pragma unroll
                for (int m = 0; m < kGeo; ++m) dy[m] += W3[nn * 32 + m] * a;
            }
            if (!sig_grad_off) dy[0] += dsig * sigma;
            if (kPose) {
                // the SH inputs' gradient (W3^T dA3)[16:32] -> the view-direction gradient
                float dsh[kSH];
#pragma unroll
                for (int m = 0; m < kSH; ++m) dsh[m] = 0.f;
#pragma unroll 4
                for (int nn = 0; nn < kHid; ++nn) {
                    const float a = row[kRh3 + nn];
#pragma unroll
                    for (int m = 0; m < kSH; ++m) dsh[m] += W3[nn * 32 + kGeo + m] * a;
                }
                const float3 gd = sh16_vjp(d.x, d.y, d.z, dsh);
                if (valid) pose_s[2 * (size_t)i + 1] = make_float4(gd.x, gd.y, gd.z, 0.f);
            }
#pragma unroll
            for (int m = 0; m < kGeo; ++m) row[kRx3 + m] = dy[m];
        }
        __syncthreads();
        tile_outer(s.act, kRx3, kRh1, kGeo, kHid, s.dW + kOffW2);   // dW2 = dy^T h1
        __syncthreads();
        // dA1 = (W2^T dy) * [h1 > 0]  (overwrites h1)
        {
            float dy[kGeo];
#pragma unroll
            for (int m = 0; m < kGeo; ++m) dy[m] = row[kRx3 + m];
#pragma unroll 4
            for (int j = 0; j < kHid; ++j) {
                float a = 0.f;
#pragma unroll
                for (int m = 0; m < kGeo; ++m) a += W2[m * kHid + j] * dy[m];
                row[kRh1 + j] = row[kRh1 + j] > 0.f ? a : 0.f;
            }
        }
        __syncthreads();
        tile_outer(s.act, kRh1, kRf, kHid, kEnc, s.dW + kOffW1);    // dW1 = dA1^T f
        // df = W1^T dA1, scattered into the tables (all lanes take part)
        {
            float df[kEnc];
#pragma unroll
            for (int k = 0; k < kEnc; ++k) df[k] = 0.f;
            if (valid) {
#pragma unroll 2
                for (int j = 0; j < kHid; ++j) {
                    const float a = row[kRh1 + j];
#pragma unroll
                    for (int k = 0; k < kEnc; ++k) df[k] += W1[j * kEnc + k] * a;
                }
            }
            hash_scatter_warp<false>(c, gtables, x, [&](int l) { return make_float2(df[2 * l], df[2 * l + 1]); },
                                     valid);
            if (kPose && valid) {
                const float3 gx = hash_grad_x(c, reinterpret_cast<const float2*>(params), x, df);
                pose_s[2 * (size_t)i] = make_float4(gx.x * c.inv_size, gx.y * c.inv_size, gx.z * c.inv_size, 0.f);
            }
        }
        __syncthreads();
    }
    float* gmlp = grads + (size_t)c.L * c.T * 2;
    for (int e = threadIdx.x; e < kMlpParams; e += blockDim.x) {
        const float v = s.dW[e];
        if (v != 0.f) atomicAdd(gmlp + e, v);
    }
}

void launch_field_bwd_fp32(const DevCfg& c, const float* params, float* grads, uint32_t n_rays,
                           const StepBufs& b, int n_sm, cudaStream_t st, bool pose) {
    const size_t smem = sizeof(SmemBwd);
    // per call: the attribute belongs to the current device (cheap next to the kernel)
    cudaFuncSetAttribute(k_field_bwd_fp32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_field_bwd_fp32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (pose)
        k_field_bwd_fp32<true><<<n_sm, kTile, smem, st>>>(c, params, grads, b.rays, b.cap_rays, b.offsets + n_rays,
                                                          b.ray_id, b.t, b.feat, b.dsig_rgb, b.pose_s);
    else
        k_field_bwd_fp32<false><<<n_sm, kTile, smem, st>>>(c, params, grads, b.rays, b.cap_rays,
                                                           b.offsets + n_rays, b.ray_id, b.t, b.feat, b.dsig_rgb,
                                                           nullptr);
}

}  // namespace nm
