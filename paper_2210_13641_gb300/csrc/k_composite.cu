// k_composite.cu - alpha compositing of colour and expected depth (Sec. 3.2,
// Eq. transmittance), the mapping loss of Eq. (mapping_loss) and its gradient with
// respect to each sample's density and colour (steps a7-a9).  FP32, one thread per
// ray over that ray's contiguous samples.
#include "internal.h"

namespace nm {

// Forward: alpha_i = 1 - exp(-sigma_i delta), T_i = exp(-sum_{j<i} sigma_j delta),
// w_i = T_i alpha_i; I* = sum w_i c_i, D* = sum w_i t_i, acc = sum w_i.
// Loss per ray: ||I - I*||^2 + lambda_D (D - D*)^2 / Sigma_D; the batch loss is the
// mean over rays.  Backward (reverse pass over the ray's samples, suffix sums
// S_i = sum_{j>i} w_j c_j and the same with t): dL/dc_i = w_i g_I and
// dL/dsigma_i = delta (g_I . (T_{i+1} c_i - S^c_i) + g_D (T_{i+1} t_i - S^d_i)), with
// g_I = -2 (I - I*) / R, g_D = -2 lambda_D (D - D*) / (Sigma_D R).
// loss[0] receives the batch loss; loss[1] and loss[2] the largest density and colour
// seed magnitudes over samples (FP32 bits), from which the tensor-core backward picks
// its gradient scales.
template <bool kBackward>
__global__ void k_composite(DevCfg c, uint32_t n_rays, const float* __restrict__ rays, uint32_t cap,
                            const uint32_t* __restrict__ offsets, const float* __restrict__ ts,
                            const float4* __restrict__ sig_rgb, float4* __restrict__ scratch,
                            float* __restrict__ ray_out, float* __restrict__ loss) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    float gmax = 0.f;  // largest per-sample density seed |dL/dsigma * sigma|
    float cmax = 0.f;  // largest per-sample colour seed |dL/dc|
    if (r < n_rays) {
        const uint32_t a = offsets[r], b = offsets[r + 1];
        const float delta = c.step_t;
        float run = 0.f, Ir = 0.f, Ig = 0.f, Ib = 0.f, Dh = 0.f, acc = 0.f;
        for (uint32_t s = a; s < b; ++s) {
            const float T = expf(-run);
            if (!kBackward && T < c.t_min) break;
            const float4 v = sig_rgb[s];
            const float tau = v.x * delta;
            const float w = T * -expm1f(-tau);
            Ir += w * v.y;
            Ig += w * v.z;
            Ib += w * v.w;
            Dh += w * ts[s];
            acc += w;
            run += tau;
            if (kBackward) scratch[s] = make_float4(w, expf(-run), 0.f, 0.f);
        }
        ray_out[0 * cap + r] = Ir;
        ray_out[1 * cap + r] = Ig;
        ray_out[2 * cap + r] = Ib;
        ray_out[3 * cap + r] = Dh;
        ray_out[4 * cap + r] = acc;
        if (kBackward) {
            const float er = rays[kIr * cap + r] - Ir;
            const float eg = rays[kIg * cap + r] - Ig;
            const float eb = rays[kIb * cap + r] - Ib;
            const float ed = rays[kD * cap + r] - Dh;
            const float V = rays[kV * cap + r];
            l = er * er + eg * eg + eb * eb + c.lambda_d * ed * ed / V;
            const float inv_n = 1.f / (float)n_rays;
            const float gr = -2.f * er * inv_n, gg = -2.f * eg * inv_n, gb = -2.f * eb * inv_n;
            const float gd = -2.f * c.lambda_d * ed / V * inv_n;
            float Sr = 0.f, Sg = 0.f, Sb = 0.f, Sd = 0.f;
            for (uint32_t s = b; s-- > a;) {
                const float4 v = sig_rgb[s];
                const float4 q = scratch[s];
                const float w = q.x, Tn = q.y, t = ts[s];
                const float dsig = delta * (gr * (Tn * v.y - Sr) + gg * (Tn * v.z - Sg) +
                                            gb * (Tn * v.w - Sb) + gd * (Tn * t - Sd));
                scratch[s] = make_float4(dsig, w * gr, w * gg, w * gb);
                gmax = fmaxf(gmax, fabsf(dsig * v.x));
                cmax = fmaxf(cmax, fmaxf(fabsf(w * gr), fmaxf(fabsf(w * gg), fabsf(w * gb))));
                Sr += w * v.y;
                Sg += w * v.z;
                Sb += w * v.w;
                Sd += w * t;
            }
        }
    }
    if (kBackward) {
        // mean over rays: warp sum, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, o);
            gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            if (l != 0.f) atomicAdd(loss, l / (float)n_rays);
            // non-negative floats order like their bit patterns
            if (gmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(loss) + 1, __float_as_uint(gmax));
            if (cmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(loss) + 2, __float_as_uint(cmax));
        }
    }
}

void launch_composite(const DevCfg& c, uint32_t n_rays, bool backward, const StepBufs& b,
                      cudaStream_t s) {
    const uint32_t grid = (n_rays + 127) / 128;
    if (backward) {
        cudaMemsetAsync(b.loss, 0, 3 * sizeof(float), s);
        k_composite<true><<<grid, 128, 0, s>>>(c, n_rays, b.rays, b.cap_rays, b.offsets, b.t,
                                               b.sig_rgb, b.dsig_rgb, b.ray_out, b.loss);
    } else {
        k_composite<false><<<grid, 128, 0, s>>>(c, n_rays, b.rays, b.cap_rays, b.offsets, b.t,
                                                b.sig_rgb, nullptr, b.ray_out, nullptr);
    }
}

}  // namespace nm

namespace nm {

// Render output: per-ray planes -> interleaved RGB [n][3], depth [n], opacity [n].
__global__ void k_write_render(const float* __restrict__ ray_out, uint32_t cap, uint32_t n,
                               float* __restrict__ rgb, float* __restrict__ depth,
                               float* __restrict__ acc) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    if (rgb) {
        rgb[3 * r] = ray_out[r];
        rgb[3 * r + 1] = ray_out[cap + r];
        rgb[3 * r + 2] = ray_out[2 * cap + r];
    }
    if (depth) depth[r] = ray_out[3 * cap + r];
    if (acc) acc[r] = ray_out[4 * cap + r];
}

void launch_write_render(const StepBufs& b, uint32_t n, float* rgb, float* depth, float* acc,
                         cudaStream_t s) {
    k_write_render<<<(n + 255) / 256, 256, 0, s>>>(b.ray_out, b.cap_rays, n, rgb, depth, acc);
}

}  // namespace nm
