// k_composite.cu - alpha compositing of colour and expected depth (Sec. 3.2,
// Eq. transmittance), the mapping loss of Eq. (mapping_loss) and its gradient with
// respect to each sample's density and colour (steps a7-a9).  FP32, one warp per
// ray: the ray's contiguous samples are taken 32 at a time (coalesced), the
// transmittance exponent is a warp prefix sum carried from chunk to chunk, and the
// backward's suffix sums are warp suffix scans over the chunks in reverse order.
#include "internal.h"

namespace nm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCompositeWarps = 8;  // warps (rays in flight) per block

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

// Inclusive prefix sum over lanes 0..lane.
__device__ __forceinline__ float warp_prefix(float x, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFull, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

// Inclusive suffix sum over lanes lane..31.
__device__ __forceinline__ float warp_suffix(float x, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(kFull, x, o);
        if (lane + (uint32_t)o < 32u) x += y;
    }
    return x;
}

}  // namespace

// Forward: alpha_i = 1 - exp(-sigma_i delta), T_i = exp(-sum_{j<i} sigma_j delta),
// w_i = T_i alpha_i; I* = sum w_i c_i, D* = sum w_i t_i, acc = sum w_i.
// Loss per ray: ||I - I*||^2 + lambda_D (D - D*)^2 / Sigma_D; the batch loss is the
// mean over rays.  Backward (suffix sums S_i = sum_{j>i} w_j c_j and the same with
// t, taken as suffix scans, never as a total minus a prefix): dL/dc_i = w_i g_I and
// dL/dsigma_i = delta (g_I . (T_{i+1} c_i - S^c_i) + g_D (T_{i+1} t_i - S^d_i)), with
// g_I = -2 (I - I*) / R, g_D = -2 lambda_D (D - D*) / (Sigma_D R).
// loss[0] receives the batch loss; loss[1] and loss[2] the largest density and colour
// seed magnitudes over samples (FP32 bits), from which the tensor-core backward picks
// its gradient scales.  In the forward-only form (render) a ray stops at the first
// sample whose transmittance is below t_min.  scratch holds (w_i, T_{i+1}) between
// the two passes and then (dL/dsigma_i, dL/dc_i).
// kGroup (render only): the rays of a grouped render, each taking its sample spacing
// and termination threshold from its piece (items[ray's kKf plane]).
// kSplit (render only) composites in two passes around the forward's two passes:
// 1 takes the first kRenderFirst samples of each ray and writes, per ray, the number of
// samples still to evaluate into `live` (0 when the ray stopped at the threshold or
// has no more samples); 2 takes the rays with live > 0 from their first sample to
// their last.  A ray is composited in 32-sample chunks from its first sample in
// every pass, so each result equals the single pass's.
static_assert(kRenderFirst % 32 == 0, "the first pass must end at a chunk boundary of the compositing");

template <bool kBackward, bool kGroup = false, int kSplit = 0>
__global__ void __launch_bounds__(kCompositeWarps * 32) k_composite(
    DevCfg c, uint32_t n_rays, const float* __restrict__ rays, uint32_t cap, const uint32_t* __restrict__ offsets,
    const float* __restrict__ ts, const float4* __restrict__ sig_rgb, float4* __restrict__ scratch,
    float* __restrict__ ray_out, float* __restrict__ loss, float* __restrict__ partials,
    const GroupItem* __restrict__ items = nullptr, uint32_t* __restrict__ live = nullptr) {
    static_assert(!(kBackward && kGroup), "grouped compositing is forward only");
    static_assert(!(kBackward && kSplit), "two-pass compositing is forward only");
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const uint32_t n_warps = gridDim.x * kCompositeWarps;
    float delta = c.step_t, t_min = c.t_min;
    float l = 0.f;     // this warp's loss sum (lane 0)
    float gmax = 0.f;  // largest per-sample density seed |dL/dsigma * sigma|
    float cmax = 0.f;  // largest per-sample colour seed |dL/dc|
    for (uint32_t r = blockIdx.x * kCompositeWarps + wib; r < n_rays; r += n_warps) {
        if (kGroup) {
            const GroupItem& it = items[__float_as_uint(rays[kKf * cap + r])];
            delta = it.c.step_t;
            t_min = it.c.t_min;
        }
        if (kSplit == 2 && live[r] == 0) continue;  // warp-uniform
        const uint32_t a = offsets[r], b_all = offsets[r + 1];
        const uint32_t b = kSplit == 1 ? min(b_all, a + kRenderFirst) : b_all;
        float carry = 0.f;  // sum of sigma delta over the earlier chunks
        float Ir = 0.f, Ig = 0.f, Ib = 0.f, Dh = 0.f, acc = 0.f;
        bool stopped = false;
        for (uint32_t base = a; base < b; base += 32) {
            const uint32_t s = base + lane;
            const bool in = s < b;
            const float4 v = in ? sig_rgb[s] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float t = in ? ts[s] : 0.f;
            const float tau = v.x * delta;
            const float incl = warp_prefix(tau, lane);
            float excl = __shfl_up_sync(kFull, incl, 1);
            if (lane == 0) excl = 0.f;
            const float T = expf(-(carry + excl));
            bool live = in;
            if (!kBackward) live = live && !(T < t_min);
            const float w = live ? T * -expm1f(-tau) : 0.f;
            Ir += w * v.y;
            Ig += w * v.z;
            Ib += w * v.w;
            Dh += w * t;
            acc += w;
            if (kBackward && in) scratch[s] = make_float4(w, expf(-(carry + incl)), 0.f, 0.f);
            carry += __shfl_sync(kFull, incl, 31);
            if (!kBackward && __any_sync(kFull, in && T < t_min)) {
                stopped = true;
                break;
            }
        }
        if (kSplit == 1 && lane == 0) live[r] = stopped ? 0u : b_all - b;
        Ir = warp_sum(Ir);
        Ig = warp_sum(Ig);
        Ib = warp_sum(Ib);
        Dh = warp_sum(Dh);
        acc = warp_sum(acc);
        if (lane == 0) {
            ray_out[0 * cap + r] = Ir;
            ray_out[1 * cap + r] = Ig;
            ray_out[2 * cap + r] = Ib;
            ray_out[3 * cap + r] = Dh;
            ray_out[4 * cap + r] = acc;
        }
        if (kBackward) {
            const float er = rays[kIr * cap + r] - Ir;
            const float eg = rays[kIg * cap + r] - Ig;
            const float eb = rays[kIb * cap + r] - Ib;
            const float ed = rays[kD * cap + r] - Dh;
            const float V = rays[kV * cap + r];
            if (lane == 0) l += er * er + eg * eg + eb * eb + c.lambda_d * ed * ed / V;
            const float inv_n = 1.f / (float)n_rays;
            const float gr = -2.f * er * inv_n, gg = -2.f * eg * inv_n, gb = -2.f * eb * inv_n;
            const float gd = -2.f * c.lambda_d * ed / V * inv_n;
            float Sr = 0.f, Sg = 0.f, Sb = 0.f, Sd = 0.f;  // suffix sums of the later chunks
            if (b > a) {
                for (uint32_t base = a + ((b - a - 1) & ~31u);; base -= 32) {
                    const uint32_t s = base + lane;
                    const bool in = s < b;
                    const float4 v = in ? sig_rgb[s] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 q = in ? scratch[s] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float t = in ? ts[s] : 0.f;
                    const float w = q.x, Tn = q.y;
                    const float xr = warp_suffix(w * v.y, lane), xg = warp_suffix(w * v.z, lane);
                    const float xb = warp_suffix(w * v.w, lane), xd = warp_suffix(w * t, lane);
                    float nr = __shfl_down_sync(kFull, xr, 1), ng = __shfl_down_sync(kFull, xg, 1);
                    float nb = __shfl_down_sync(kFull, xb, 1), nd = __shfl_down_sync(kFull, xd, 1);
                    if (lane == 31) nr = ng = nb = nd = 0.f;
                    const float dsig = delta * (gr * (Tn * v.y - (Sr + nr)) + gg * (Tn * v.z - (Sg + ng)) +
                                                gb * (Tn * v.w - (Sb + nb)) + gd * (Tn * t - (Sd + nd)));
                    if (in) {
                        scratch[s] = make_float4(dsig, w * gr, w * gg, w * gb);
                        gmax = fmaxf(gmax, fabsf(dsig * v.x));
                        cmax = fmaxf(cmax, fmaxf(fabsf(w * gr), fmaxf(fabsf(w * gg), fabsf(w * gb))));
                    }
                    Sr += __shfl_sync(kFull, xr, 0);
                    Sg += __shfl_sync(kFull, xg, 0);
                    Sb += __shfl_sync(kFull, xb, 0);
                    Sd += __shfl_sync(kFull, xd, 0);
                    if (base == a) break;
                }
            }
        }
    }
    if (kBackward) {
        // Per block: warp sums / maxima through shared memory into partials[block];
        // the last block to finish reduces all partials in a fixed order, so the
        // batch loss does not depend on the order in which blocks finish.
        __shared__ float sl[kCompositeWarps], sg[kCompositeWarps], sc[kCompositeWarps];
        __shared__ bool last;
        l = warp_sum(l);
        gmax = warp_max(gmax);
        cmax = warp_max(cmax);
        if (lane == 0) {
            sl[wib] = l;
            sg[wib] = gmax;
            sc[wib] = cmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float L = 0.f, G = 0.f, C = 0.f;
            for (int i = 0; i < kCompositeWarps; ++i) {
                L += sl[i];
                G = fmaxf(G, sg[i]);
                C = fmaxf(C, sc[i]);
            }
            partials[4 * blockIdx.x + 0] = L;
            partials[4 * blockIdx.x + 1] = G;
            partials[4 * blockIdx.x + 2] = C;
            __threadfence();
            const uint32_t ticket = atomicAdd(reinterpret_cast<unsigned int*>(loss) + 3, 1u);
            last = ticket == gridDim.x - 1;
        }
        __syncthreads();
        if (last && wib == 0) {
            __threadfence();
            float L = 0.f, G = 0.f, C = 0.f;
            for (uint32_t i = lane; i < gridDim.x; i += 32) {
                L += __ldcg(partials + 4 * i + 0);
                G = fmaxf(G, __ldcg(partials + 4 * i + 1));
                C = fmaxf(C, __ldcg(partials + 4 * i + 2));
            }
            L = warp_sum(L);
            G = warp_max(G);
            C = warp_max(C);
            if (lane == 0) {
                loss[0] = L / (float)n_rays;
                // non-negative floats order like their bit patterns
                reinterpret_cast<unsigned int*>(loss)[1] = __float_as_uint(G);
                reinterpret_cast<unsigned int*>(loss)[2] = __float_as_uint(C);
                reinterpret_cast<unsigned int*>(loss)[3] = 0u;
            }
        }
    }
}

static uint32_t composite_grid(uint32_t n_rays) {
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 148;
    uint32_t grid = (n_rays + kCompositeWarps - 1) / kCompositeWarps;
    uint32_t cap = (uint32_t)n_sm * 8;  // persistent warps loop over the rays
    if (cap > kCompositeMaxBlocks) cap = kCompositeMaxBlocks;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    return grid;
}

void launch_composite_group(const GroupItem* items, uint32_t n_rays, const StepBufs& b, cudaStream_t s, int pass,
                            uint32_t* live) {
    DevCfg unused{};
    const uint32_t grid = composite_grid(n_rays);
    if (pass == 0)
        k_composite<false, true><<<grid, kCompositeWarps * 32, 0, s>>>(
            unused, n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr, items);
    else if (pass == 1)
        k_composite<false, true, 1><<<grid, kCompositeWarps * 32, 0, s>>>(
            unused, n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr, items,
            live);
    else
        k_composite<false, true, 2><<<grid, kCompositeWarps * 32, 0, s>>>(
            unused, n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr, items,
            live);
}

void launch_composite_split(const DevCfg& c, uint32_t n_rays, int pass, uint32_t* live, const StepBufs& b,
                            cudaStream_t s) {
    const uint32_t grid = composite_grid(n_rays);
    if (pass == 1)
        k_composite<false, false, 1><<<grid, kCompositeWarps * 32, 0, s>>>(
            c, n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr, nullptr,
            live);
    else
        k_composite<false, false, 2><<<grid, kCompositeWarps * 32, 0, s>>>(
            c, n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr, nullptr,
            live);
}

void launch_composite(const DevCfg& c, uint32_t n_rays, bool backward, const StepBufs& b,
                      cudaStream_t s) {
    const uint32_t grid = composite_grid(n_rays);
    if (backward) {
        cudaMemsetAsync(b.loss, 0, 4 * sizeof(float), s);
        k_composite<true><<<grid, kCompositeWarps * 32, 0, s>>>(c, n_rays, b.rays, b.cap_rays, b.offsets, b.t,
                                                                b.sig_rgb, b.dsig_rgb, b.ray_out, b.loss,
                                                                b.partials);
    } else {
        k_composite<false><<<grid, kCompositeWarps * 32, 0, s>>>(c, n_rays, b.rays, b.cap_rays, b.offsets, b.t,
                                                                 b.sig_rgb, nullptr, b.ray_out, nullptr, nullptr);
    }
}

}  // namespace nm

namespace nm {

// Render output: per-ray planes -> interleaved RGB [n][3], depth [n], opacity [n].
// Also adds the chunk's retained sample count (offsets[n] of the march's scan) to the
// render's running total.
__global__ void k_write_render(const float* __restrict__ ray_out, uint32_t cap, uint32_t n,
                               float* __restrict__ rgb, float* __restrict__ depth,
                               float* __restrict__ acc, const uint32_t* __restrict__ chunk_total,
                               unsigned long long* __restrict__ render_samples,
                               unsigned long long* __restrict__ evaluated) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        atomicAdd(render_samples, (unsigned long long)*chunk_total);
        if (evaluated) atomicAdd(evaluated, (unsigned long long)*chunk_total);  // single pass: all of them
    }
    if (r >= n) return;
    if (rgb) {
        rgb[3 * r] = ray_out[r];
        rgb[3 * r + 1] = ray_out[cap + r];
        rgb[3 * r + 2] = ray_out[2 * cap + r];
    }
    if (depth) depth[r] = ray_out[3 * cap + r];
    if (acc) acc[r] = ray_out[4 * cap + r];
}

// Grouped render output: ray r of piece j is pixel pix0 + (r - ray0) of that piece's view.
__global__ void k_write_group(const GroupItem* __restrict__ items, const float* __restrict__ rays,
                              const float* __restrict__ ray_out, uint32_t cap, uint32_t n) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const GroupItem& it = items[__float_as_uint(rays[kKf * cap + r])];
    const size_t p = it.pix0 + (r - it.ray0);
    if (it.out_rgb) {
        it.out_rgb[3 * p] = ray_out[r];
        it.out_rgb[3 * p + 1] = ray_out[cap + r];
        it.out_rgb[3 * p + 2] = ray_out[2 * cap + r];
    }
    if (it.out_depth) it.out_depth[p] = ray_out[3 * cap + r];
}

void launch_write_group(const GroupItem* items, uint32_t n_rays, const StepBufs& b, cudaStream_t s) {
    k_write_group<<<(n_rays + 255) / 256, 256, 0, s>>>(items, b.rays, b.ray_out, b.cap_rays, n_rays);
}

void launch_write_render(const StepBufs& b, uint32_t n, float* rgb, float* depth, float* acc, bool single_pass,
                         cudaStream_t s) {
    k_write_render<<<(n + 255) / 256, 256, 0, s>>>(b.ray_out, b.cap_rays, n, rgb, depth, acc, b.offsets + n,
                                                   render_sample_counter(b),
                                                   single_pass ? render_eval_counter(b) : nullptr);
}

}  // namespace nm
