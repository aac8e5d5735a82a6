// k_rays.cu - keyframe texels, ray generation, march with occupancy test, and the
// exclusive scan that compacts the retained samples (steps a1-a2 of the mapping
// step; sampling follows Sec. 3.2 of the paper, the ray draw Sec. 3.3).
#include "internal.h"
#include "rays.cuh"

namespace nm {

// ---------------------------------------------------------------- keyframe texels
// Converts a keyframe to the store's texel layout.  z-depth is turned into distance
// along the unit ray: D = z * s, Sigma_D = var * s^2, s = ||K^-1 [u+1/2, v+1/2, 1]||.
__global__ void k_keyframe_texels(const float* __restrict__ rgb, const float* __restrict__ depth,
                                  const float* __restrict__ var, uint32_t W, uint32_t H,
                                  float fx, float fy, float cx, float cy, int depth_is_z,
                                  float4* __restrict__ tex) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= W * H) return;
    const uint32_t u = p % W, v = p / W;
    float D = depth[p], V = var[p];
    if (depth_is_z) {
        const float sx = ((float)u + 0.5f - cx) / fx;
        const float sy = ((float)v + 0.5f - cy) / fy;
        const float s2 = sx * sx + sy * sy + 1.f;
        D *= sqrtf(s2);
        V *= s2;
    }
    tex[2 * p] = make_float4(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2], D);
    tex[2 * p + 1] = make_float4(V, 0.f, 0.f, 0.f);
}

// Writes one keyframe descriptor into the device table (stream ordered; the
// descriptor travels as a kernel argument, so no host buffer has to outlive the call).
__global__ void k_set_kf_desc(KfDesc* __restrict__ table, uint32_t idx, KfDesc d) { table[idx] = d; }

void launch_set_kf_desc(KfDesc* table, uint32_t idx, const KfDesc& d, cudaStream_t s) {
    k_set_kf_desc<<<1, 1, 0, s>>>(table, idx, d);
}

void launch_keyframe_texels(const float* rgb, const float* depth, const float* var, uint32_t W,
                            uint32_t H, const float* K, int depth_is_z, float4* texels,
                            cudaStream_t s) {
    const uint32_t n = W * H;
    k_keyframe_texels<<<(n + 255) / 256, 256, 0, s>>>(rgb, depth, var, W, H, K[0], K[1], K[2],
                                                       K[3], depth_is_z, texels);
}

// Uniform draw with replacement over (keyframe, pixel): keyframe = r0 mod n_kf,
// pixel = r1 mod (W*H), with r0, r1 the two counter draws of the ray.  With an active
// list (keyframes streamed out to the host are not drawn) the k-th active keyframe is
// slot active[k]; without one, slot k.
__global__ void k_ray_gen(const KfDesc* __restrict__ kfs, const uint32_t* __restrict__ active, uint32_t n_kf,
                          uint64_t seed, uint64_t step, uint32_t n_rays, float* __restrict__ rays, uint32_t cap) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const uint64_t r0 = counter_rand(seed, step, r, 0);
    const uint64_t r1 = counter_rand(seed, step, r, 1);
    const uint32_t k = (uint32_t)(r0 % n_kf);
    const uint32_t slot = active ? active[k] : k;
    const KfDesc& kf = kfs[slot];
    const uint64_t pix = r1 % ((uint64_t)kf.W * kf.H);
    const uint32_t u = (uint32_t)(pix % kf.W), v = (uint32_t)(pix / kf.W);
    float3 o, d;
    cast_ray(kf.c2w, kf.K, u, v, o, d);
    const float4 t0 = __ldg(kf.texels + 2 * pix);
    const float4 t1 = __ldg(kf.texels + 2 * pix + 1);
    store_ray(rays, cap, r, o, d, t0, t1.x, slot);
}

void launch_ray_gen(const KfDesc* kfs, const uint32_t* active, uint32_t n_kf, uint64_t seed, uint64_t step,
                    uint32_t n_rays, const StepBufs& b, cudaStream_t s) {
    k_ray_gen<<<(n_rays + 255) / 256, 256, 0, s>>>(kfs, active, n_kf, seed, step, n_rays, b.rays,
                                                   b.cap_rays);
}

struct ViewCam {
    float c2w[12];
    float K[4];
};

// Rays of pixels p0 .. p0 + cnt - 1 of a W-wide view (row-major), as rays 0 .. cnt - 1.
__global__ void k_ray_gen_view(ViewCam cam, uint32_t W, uint32_t p0, uint32_t cnt, float* __restrict__ rays,
                               uint32_t cap) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= cnt) return;
    const uint32_t pix = p0 + r;
    float3 o, d;
    cast_ray(cam.c2w, cam.K, pix % W, pix / W, o, d);
    store_ray(rays, cap, r, o, d, make_float4(0.f, 0.f, 0.f, 0.f), 1.f, 0u);
}

void launch_ray_gen_view(const float* c2w, const float* K, uint32_t W, uint32_t p0, uint32_t cnt,
                         const StepBufs& b, cudaStream_t s) {
    ViewCam cam;
    for (int i = 0; i < 12; ++i) cam.c2w[i] = c2w[i];
    for (int i = 0; i < 4; ++i) cam.K[i] = K[i];
    k_ray_gen_view<<<(cnt + 255) / 256, 256, 0, s>>>(cam, W, p0, cnt, b.rays, b.cap_rays);
}

// ---------------------------------------------------------------- march
// One pass over the steps of each ray, one warp per ray: the 32 lanes test 32
// consecutive steps at a time and a ballot gives each retained step its place in
// the ray's slot row (max_samples floats per ray, in step order); the count goes to
// counts[r].  After the scan, k_compact copies each ray's row to its offset (one
// warp per ray, coalesced) and writes the ray index beside each sample.
__global__ void k_march(DevCfg c, const uint32_t* __restrict__ bits, uint32_t n_rays,
                        const float* __restrict__ rays, uint32_t cap, uint32_t* __restrict__ counts,
                        float* __restrict__ slots) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n_rays) return;  // whole warps
    const float3 o = make_float3(rays[kOx * cap + r], rays[kOy * cap + r], rays[kOz * cap + r]);
    const float3 d = make_float3(rays[kDx * cap + r], rays[kDy * cap + r], rays[kDz * cap + r]);
    float* row = slots + (size_t)r * c.max_samples;
    uint32_t i_lo, i_hi;
    box_step_range(c, o, d, i_lo, i_hi);
    uint32_t n = 0;
    for (uint32_t i0 = i_lo; i0 < i_hi && n < c.max_samples; i0 += 32) {
        const uint32_t i = i0 + lane;
        bool keep = false;
        float t = 0.f;
        if (i < i_hi) {
            t = sample_t(c, i);
            const float3 x = grid_pos(c, o, d, t);
            keep = in_box(c, x) && occupied(c, bits, x);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        const uint32_t pos = n + __popc(m & ((1u << lane) - 1u));
        if (keep && pos < c.max_samples) row[pos] = t;
        n += __popc(m);
    }
    if (lane == 0) counts[r] = n < c.max_samples ? n : c.max_samples;
}

__global__ void k_compact(uint32_t n_rays, uint32_t max_samples, const uint32_t* __restrict__ offsets,
                          const float* __restrict__ slots, uint32_t* __restrict__ ray_id, float* __restrict__ ts) {
    const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (r >= n_rays) return;
    const uint32_t a = offsets[r], n = offsets[r + 1] - a;
    const float* row = slots + (size_t)r * max_samples;
    for (uint32_t k = lane; k < n; k += 32) {
        ts[a + k] = row[k];
        ray_id[a + k] = r;
    }
}

// Exclusive scan of counts[0..n) into offsets[0..n], offsets[n] = total.
// Level 1: each 1024-thread block scans 4096 entries and writes its block total.

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    const uint32_t before = wid > 0 ? warp_tot[wid - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in,
                                                              uint32_t n, uint32_t* __restrict__ out,
                                                              uint32_t* __restrict__ tile_sums) {
    __shared__ uint32_t warp_tot[32];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, warp_tot, total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Level 2: one block scans the tile totals (at most kScanTile of them) in place.
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* __restrict__ tile_sums,
                                                            uint32_t n_tiles,
                                                            uint32_t* __restrict__ total_out) {
    __shared__ uint32_t warp_tot[32];
    const uint32_t base = threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n_tiles) ? tile_sums[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, warp_tot, total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n_tiles) tile_sums[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) *total_out = total;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, uint32_t n,
                           const uint32_t* __restrict__ tile_sums) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
}

// Selection of a render pass's samples: ray r contributes count[r] samples, its samples
// k0 .. k0 + count[r] - 1 (counted from its first), at sel[sel_off[r] ...].
__global__ void k_sel_emit(uint32_t n_rays, const uint32_t* __restrict__ offsets,
                           const uint32_t* __restrict__ sel_off, const uint32_t* __restrict__ count, uint32_t k0,
                           uint32_t* __restrict__ sel, unsigned long long* __restrict__ evaluated) {
    const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(evaluated, (unsigned long long)sel_off[n_rays]);
    if (r >= n_rays) return;
    const uint32_t n = count[r], dst = sel_off[r], src = offsets[r] + k0;
    for (uint32_t k = lane; k < n; k += 32) sel[dst + k] = src + k;
}

// count[r] = min(first, samples of ray r): the first pass's share of each ray.
__global__ void k_sel_first(uint32_t n_rays, const uint32_t* __restrict__ offsets, uint32_t first,
                            uint32_t* __restrict__ count) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const uint32_t n = offsets[r + 1] - offsets[r];
    count[r] = n < first ? n : first;
}

void launch_render_select(uint32_t n_rays, const uint32_t* offsets, uint32_t* count, bool first_pass,
                          uint32_t first, uint32_t* sel_off, uint32_t* tile_sums, uint32_t* sel,
                          unsigned long long* evaluated, cudaStream_t s) {
    if (first_pass) k_sel_first<<<(n_rays + 255) / 256, 256, 0, s>>>(n_rays, offsets, first, count);
    launch_scan_counts(count, n_rays, sel_off, tile_sums, s);
    k_sel_emit<<<(n_rays + 7) / 8, 256, 0, s>>>(n_rays, offsets, sel_off, count, first_pass ? 0u : first, sel,
                                                 evaluated);
}

void launch_compact(uint32_t n_rays, uint32_t row_stride, const uint32_t* offsets, const float* slots,
                    uint32_t* ray_id, float* ts, cudaStream_t s) {
    k_compact<<<(n_rays + 7) / 8, 256, 0, s>>>(n_rays, row_stride, offsets, slots, ray_id, ts);
}

void launch_march(const DevCfg& c, const uint32_t* occ_bits, uint32_t n_rays, const StepBufs& b,
                  cudaStream_t s) {
    // slot rows live in the (not yet used) per-sample colour buffer: cap_samples floats
    float* slots = reinterpret_cast<float*>(b.sig_rgb);
    k_march<<<(n_rays + 7) / 8, 256, 0, s>>>(c, occ_bits, n_rays, b.rays, b.cap_rays, b.counts, slots);
    const uint32_t n_tiles = (n_rays + kScanTile - 1) / kScanTile;  // <= kScanTile (n <= 2^24)
    k_scan_tiles<<<n_tiles, kScanThreads, 0, s>>>(b.counts, n_rays, b.offsets, b.block_sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(b.block_sums, n_tiles, b.offsets + n_rays);
    k_scan_add<<<(n_rays + 255) / 256, 256, 0, s>>>(b.offsets, n_rays, b.block_sums);
    k_compact<<<(n_rays + 7) / 8, 256, 0, s>>>(n_rays, c.max_samples, b.offsets, slots, b.ray_id, b.t);
}

}  // namespace nm

namespace nm {

// Exclusive scan of counts[0..n) into offsets[0..n] with caller-provided tile-sum
// storage of at least ceil(n / 4096) entries (used by the allocation-free march).
void launch_scan_counts(const uint32_t* counts, uint32_t n, uint32_t* offsets, uint32_t* tile_sums,
                        cudaStream_t s) {
    const uint32_t n_tiles = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<n_tiles, kScanThreads, 0, s>>>(counts, n, offsets, tile_sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(tile_sums, n_tiles, offsets + n);
    k_scan_add<<<(n + 255) / 256, 256, 0, s>>>(offsets, n, tile_sums);
}

}  // namespace nm
