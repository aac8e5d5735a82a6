// k_pose.cu - the keyframe pose gradient of the mapping loss (joint pose refinement:
// Sec. 3.2 minimises L_M over the poses T as well as the map).  The field backward
// kernels leave, per sample, dL/dp (the gradient at the sample's world position) and
// the view-direction gradient that reaches the sample through its SH encoding; here
// one warp per ray sums them along the ray (p = o + t d, t fixed), giving dL/do and
// dL/dd, and turns them into the gradient of the ray's keyframe pose under the left
// world-frame perturbation T <- exp(xi) T, xi = (rho, phi):
//   dL/drho = dL/do,   dL/dphi = o x dL/do + d x dL/dd,
// accumulated per keyframe slot with FP32 atomics.
#include "internal.h"

namespace nm {

namespace {
constexpr unsigned kFullMask = 0xffffffffu;
}

__global__ void __launch_bounds__(256) k_pose_reduce(uint32_t n_rays, const float* __restrict__ rays, uint32_t cap,
                                                     const uint32_t* __restrict__ offsets,
                                                     const float* __restrict__ ts,
                                                     const float4* __restrict__ pose_s, float* __restrict__ pose_g) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rays; r += n_warps) {
        const uint32_t a = offsets[r], b = offsets[r + 1];
        if (a == b) continue;  // warp-uniform
        float go[3] = {0.f, 0.f, 0.f}, gd[3] = {0.f, 0.f, 0.f};
        for (uint32_t s = a + lane; s < b; s += 32) {
            const float4 p = pose_s[2 * s], q = pose_s[2 * s + 1];
            const float t = ts[s];
            go[0] += p.x;
            go[1] += p.y;
            go[2] += p.z;
            gd[0] += t * p.x + q.x;
            gd[1] += t * p.y + q.y;
            gd[2] += t * p.z + q.z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                go[k] += __shfl_xor_sync(kFullMask, go[k], o);
                gd[k] += __shfl_xor_sync(kFullMask, gd[k], o);
            }
        }
        if (lane == 0) {
            const float ox = rays[kOx * cap + r], oy = rays[kOy * cap + r], oz = rays[kOz * cap + r];
            const float dx = rays[kDx * cap + r], dy = rays[kDy * cap + r], dz = rays[kDz * cap + r];
            const uint32_t kf = __float_as_uint(rays[kKf * cap + r]);
            float* g = pose_g + 8 * (size_t)kf;
            atomicAdd(g + 0, go[0]);
            atomicAdd(g + 1, go[1]);
            atomicAdd(g + 2, go[2]);
            atomicAdd(g + 3, (oy * go[2] - oz * go[1]) + (dy * gd[2] - dz * gd[1]));
            atomicAdd(g + 4, (oz * go[0] - ox * go[2]) + (dz * gd[0] - dx * gd[2]));
            atomicAdd(g + 5, (ox * go[1] - oy * go[0]) + (dx * gd[1] - dy * gd[0]));
        }
    }
}

void launch_pose_reduce(const DevCfg& c, uint32_t n_rays, const StepBufs& b, float* pose_g, cudaStream_t s) {
    (void)c;
    uint32_t grid = (n_rays + 7) / 8;
    if (grid > 152u * 16u) grid = 152u * 16u;
    k_pose_reduce<<<grid, 256, 0, s>>>(n_rays, b.rays, b.cap_rays, b.offsets, b.t, b.pose_s, pose_g);
}

}  // namespace nm
