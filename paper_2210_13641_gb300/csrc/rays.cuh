// rays.cuh - pinhole ray casting and the ray batch's structure-of-arrays store,
// shared by the mapping step's ray draw, the render's view rays and the grouped
// render of several views (step a1).
#pragma once

#include "internal.h"

namespace nm {

// Back-projection of the pixel centre, rotation to world, normalisation; exact
// FP32 operation order (the same integer decisions follow from these values).
__device__ __forceinline__ void cast_ray(const float* c2w, const float* K, uint32_t u,
                                         uint32_t v, float3& o, float3& d) {
    const float dx = fdiv(fsub(fadd((float)u, 0.5f), K[2]), K[0]);
    const float dy = fdiv(fsub(fadd((float)v, 0.5f), K[3]), K[1]);
    const float wx = fadd(fadd(fmul(c2w[0], dx), fmul(c2w[1], dy)), c2w[2]);
    const float wy = fadd(fadd(fmul(c2w[4], dx), fmul(c2w[5], dy)), c2w[6]);
    const float wz = fadd(fadd(fmul(c2w[8], dx), fmul(c2w[9], dy)), c2w[10]);
    const float n = __fsqrt_rn(fadd(fadd(fmul(wx, wx), fmul(wy, wy)), fmul(wz, wz)));
    d = make_float3(fdiv(wx, n), fdiv(wy, n), fdiv(wz, n));
    o = make_float3(c2w[3], c2w[7], c2w[11]);
}

__device__ __forceinline__ void store_ray(float* rays, uint32_t cap, uint32_t r, float3 o,
                                          float3 d, float4 t0, float V, uint32_t kf) {
    rays[kOx * cap + r] = o.x;
    rays[kOy * cap + r] = o.y;
    rays[kOz * cap + r] = o.z;
    rays[kDx * cap + r] = d.x;
    rays[kDy * cap + r] = d.y;
    rays[kDz * cap + r] = d.z;
    rays[kIr * cap + r] = t0.x;
    rays[kIg * cap + r] = t0.y;
    rays[kIb * cap + r] = t0.z;
    rays[kD * cap + r] = t0.w;
    rays[kV * cap + r] = V;
    rays[kKf * cap + r] = __uint_as_float(kf);
}

}  // namespace nm
