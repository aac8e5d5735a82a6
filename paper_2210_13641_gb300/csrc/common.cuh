// common.cuh - device-side definitions shared by the mapping kernels.
//
// Integer decisions (ray draw, sample positions, box / occupancy tests, grid cells)
// are taken in IEEE float32 with an explicit operation order: every product and sum
// on that path uses the _rn intrinsics so the compiler cannot contract it into an
// FMA.  Everything else may use ordinary FP32 arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nm {

constexpr int kMaxLevels = 32;
constexpr int kEnc = 32;       // density-MLP input width (L*F zero padded)
constexpr int kHid = 64;       // hidden width of both MLPs
constexpr int kGeo = 16;       // density-MLP output width
constexpr int kSH = 16;        // SH coefficients, bands 0..3
constexpr int kW1 = kHid * kEnc;          // 2048
constexpr int kW2 = kGeo * kHid;          // 1024
constexpr int kW3 = kHid * (kGeo + kSH);  // 2048
constexpr int kW4 = kHid * kHid;          // 4096
constexpr int kW5 = 3 * kHid;             // 192
constexpr int kMlpParams = kW1 + kW2 + kW3 + kW4 + kW5;  // 9408
// Density activation: sigma = exp(min(h_0, kSigmaHMax)), an exponential whose value
// is capped (a reading: the paper defers the activation to its map).  Beyond the cap
// a sample is opaque already (sigma * delta > 10^4 at every spacing used here) and
// sigma stays finite in FP32 through long fits; dsigma/dh_0 = 0 above it.  This is
// not Instant-NGP's "truncated exponential", which leaves the value alone and clamps
// the argument of the derivative instead.
constexpr float kSigmaHMax = 15.f;
constexpr int kOffW1 = 0, kOffW2 = kW1, kOffW3 = kW1 + kW2, kOffW4 = kOffW3 + kW3,
              kOffW5 = kOffW4 + kW4;

// Kernel-side copy of the configuration (passed by value).
struct DevCfg {
    uint32_t L;
    uint32_t log2T;
    uint32_t T;
    uint32_t dense_mask;          // bit l: level l indexed densely
    uint32_t res[kMaxLevels];     // N_l
    float near_t, step_t;
    uint32_t n_steps, max_samples;
    float org[3];
    float inv_size;
    float box[3];
    uint32_t occ_res;
    float lambda_d;
    float t_min;                  // render early-termination threshold (0: none)
    uint32_t wait_polls;          // poll limit of each MMA-completion wait (tensor-core kernels)
};

// Default poll limit of a bounded MMA-completion wait: far beyond any MMA chain's
// latency, far below a watchdog's reach.
constexpr uint32_t kWaitPollsDefault = 1u << 24;

// ----------------------------------------------------------------- exact FP32

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// ----------------------------------------------------------------- SplitMix64
// Published SplitMix64 output function (Steele, Lea & Flood 2014): advance by the
// golden gamma, then xor-shift 30 / multiply, xor-shift 27 / multiply, xor-shift 31.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Counter-based draw: counter = stream << 33 | index << 1 | k, output = mix(seed ^ ctr).
__host__ __device__ __forceinline__ uint64_t counter_rand(uint64_t seed, uint64_t stream,
                                                          uint64_t index, uint64_t k) {
    return splitmix64(seed ^ ((stream << 33) | (index << 1) | k));
}

constexpr uint64_t kOccStream = 1ull << 30;

// ----------------------------------------------------------------- geometry

// Grid position of step i of a ray: t = near + i*step, x = (o + t d - org) * inv.
__device__ __forceinline__ float sample_t(const DevCfg& c, uint32_t i) {
    return fadd(c.near_t, fmul((float)i, c.step_t));
}

__device__ __forceinline__ float3 grid_pos(const DevCfg& c, float3 o, float3 d, float t) {
    float3 x;
    x.x = fmul(fsub(fadd(o.x, fmul(t, d.x)), c.org[0]), c.inv_size);
    x.y = fmul(fsub(fadd(o.y, fmul(t, d.y)), c.org[1]), c.inv_size);
    x.z = fmul(fsub(fadd(o.z, fmul(t, d.z)), c.org[2]), c.inv_size);
    return x;
}

__device__ __forceinline__ bool in_box(const DevCfg& c, float3 x) {
    return x.x >= 0.f && x.y >= 0.f && x.z >= 0.f && x.x < c.box[0] && x.y < c.box[1] &&
           x.z < c.box[2];
}

__device__ __forceinline__ int cell_of(float x, uint32_t res) {
    int ci = (int)floorf(fmul(x, (float)res));
    ci = ci < 0 ? 0 : ci;
    return ci > (int)res - 1 ? (int)res - 1 : ci;
}

__device__ __forceinline__ bool occupied(const DevCfg& c, const uint32_t* __restrict__ bits,
                                         float3 x) {
    if (c.occ_res == 0) return true;
    const uint32_t R = c.occ_res;
    uint32_t b = (uint32_t)cell_of(x.x, R) + R * ((uint32_t)cell_of(x.y, R) + R * (uint32_t)cell_of(x.z, R));
    return (__ldg(bits + (b >> 5)) >> (b & 31)) & 1u;
}

// Step range [i_lo, i_hi) outside which no step of the ray can pass the box test.
// The slab interval [t_in, t_out] of the ray in grid coordinates is computed in
// FP32 and widened by two steps plus a relative 1e-5: the positions of the steps
// are rounded by about 1e-7 of their magnitude, far inside that margin, so every
// step whose FP32 position is in the box lies in the range (the box test itself
// is still taken per step).
__device__ __forceinline__ void box_step_range(const DevCfg& c, float3 o, float3 d, uint32_t& i_lo,
                                               uint32_t& i_hi) {
    const float xo[3] = {(o.x - c.org[0]) * c.inv_size, (o.y - c.org[1]) * c.inv_size,
                         (o.z - c.org[2]) * c.inv_size};
    const float xd[3] = {d.x * c.inv_size, d.y * c.inv_size, d.z * c.inv_size};
    float t_in = -3.0e38f, t_out = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (fabsf(xd[a]) > 1e-20f) {
            const float t0 = (0.f - xo[a]) / xd[a], t1 = (c.box[a] - xo[a]) / xd[a];
            t_in = fmaxf(t_in, fminf(t0, t1));
            t_out = fminf(t_out, fmaxf(t0, t1));
        } else if (!(xo[a] >= -1e-6f && xo[a] <= c.box[a] + 1e-6f)) {
            t_out = -3.0e38f;  // parallel to this slab and outside it
        }
    }
    const float margin_lo = 2.f * c.step_t + 1e-5f * fabsf(t_in);
    const float margin_hi = 2.f * c.step_t + 1e-5f * fabsf(t_out);
    const float lo = (t_in - margin_lo - c.near_t) / c.step_t;
    const float hi = (t_out + margin_hi - c.near_t) / c.step_t;
    if (!(hi >= lo) || hi < 0.f) {  // misses the box even with the margins
        i_lo = i_hi = 0;
        return;
    }
    i_lo = lo <= 0.f ? 0u : (lo >= (float)c.n_steps ? c.n_steps : (uint32_t)lo);
    i_hi = hi >= (float)c.n_steps ? c.n_steps : (uint32_t)hi + 1u;
}

// ----------------------------------------------------------------- hash grid

// Table slot of vertex (cx, cy, cz) at resolution N of a level (dense or hashed).
__device__ __forceinline__ uint32_t vertex_slot(uint32_t cx, uint32_t cy, uint32_t cz,
                                                uint32_t N, bool dense, uint32_t Tmask) {
    if (dense) {
        const uint32_t s = N + 1;
        return cx + s * (cy + s * cz);
    }
    return (cx ^ (cy * 2654435761u) ^ (cz * 805459861u)) & Tmask;
}

// Cell and fractional offset at resolution N: q = x*N, c = min(floor q, N-1), w = q - c.
__device__ __forceinline__ void level_cell(float x, uint32_t N, uint32_t& ci, float& w) {
    const float q = fmul(x, (float)N);
    int c = (int)floorf(q);
    c = c > (int)N - 1 ? (int)N - 1 : c;
    c = c < 0 ? 0 : c;
    ci = (uint32_t)c;
    w = fsub(q, (float)c);
}

// ----------------------------------------------------------------- SH bands 0..3
// Real orthonormal spherical harmonics (Condon-Shortley phase); the constants are
// the Legendre normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2, m != 0).
__device__ __forceinline__ void sh16(float x, float y, float z, float* out) {
    const float kPi = 3.14159265358979323846f;
    const float c0 = 0.5f * sqrtf(1.f / kPi);
    const float c1 = sqrtf(3.f / (4.f * kPi));
    const float c2a = 0.5f * sqrtf(15.f / kPi);
    const float c2b = 0.25f * sqrtf(5.f / kPi);
    const float c2c = 0.25f * sqrtf(15.f / kPi);
    const float c3a = 0.25f * sqrtf(35.f / (2.f * kPi));
    const float c3b = 0.5f * sqrtf(105.f / kPi);
    const float c3c = 0.25f * sqrtf(21.f / (2.f * kPi));
    const float c3d = 0.25f * sqrtf(7.f / kPi);
    const float c3e = 0.25f * sqrtf(105.f / kPi);
    const float xx = x * x, yy = y * y, zz = z * z;
    out[0] = c0;
    out[1] = -c1 * y;
    out[2] = c1 * z;
    out[3] = -c1 * x;
    out[4] = c2a * x * y;
    out[5] = -c2a * y * z;
    out[6] = c2b * (3.f * zz - 1.f);
    out[7] = -c2a * x * z;
    out[8] = c2c * (xx - yy);
    out[9] = -c3a * y * (3.f * xx - yy);
    out[10] = c3b * x * y * z;
    out[11] = -c3c * y * (5.f * zz - 1.f);
    out[12] = c3d * z * (5.f * zz - 3.f);
    out[13] = -c3c * x * (5.f * zz - 1.f);
    out[14] = c3e * z * (xx - yy);
    out[15] = -c3a * x * (xx - 3.f * yy);
}

// J^T g for the Jacobian J [16 x 3] of sh16 with respect to the direction (each
// basis function differentiated as the polynomial in x, y, z that sh16 evaluates).
__device__ __forceinline__ float3 sh16_vjp(float x, float y, float z, const float* g) {
    const float kPi = 3.14159265358979323846f;
    const float c1 = sqrtf(3.f / (4.f * kPi));
    const float c2a = 0.5f * sqrtf(15.f / kPi);
    const float c2b = 0.25f * sqrtf(5.f / kPi);
    const float c2c = 0.25f * sqrtf(15.f / kPi);
    const float c3a = 0.25f * sqrtf(35.f / (2.f * kPi));
    const float c3b = 0.5f * sqrtf(105.f / kPi);
    const float c3c = 0.25f * sqrtf(21.f / (2.f * kPi));
    const float c3d = 0.25f * sqrtf(7.f / kPi);
    const float c3e = 0.25f * sqrtf(105.f / kPi);
    const float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    // band 1: -c1 y, c1 z, -c1 x
    gy -= c1 * g[1];
    gz += c1 * g[2];
    gx -= c1 * g[3];
    // band 2
    gx += c2a * y * g[4];
    gy += c2a * x * g[4];
    gy -= c2a * z * g[5];
    gz -= c2a * y * g[5];
    gz += 6.f * c2b * z * g[6];
    gx -= c2a * z * g[7];
    gz -= c2a * x * g[7];
    gx += 2.f * c2c * x * g[8];
    gy -= 2.f * c2c * y * g[8];
    // band 3
    gx -= 6.f * c3a * x * y * g[9];
    gy -= c3a * (3.f * xx - 3.f * yy) * g[9];
    gx += c3b * y * z * g[10];
    gy += c3b * x * z * g[10];
    gz += c3b * x * y * g[10];
    gy -= c3c * (5.f * zz - 1.f) * g[11];
    gz -= 10.f * c3c * y * z * g[11];
    gz += c3d * (15.f * zz - 3.f) * g[12];
    gx -= c3c * (5.f * zz - 1.f) * g[13];
    gz -= 10.f * c3c * x * z * g[13];
    gx += 2.f * c3e * x * z * g[14];
    gy -= 2.f * c3e * y * z * g[14];
    gz += c3e * (xx - yy) * g[14];
    gx -= c3a * (3.f * xx - 3.f * yy) * g[15];
    gy += 6.f * c3a * x * y * g[15];
    return make_float3(gx, gy, gz);
}

// ----------------------------------------------------------------- error flag
// Kernels record an out-of-range condition (which they then skip) in a device word
// the host reads after the step; nothing on the device traps.
enum : uint32_t { kErrNone = 0, kErrSampleOverflow = 1, kErrBadRay = 2, kErrTimeout = 4 };

}  // namespace nm
