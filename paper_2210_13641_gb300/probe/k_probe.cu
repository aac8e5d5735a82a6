// k_probe.cu - measurement kernels of the benchmark (no counterpart in the paper and
// not part of the mapping library's ABI): the ceilings the hash-grid traffic of the
// field kernels is reported against.  Built into its own library,
// libnerfmap_probe.so, which only the benchmark loads.
//
//  nmprobe_random_access  uniformly random 8-byte reads, or 8-byte FP32 vector
//                         reductions, into a table of a given size (L2-resident when
//                         smaller than L2, HBM-resident when larger);
//  nmprobe_l2_stream      coalesced 16-byte reads (cached in L2 only) or 16-byte FP32
//                         vector reductions sweeping a buffer again and again: the
//                         streaming bandwidth of the L2 for a working set of that
//                         size, the roofline denominator of L2-resident tables.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kOk = 0, kInval = -1, kCuda = -5;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output function (Steele, Lea & Flood 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_probe_random(float2* __restrict__ table, uint64_t n_entries, uint32_t per_thread, int mode,
                               uint64_t seed, float2* __restrict__ sink) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t mask = n_entries - 1;  // n_entries is a power of two
    float ax = 0.f, ay = 0.f;
    uint64_t r = mix64(seed ^ (tid << 1));
#pragma unroll 8
    for (uint32_t i = 0; i < per_thread; ++i) {
        r = r * 6364136223846793005ull + 1442695040888963407ull;  // LCG step (Knuth MMIX constants)
        const uint64_t slot = (r >> 20) & mask;
        if (mode == 0) {
            const float2 v = __ldg(table + slot);
            ax += v.x;
            ay += v.y;
        } else {
            atomicAdd(table + slot, make_float2(1e-30f, 1e-30f));
        }
    }
    if (mode == 0 && ax == 12345.f) sink[0] = make_float2(ax, ay);  // keeps the loads alive
}

// Every thread walks the buffer with a grid-wide stride, `reps` times: mode 0 reads
// with ld.global.cg (L2 only, so no L1 hit inflates the figure), mode 1 adds with
// 16-byte FP32 vector reductions.
__global__ void k_probe_stream(float4* __restrict__ buf, uint64_t n_vec, uint32_t reps, int mode,
                               float4* __restrict__ sink) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t rep = 0; rep < reps; ++rep) {
        if (mode == 0) {
#pragma unroll 4
            for (uint64_t i = first; i < n_vec; i += stride) {
                const float4 v = __ldcg(buf + i);
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
        } else {
#pragma unroll 4
            for (uint64_t i = first; i < n_vec; i += stride) atomicAdd(buf + i, make_float4(1e-30f, 1e-30f, 1e-30f, 1e-30f));
        }
    }
    if (mode == 0 && acc.x == 12345.f) sink[0] = acc;  // keeps the loads alive
}

}  // namespace

extern "C" int nmprobe_random_access(float* table, uint64_t n_entries, uint32_t n_threads, uint32_t per_thread,
                                     int mode, uint64_t seed, float* sink, void* stream) {
    if (!table || !sink || n_entries < 2 || (n_entries & (n_entries - 1)) || n_threads == 0 || mode < 0 || mode > 1)
        return kInval;
    const uint32_t blocks = (n_threads + 255) / 256;
    k_probe_random<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<float2*>(table), n_entries, per_thread,
                                                             mode, seed, reinterpret_cast<float2*>(sink));
    return cudaGetLastError() == cudaSuccess ? kOk : kCuda;
}

// buf: device, n_vec float4 (16-byte aligned); blocks of 512 threads.
extern "C" int nmprobe_l2_stream(float* buf, uint64_t n_vec, uint32_t n_blocks, uint32_t reps, int mode, float* sink,
                                 void* stream) {
    if (!buf || !sink || n_vec == 0 || n_blocks == 0 || reps == 0 || mode < 0 || mode > 1 ||
        ((uintptr_t)buf & 15u) || ((uintptr_t)sink & 15u))
        return kInval;
    k_probe_stream<<<n_blocks, 512, 0, (cudaStream_t)stream>>>(reinterpret_cast<float4*>(buf), n_vec, reps, mode,
                                                               reinterpret_cast<float4*>(sink));
    return cudaGetLastError() == cudaSuccess ? kOk : kCuda;
}
