// k_probe.cu - random-access throughput probe: the ceiling the hash-grid gathers
// and gradient scatter are measured against.  Uniformly random 8-byte reads, or
// 8-byte FP32 vector reductions, into a table of a given size (resident in L2 when
// it is smaller than L2, streamed from HBM when it is larger).
#include "../../include/nerfmap.h"
#include "internal.h"

namespace nm {

__global__ void k_probe_random(float2* __restrict__ table, uint64_t n_entries, uint32_t per_thread, int mode,
                               uint64_t seed, float2* __restrict__ sink) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t mask = n_entries - 1;  // n_entries is a power of two
    float ax = 0.f, ay = 0.f;
    uint64_t r = counter_rand(seed, 5ull << 30, tid, 0);
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

}  // namespace nm

extern "C" int map_probe_random_access(float* table, uint64_t n_entries, uint32_t n_threads, uint32_t per_thread,
                                       int mode, uint64_t seed, float* sink, void* stream) {
    if (!table || !sink || n_entries < 2 || (n_entries & (n_entries - 1)) || n_threads == 0 || mode < 0 || mode > 1)
        return MAP_EINVAL;
    const uint32_t blocks = (n_threads + 255) / 256;
    nm::k_probe_random<<<blocks, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<float2*>(table), n_entries,
                                                                  per_thread, mode, seed,
                                                                  reinterpret_cast<float2*>(sink));
    return cudaGetLastError() == cudaSuccess ? MAP_OK : MAP_ECUDA;
}
