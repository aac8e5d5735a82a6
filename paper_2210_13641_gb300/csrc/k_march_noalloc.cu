// k_march_noalloc.cu - march and sample compaction for callers that cannot
// allocate device memory.
//
// Who needs it: a caller whose device memory is owned by someone else (a
// framework's caching allocator that has reserved the GPU's memory, or a fixed
// per-process budget), and a latency-critical host loop such as a tracking
// thread, for which a cudaMalloc may synchronise the device and stall.  map_step
// and map_render keep their work buffers inside a map handle, which allocates;
// map_march_noalloc takes every input and output from the caller and keeps its
// only scratch (per-ray sample counts and the scan's tile totals) in the
// statically sized device array below.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (kMarchScratchWords * 4 bytes, about 4 MB) until the process
// exits.  Host code cannot use the array's name as a device address; its address
// is looked up once per device with cudaGetSymbolAddress.  All calls share the
// array, so calls whose work overlaps on the GPU (different streams, or different
// host threads on one device) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/nerfmap.h"
#include "internal.h"

namespace nm {

constexpr uint32_t kMarchNoAllocMaxRays = 1u << 20;
constexpr uint32_t kMarchNoAllocTiles = (kMarchNoAllocMaxRays + 4095) / 4096;  // scan tiles of 4096
constexpr uint32_t kMarchScratchWords = kMarchNoAllocMaxRays + kMarchNoAllocTiles;

// counts[0 .. 2^20) then the scan's tile totals.  Every word a call reads is first
// written by the same call (counts by the count pass, tile totals by the scan), so
// nothing needs clearing between calls.
static __device__ __align__(256) uint32_t g_march_scratch[kMarchScratchWords];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
uint32_t* g_scratch_addr[kMaxDevices] = {};
thread_local char g_noalloc_error[160] = {0};

void set_error(const char* msg) {
    size_t i = 0;
    for (; msg[i] && i + 1 < sizeof(g_noalloc_error); ++i) g_noalloc_error[i] = msg[i];
    g_noalloc_error[i] = 0;
}

// Device address of the scratch array on the current device (looked up once per
// device, with that device current).
cudaError_t scratch_address(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_march_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// Same march as the mapping step (step i of a ray at t_i = near + i * step, kept
// inside the box and in occupied cells, first max_samples kept), reading the rays
// as [n][3] arrays.  Pass 1 counts, pass 2 writes (ray, t) at the scanned offsets.
template <bool kEmit>
__global__ void k_march_rows(DevCfg c, const uint32_t* __restrict__ bits, uint32_t n_rays,
                             const float* __restrict__ ro, const float* __restrict__ rd,
                             uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                             uint32_t* __restrict__ ray_id, float* __restrict__ ts) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float3 o = make_float3(ro[3 * r], ro[3 * r + 1], ro[3 * r + 2]);
    const float3 d = make_float3(rd[3 * r], rd[3 * r + 1], rd[3 * r + 2]);
    uint32_t n = 0;
    const uint32_t base = kEmit ? offsets[r] : 0;
    for (uint32_t i = 0; i < c.n_steps && n < c.max_samples; ++i) {
        const float t = sample_t(c, i);
        const float3 x = grid_pos(c, o, d, t);
        if (!in_box(c, x) || !occupied(c, bits, x)) continue;
        if (kEmit) {
            ray_id[base + n] = r;
            ts[base + n] = t;
        }
        ++n;
    }
    if (!kEmit) counts[r] = n;
}

}  // namespace nm

using namespace nm;

extern "C" int map_march_noalloc(const map_config* cfg, const uint8_t* occ_bits, const float* rays_o,
                                 const float* rays_d, uint32_t n_rays, uint32_t* offsets, uint32_t* ray_id,
                                 float* t, size_t cap_samples, void* stream) {
    if (!cfg || !rays_o || !rays_d || !offsets || !ray_id || !t) {
        set_error("map_march_noalloc: null pointer argument");
        return MAP_EINVAL;
    }
    if (n_rays == 0 || n_rays > kMarchNoAllocMaxRays) {
        set_error("map_march_noalloc: n_rays must be 1 .. 1048576 (the size of the static scratch)");
        return MAP_EINVAL;
    }
    if (!(cfg->step_t > 0.f) || cfg->n_steps == 0 || cfg->max_samples == 0 || cfg->max_samples > 1024 ||
        !(cfg->grid_inv_size > 0.f) || cfg->occ_res % 8 != 0 || cfg->occ_res > 1024) {
        set_error("map_march_noalloc: invalid march fields in the configuration");
        return MAP_EINVAL;
    }
    if (cfg->occ_res && !occ_bits) {
        set_error("map_march_noalloc: occ_res > 0 needs the occupancy bitfield");
        return MAP_EINVAL;
    }
    if (cap_samples < (size_t)n_rays * cfg->max_samples) {
        set_error("map_march_noalloc: cap_samples must be at least n_rays * max_samples");
        return MAP_EINVAL;
    }
    uint32_t* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_error("map_march_noalloc: cudaGetSymbolAddress of the static scratch failed");
        return MAP_ECUDA;
    }
    DevCfg c{};
    c.near_t = cfg->near_t;
    c.step_t = cfg->step_t;
    c.n_steps = cfg->n_steps;
    c.max_samples = cfg->max_samples;
    for (int a = 0; a < 3; ++a) {
        c.org[a] = cfg->grid_origin[a];
        c.box[a] = cfg->box_max[a];
    }
    c.inv_size = cfg->grid_inv_size;
    c.occ_res = cfg->occ_res;
    const uint32_t* bits = cfg->occ_res ? reinterpret_cast<const uint32_t*>(occ_bits) : nullptr;
    uint32_t* counts = scratch;
    uint32_t* tile_sums = scratch + kMarchNoAllocMaxRays;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t grid = (n_rays + 127) / 128;
    k_march_rows<false><<<grid, 128, 0, s>>>(c, bits, n_rays, rays_o, rays_d, counts, nullptr, nullptr, nullptr);
    launch_scan_counts(counts, n_rays, offsets, tile_sums, s);
    k_march_rows<true><<<grid, 128, 0, s>>>(c, bits, n_rays, rays_o, rays_d, nullptr, offsets, ray_id, t);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("map_march_noalloc: kernel launch failed");
        return MAP_ECUDA;
    }
    g_noalloc_error[0] = 0;
    return MAP_OK;
}

// Message of this thread's last failed map_march_noalloc call ("" if its last
// call succeeded); used by map_last_error(NULL).
const char* nm_noalloc_last_error() { return g_noalloc_error; }
