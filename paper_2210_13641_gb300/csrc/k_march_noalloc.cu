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
// one tile total per scan tile of the largest call
constexpr uint32_t kMarchNoAllocTiles = (kMarchNoAllocMaxRays + kScanTile - 1) / kScanTile;
constexpr uint32_t kMarchScratchWords = kMarchNoAllocMaxRays + kMarchNoAllocTiles;
static_assert((uint64_t)kMarchNoAllocTiles * kScanTile >= kMarchNoAllocMaxRays,
              "the tile-total scratch must cover every scan tile of the largest call");

// counts[0 .. 2^20) then the scan's tile totals.  Every word a call reads is first
// written by the same call (counts by the count pass, tile totals by the scan), so
// nothing needs clearing between calls.
static __device__ __align__(256) uint32_t g_march_scratch[kMarchScratchWords];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
uint32_t* g_scratch_addr[kMaxDevices] = {};
void set_error(const char* msg) { set_global_error(msg); }

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

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
// Only the steps of the ray's conservative box step range are tested (the range
// contains every step whose position passes the box test), as in the map's march.
template <bool kEmit>
__global__ void k_march_rows(DevCfg c, const uint32_t* __restrict__ bits, uint32_t n_rays,
                             const float* __restrict__ ro, const float* __restrict__ rd,
                             uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets,
                             uint32_t* __restrict__ ray_id, float* __restrict__ ts) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const float3 o = make_float3(ro[3 * r], ro[3 * r + 1], ro[3 * r + 2]);
    const float3 d = make_float3(rd[3 * r], rd[3 * r + 1], rd[3 * r + 2]);
    uint32_t i_lo, i_hi;
    box_step_range(c, o, d, i_lo, i_hi);
    uint32_t n = 0;
    const uint32_t base = kEmit ? offsets[r] : 0;
    for (uint32_t i = i_lo; i < i_hi && n < c.max_samples; ++i) {
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
    clear_global_error();
    if (!cfg || !rays_o || !rays_d || !offsets || !ray_id || !t) {
        set_error("map_march_noalloc: null pointer argument");
        return MAP_EINVAL;
    }
    // the kernels read the bitfield as 32-bit words and the other arrays as 4-byte
    // values: a misaligned address would fault on the device, so it is refused here
    if (!aligned4(rays_o) || !aligned4(rays_d) || !aligned4(offsets) || !aligned4(ray_id) || !aligned4(t) ||
        (cfg->occ_res && occ_bits && !aligned4(occ_bits))) {
        set_error("map_march_noalloc: every device array (occ_bits included) must be 4-byte aligned");
        return MAP_EINVAL;
    }
    if (n_rays == 0 || n_rays > kMarchNoAllocMaxRays) {
        set_error("map_march_noalloc: n_rays must be 1 .. 1048576 (the size of the static scratch)");
        return MAP_EINVAL;
    }
    if (!(cfg->step_t > 0.f) || cfg->n_steps == 0 || cfg->n_steps > 65536 || cfg->max_samples == 0 ||
        cfg->max_samples > 1024 ||
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
    return MAP_OK;
}
