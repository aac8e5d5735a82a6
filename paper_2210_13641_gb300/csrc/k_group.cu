// k_group.cu - grouped render: novel-view queries of several scenes and several
// resolutions, evaluated together in shared launches (the serving pattern; Sec. 3.3's
// mapping thread renders views while it maps, here for several resident scenes at
// once).  A batch of at most cap_rays rays is cut from the views in order; each piece
// (GroupItem) is a run of one view's pixels.  The launches are those of one render -
// ray casting, march with the scene's box and occupancy, count scan and compaction,
// the tensor-core field forward, compositing and the output write - with each ray
// taking its scene's configuration, parameters and bitfield from its piece.  The
// field forward runs over 128-sample tiles that never mix two pieces, so every sample
// goes through exactly the arithmetic of a render of its view alone; like map_render,
// the field is evaluated in two passes when a threshold is set (the first
// kRenderFirst samples of every ray, then the rays still above it), and the grouped
// result equals the single-view render bit for bit.
#include <algorithm>

#include "../../include/nerfmap.h"
#include "internal.h"
#include "rays.cuh"

namespace nm {

static_assert(sizeof(GroupItems) <= 4000, "the piece table must fit the kernel-argument space");

namespace {

// The piece table travels as a kernel argument (no host buffer outlives the call)
// and is written to device memory in stream order.
__global__ void k_set_group_items(GroupItems its, uint32_t n, GroupItem* __restrict__ dst) {
    const uint32_t j = threadIdx.x;
    if (j < n) dst[j] = its.it[j];
}

// The piece of ray r: the last piece whose first ray is <= r (at most kGroupMaxItems).
__device__ __forceinline__ uint32_t piece_of(const GroupItem* __restrict__ items, uint32_t n_items, uint32_t r) {
    uint32_t j = 0;
    while (j + 1 < n_items && items[j + 1].ray0 <= r) ++j;
    return j;
}

__global__ void k_group_raygen(const GroupItem* __restrict__ items, uint32_t n_items, uint32_t n_rays,
                               float* __restrict__ rays, uint32_t cap) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const uint32_t j = piece_of(items, n_items, r);
    const GroupItem& it = items[j];
    const uint32_t pix = it.pix0 + (r - it.ray0);
    float3 o, d;
    cast_ray(it.c2w, it.K, pix % it.W, pix / it.W, o, d);
    store_ray(rays, cap, r, o, d, make_float4(0.f, 0.f, 0.f, 0.f), 1.f, j);
}

// The march of k_march (one warp per ray, 32 consecutive steps per ballot, the
// conservative box step range first), with each ray's configuration and bitfield
// taken from its piece; slot rows of row_stride floats.
__global__ void k_group_march(const GroupItem* __restrict__ items, uint32_t n_rays, const float* __restrict__ rays,
                              uint32_t cap, uint32_t* __restrict__ counts, float* __restrict__ slots,
                              uint32_t row_stride) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n_rays) return;  // whole warps
    const GroupItem& it = items[__float_as_uint(rays[kKf * cap + r])];
    const DevCfg& c = it.c;
    const uint32_t* bits = it.occ;
    const float3 o = make_float3(rays[kOx * cap + r], rays[kOy * cap + r], rays[kOz * cap + r]);
    const float3 d = make_float3(rays[kDx * cap + r], rays[kDy * cap + r], rays[kDz * cap + r]);
    float* row = slots + (size_t)r * row_stride;
    const uint32_t max_samples = c.max_samples;
    uint32_t i_lo, i_hi;
    box_step_range(c, o, d, i_lo, i_hi);
    uint32_t n = 0;
    for (uint32_t i0 = i_lo; i0 < i_hi && n < max_samples; i0 += 32) {
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
        if (keep && pos < max_samples) row[pos] = t;
        n += __popc(m);
    }
    if (lane == 0) counts[r] = n < max_samples ? n : max_samples;
}

// After a scan over the rays (the march's, or a render pass's selection): each
// piece's run of samples (contiguous: the batch is ray-major) and its tiles; the
// batch's tile count.
__global__ void k_group_tiles(GroupItem* __restrict__ items, uint32_t n_items, const uint32_t* __restrict__ offsets,
                              uint32_t* __restrict__ n_tiles) {
    if (threadIdx.x != 0) return;
    uint32_t tiles = 0;
    for (uint32_t j = 0; j < n_items; ++j) {
        GroupItem& it = items[j];
        it.s0 = offsets[it.ray0];
        it.n_s = offsets[it.ray0 + it.n_rays] - it.s0;
        it.tile0 = tiles;
        it.n_tiles = (it.n_s + 127) / 128;
        tiles += it.n_tiles;
    }
    *n_tiles = tiles;
}

}  // namespace

int group_bufs_alloc(GroupBufs& g, uint32_t cap_rays, uint32_t row_stride) {
    StepBufs b{};
    const uint64_t cs = (uint64_t)cap_rays * row_stride;
    const uint32_t n_tiles = (cap_rays + kScanTile - 1) / kScanTile;
    struct Req {
        void** p;
        size_t bytes;
    };
    Req reqs[] = {
        {(void**)&b.rays, sizeof(float) * kRayPlanes * cap_rays},
        {(void**)&b.counts, sizeof(uint32_t) * cap_rays},
        {(void**)&b.offsets, sizeof(uint32_t) * (cap_rays + 1)},
        {(void**)&b.block_sums, sizeof(uint32_t) * (n_tiles + 1)},
        {(void**)&b.ray_id, sizeof(uint32_t) * cs},
        {(void**)&b.t, sizeof(float) * cs},
        {(void**)&b.sig_rgb, sizeof(float4) * cs},
        {(void**)&b.ray_out, sizeof(float) * 5 * cap_rays},
        {(void**)&b.err, 64},
        {(void**)&g.items, sizeof(GroupItem) * kGroupMaxItems},
        {(void**)&g.n_tiles, 64},
        {(void**)&g.sel, sizeof(uint32_t) * cs},
        {(void**)&g.sel_off, sizeof(uint32_t) * (cap_rays + 1)},
        {(void**)&b.loss, 64},
    };
    for (auto& r : reqs) {
        if (cudaMalloc(r.p, r.bytes) != cudaSuccess) {
            cudaGetLastError();
            g.b = b;
            group_bufs_free(g);
            return MAP_ENOMEM;
        }
    }
    cudaMemset(b.err, 0, 64);
    cudaMemset(b.loss, 0, 64);
    b.cap_rays = cap_rays;
    b.cap_samples = cs;
    g.b = b;
    g.row_stride = row_stride;
    return MAP_OK;
}

void group_bufs_free(GroupBufs& g) {
    void* ps[] = {g.b.rays, g.b.counts, g.b.offsets, g.b.block_sums, g.b.ray_id, g.b.t, g.b.sig_rgb,
                  g.b.ray_out, g.b.err, g.items, g.n_tiles, g.sel, g.sel_off, g.b.loss};
    for (void* p : ps)
        if (p) cudaFree(p);
    g = GroupBufs{};
}

int render_group(const GroupView* views, uint32_t n, bool bf16, GroupBufs& g, int n_sm, cudaStream_t s,
                 uint64_t* launches) {
    const StepBufs& b = g.b;
    for (uint32_t v = 0; v < n; ++v)
        if (views[v].scene.dc.max_samples > g.row_stride || views[v].scene.precision == MAP_PREC_FP32 ||
            (views[v].scene.precision == MAP_PREC_BF16) != bf16)
            return MAP_EINVAL;
    bool two_pass = false;  // early termination saves field work when a view has a threshold
    for (uint32_t k = 0; k < n; ++k) two_pass |= views[k].scene.dc.t_min > 0.f;
    uint32_t v = 0, p = 0;  // next view and its next pixel
    while (v < n) {
        GroupItems its{};
        uint32_t n_items = 0, rays = 0;
        while (v < n && n_items < (uint32_t)kGroupMaxItems && rays < b.cap_rays) {
            const GroupView& gv = views[v];
            const uint32_t pixels = gv.W * gv.H;
            const uint32_t take = std::min(pixels - p, b.cap_rays - rays);
            GroupItem& it = its.it[n_items++];
            it.c = gv.scene.dc;
            it.params = gv.scene.params;
            it.occ = gv.scene.dc.occ_res ? gv.scene.occ : nullptr;
            for (int k = 0; k < 12; ++k) it.c2w[k] = gv.c2w[k];
            for (int k = 0; k < 4; ++k) it.K[k] = gv.K[k];
            it.W = gv.W;
            it.pix0 = p;
            it.ray0 = rays;
            it.n_rays = take;
            it.out_rgb = gv.out_rgb;
            it.out_depth = gv.out_depth;
            rays += take;
            p += take;
            if (p == pixels) {
                ++v;
                p = 0;
            }
        }
        k_set_group_items<<<1, kGroupMaxItems, 0, s>>>(its, n_items, g.items);
        k_group_raygen<<<(rays + 255) / 256, 256, 0, s>>>(g.items, n_items, rays, b.rays, b.cap_rays);
        float* slots = reinterpret_cast<float*>(b.sig_rgb);
        k_group_march<<<(rays + 7) / 8, 256, 0, s>>>(g.items, rays, b.rays, b.cap_rays, b.counts, slots,
                                                     g.row_stride);
        launch_scan_counts(b.counts, rays, b.offsets, b.block_sums, s);
        launch_compact(rays, g.row_stride, b.offsets, slots, b.ray_id, b.t, s);
        if (!two_pass) {
            k_group_tiles<<<1, 32, 0, s>>>(g.items, n_items, b.offsets, g.n_tiles);
            launch_group_fwd_tc(g.items, n_items, g.n_tiles, b, bf16, n_sm, s);
            launch_composite_group(g.items, rays, b, s);
            if (launches) *launches += 11;  // items, rays, march, 3 scan passes, compaction, tiles, field, composite, write
        } else {
            // as map_render: the field for the first kRenderFirst samples of every ray,
            // then for the rays still above their threshold (pieces index the selection)
            for (int pass = 1; pass <= 2; ++pass) {
                launch_render_select(rays, b.offsets, b.counts, pass == 1, kRenderFirst, g.sel_off, b.block_sums,
                                     g.sel, render_eval_counter(b), s);
                k_group_tiles<<<1, 32, 0, s>>>(g.items, n_items, g.sel_off, g.n_tiles);
                launch_group_fwd_tc(g.items, n_items, g.n_tiles, b, bf16, n_sm, s, g.sel);
                launch_composite_group(g.items, rays, b, s, pass, b.counts);
            }
            if (launches) *launches += 23;
        }
        launch_write_group(g.items, rays, b, s);
        if (cudaGetLastError() != cudaSuccess) return MAP_ECUDA;
    }
    return MAP_OK;
}

}  // namespace nm
