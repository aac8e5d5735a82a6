// internal.h - host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

struct map_scene;  // the state behind a map_handle (api.cu)

namespace nm {

// Message slot of the calls that take no map handle (map_create,
// map_march_noalloc, map_marginal_covariances), read by map_last_error(NULL): one
// slot per host thread, cleared when such a call starts and set when it fails.
void clear_global_error();
void set_global_error(const char* msg);

// One keyframe in the device store.  texels: 8 floats per pixel
// {r, g, b, D, Sigma_D, 0, 0, 0} (one 32-byte sector), D and Sigma_D in ray units.
struct KfDesc {
    float c2w[12];
    float K[4];
    uint32_t W, H;
    const float4* texels;
};

// Ray batch, structure of arrays: 12 planes of `cap` floats (kKf holds the ray's
// keyframe slot as the bits of a uint32).
enum RayPlane { kOx = 0, kOy, kOz, kDx, kDy, kDz, kIr, kIg, kIb, kD, kV, kKf, kRayPlanes };

constexpr uint32_t kCompositeMaxBlocks = 4096;

// Exclusive scan of per-ray counts (k_rays.cu): one 1024-thread block scans a tile of
// kScanTile counts and writes the tile's total; a second pass scans the totals.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

struct StepBufs {
    float* rays;            // [kRayPlanes][cap_rays]
    uint32_t cap_rays;
    uint32_t* counts;       // [cap_rays]
    uint32_t* offsets;      // [cap_rays + 1] exclusive scan, offsets[n] = total
    uint32_t* block_sums;   // scan scratch
    uint32_t* ray_id;       // [cap_samples]
    float* t;               // [cap_samples]
    float4* sig_rgb;        // [cap_samples] sigma, r, g, b
    float4* dsig_rgb;       // [cap_samples] dL/dsigma, dL/dr, dL/dg, dL/db (w_i while compositing)
    float* feat;            // [cap_samples][32] stored encodings (FP32)
    float* ray_out;         // [5][cap_rays] I*r, I*g, I*b, D*, acc
    float* loss;            // [0] batch loss, [1] [2] largest seeds (FP32 bits), [3] block counter,
                            // bytes 32..39: retained samples of the current render (all chunks)
    float* partials;        // [kCompositeMaxBlocks][4] per-block sums of the compositing kernel
    float4* pose_s;         // [cap_samples][2] per-sample pose terms (dL/dp, dL/dd via SH); lazily
    uint32_t* err;          // [1]
    uint64_t cap_samples;
};

inline unsigned long long* render_sample_counter(const StepBufs& b) {
    return reinterpret_cast<unsigned long long*>(b.loss + 8);
}
// bytes 40..47 of the loss buffer: samples a render's field forward evaluated (all chunks)
inline unsigned long long* render_eval_counter(const StepBufs& b) {
    return reinterpret_cast<unsigned long long*>(b.loss + 10);
}

// ---------------------------------------------------------------- two-pass render
// A render evaluates the field for the first kSplitFirst samples of every ray, then
// only for the rays whose transmittance is still above the threshold (k_composite.cu).
constexpr uint32_t kRenderFirst = 32;
// k_rays.cu: the selection of a pass's samples.  first_pass: count[r] = min(first,
// samples of ray r), samples 0 .. count[r] - 1 of each ray; otherwise count[r] is given
// (the composite's live counts) and the samples first .. first + count[r] - 1 are taken.
// sel_off: [n_rays + 1] (sel_off[n_rays] = the pass's total), tile_sums: scan scratch,
// sel: the selected sample indices; evaluated accumulates the totals.
void launch_render_select(uint32_t n_rays, const uint32_t* offsets, uint32_t* count, bool first_pass,
                          uint32_t first, uint32_t* sel_off, uint32_t* tile_sums, uint32_t* sel,
                          unsigned long long* evaluated, cudaStream_t s);
// k_composite.cu: pass 1 (first kRenderFirst samples, live counts out) or pass 2 (the
// live rays, from their first sample).
void launch_composite_split(const DevCfg& c, uint32_t n_rays, int pass, uint32_t* live, const StepBufs& b,
                            cudaStream_t s);

// ---------------------------------------------------------------- grouped render
// One piece of a grouped render (several views of several scenes in shared
// launches): pixels pix0 .. pix0 + n_rays - 1 of a W-wide view of one scene, which are
// rays ray0 .. ray0 + n_rays - 1 of the batch.  s0, n_s, tile0, n_tiles are written on
// the device after the march's scan: the piece's samples s0 .. s0 + n_s - 1 and its
// 128-sample tiles tile0 .. tile0 + n_tiles - 1 of the batch.
struct GroupItem {
    DevCfg c;                 // the scene's configuration (t_min: its render threshold)
    const float* params;      // the scene's parameters (tables, then MLP weights)
    const uint32_t* occ;      // its occupancy bitfield (nullptr: none)
    float c2w[12];
    float K[4];
    uint32_t W;
    uint32_t pix0, ray0, n_rays;
    float* out_rgb;           // the view's device outputs: [pixels][3] colour, [pixels] depth
    float* out_depth;
    uint32_t s0, n_s, tile0, n_tiles;
};
constexpr int kGroupMaxItems = 8;
struct GroupItems {
    GroupItem it[kGroupMaxItems];
};

// Work buffers of grouped renders: a ray batch of cap_rays rays with row_stride slots
// per ray (the largest max_samples of the scenes it serves), the piece table and the
// batch's tile count.
struct GroupBufs {
    StepBufs b{};
    uint32_t row_stride = 0;
    GroupItem* items = nullptr;     // [kGroupMaxItems], device
    uint32_t* n_tiles = nullptr;    // [1], device
    uint32_t* sel = nullptr;        // [cap_samples] a render pass's selected samples
    uint32_t* sel_off = nullptr;    // [cap_rays + 1] its scan
};

// A scene's state as a grouped render needs it (api.cu).
struct SceneView {
    DevCfg dc;                      // t_min set to the scene's render threshold
    const float* params;
    const uint32_t* occ;
    uint32_t precision;             // MAP_PREC_*
};
bool scene_view(const ::map_scene* h, SceneView* out);

// One view of a grouped render: the scene, the camera and the device outputs.
struct GroupView {
    SceneView scene;
    float c2w[12];
    float K[4];
    uint32_t W, H;
    float* out_rgb;                 // device, [H*W][3]
    float* out_depth;               // device, [H*W]
};

// k_group.cu: allocation of the work buffers, and the grouped render of `n` views whose
// scenes all use the FP16 (bf16 = false) or all the BF16 tensor-core MLP, in chunks of
// at most cap_rays rays / kGroupMaxItems pieces; every launch is queued on s.
int group_bufs_alloc(GroupBufs& g, uint32_t cap_rays, uint32_t row_stride);
void group_bufs_free(GroupBufs& g);
// launches (nullable) is increased by the number of kernels launched.
int render_group(const GroupView* views, uint32_t n, bool bf16, GroupBufs& g, int n_sm, cudaStream_t s,
                 uint64_t* launches);

// k_field_tc.cu: the grouped forward (persistent; switches weights where the scene
// changes between tiles).
// sel (nullable): the pieces' sample runs index this selection (a render pass).
void launch_group_fwd_tc(const GroupItem* items, uint32_t n_items, const uint32_t* n_tiles, const StepBufs& b,
                         bool bf16, int n_sm, cudaStream_t s, const uint32_t* sel = nullptr);
// k_composite.cu: the grouped render's compositing (each ray's spacing and
// termination threshold from its piece; pass 0: single pass, 1 / 2: the two render
// passes with the live counts) and output write.
void launch_composite_group(const GroupItem* items, uint32_t n_rays, const StepBufs& b, cudaStream_t s,
                            int pass = 0, uint32_t* live = nullptr);
void launch_write_group(const GroupItem* items, uint32_t n_rays, const StepBufs& b, cudaStream_t s);

// k_rays.cu
void launch_set_kf_desc(KfDesc* table, uint32_t idx, const KfDesc& d, cudaStream_t s);
void launch_keyframe_texels(const float* rgb, const float* depth, const float* var, uint32_t W,
                            uint32_t H, const float* K, int depth_is_z, float4* texels,
                            cudaStream_t s);
void launch_ray_gen(const KfDesc* kfs, const uint32_t* active, uint32_t n_kf, uint64_t seed, uint64_t step,
                    uint32_t n_rays, const StepBufs& b, cudaStream_t s);
void launch_ray_gen_view(const float* c2w, const float* K, uint32_t W, uint32_t p0, uint32_t cnt,
                         const StepBufs& b, cudaStream_t s);
void launch_march(const DevCfg& c, const uint32_t* occ_bits, uint32_t n_rays, const StepBufs& b,
                  cudaStream_t s);

// tile_sums: at least ceil(n / kScanTile) words.
// k_compact: each ray's retained steps from its slot row (row_stride floats per ray)
// to its scanned offset, with the ray index beside each sample.
void launch_compact(uint32_t n_rays, uint32_t row_stride, const uint32_t* offsets, const float* slots,
                    uint32_t* ray_id, float* ts, cudaStream_t s);

void launch_scan_counts(const uint32_t* counts, uint32_t n, uint32_t* offsets, uint32_t* tile_sums,
                        cudaStream_t s);

// k_field_fp32.cu
void launch_field_fwd_fp32(const DevCfg& c, const float* params, uint32_t n_rays,
                           const StepBufs& b, bool store_feat, int n_sm, cudaStream_t s);
// pose: also write the per-sample pose terms into b.pose_s (joint pose refinement).
void launch_field_bwd_fp32(const DevCfg& c, const float* params, float* grads, uint32_t n_rays,
                           const StepBufs& b, int n_sm, cudaStream_t s, bool pose = false);

// The forward over a selection of the batch's samples, sel[0 .. *n_sel) (a render's
// passes; the encodings are not stored).
void launch_field_fwd_fp32_sel(const DevCfg& c, const float* params, const uint32_t* sel, const uint32_t* n_sel,
                               const StepBufs& b, int n_sm, cudaStream_t s);

// k_field_tc.cu (FP16 / BF16 tensor-core MLP)
void launch_field_fwd_tc_sel(const DevCfg& c, const float* params, const uint32_t* sel, const uint32_t* n_sel,
                             const StepBufs& b, bool bf16, int n_sm, cudaStream_t s);
void launch_field_fwd_tc(const DevCfg& c, const float* params, uint32_t n_rays, const StepBufs& b,
                         bool store_feat, bool bf16, int n_sm, cudaStream_t s);
void launch_field_bwd_tc(const DevCfg& c, const float* params, float* grads, uint32_t n_rays,
                         const StepBufs& b, bool bf16, int n_sm, cudaStream_t s, bool pose = false);

// k_pose.cu: per-ray sums of the per-sample pose terms, accumulated per keyframe slot
// into pose_g[slot][8] = (dL/drho, dL/dphi, 0, 0); pose_g must be zeroed first.
void launch_pose_reduce(const DevCfg& c, uint32_t n_rays, const StepBufs& b, float* pose_g, cudaStream_t s);

// k_composite.cu
void launch_composite(const DevCfg& c, uint32_t n_rays, bool backward, const StepBufs& b,
                      cudaStream_t s);
// single_pass: the render evaluated every retained sample (counted as evaluated here).
void launch_write_render(const StepBufs& b, uint32_t n, float* rgb, float* depth, float* acc, bool single_pass,
                         cudaStream_t s);

// k_adam_occ.cu
void launch_adam(float* p, float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                 float eps, float c1, float c2, cudaStream_t s);
void launch_init_params(float* p, size_t n_table, uint64_t seed, cudaStream_t s);
void launch_occ_refresh(const DevCfg& c, const float* params, float* density, uint32_t* bits,
                        uint64_t seed, uint64_t refresh_idx, float decay, float thresh,
                        cudaStream_t s);
void launch_occ_from_bits(const uint32_t* bits, float* density, uint32_t n_cells, cudaStream_t s);

}  // namespace nm
