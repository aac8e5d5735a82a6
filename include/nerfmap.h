/*
 * nerfmap.h - C ABI of the GB300 mapping library (NeRF-SLAM mapping stage,
 * arXiv 2210.13641).
 *
 * The library fits a multiresolution hash-grid radiance field to posed keyframes
 * that carry colour, dense depth and a per-pixel depth variance, by minimising the
 * mapping loss L_M = L_rgb + lambda_D * L_D of the paper's Eq. (mapping_loss)
 * (Sec. 3.2), and renders views of the fitted field (Sec. 3.3, the mapping thread
 * renders for visualisation).  Every step of that path runs in the library's own
 * CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions for every call
 *  - Return value: MAP_OK (0) on success, a negative MAP_E* code otherwise; the
 *    message of the last failure is available from map_last_error().
 *  - Camera model: pinhole K = {fx, fy, cx, cy}; pixel (u, v) casts its ray through
 *    its centre (u + 1/2, v + 1/2); OpenCV axes (x right, y down, z forward);
 *    c2w is the row-major 3x4 camera-to-world matrix [R | t].
 *  - Images are row-major (v outer, u inner).
 *  - mem_kind says where a caller buffer lives: MAP_MEM_HOST (ordinary or pinned
 *    host memory) or MAP_MEM_DEVICE (device memory of the GPU that was current
 *    when the map was created).  The caller owns every buffer it passes; the
 *    library owns all state behind a map_handle.
 *  - stream: a cudaStream_t (NULL = legacy default stream).  All work of a call
 *    is ordered on that stream.  Calls that return a value to host memory
 *    synchronise that stream before returning; the others return as soon as the
 *    work is queued, and input buffers may be reused as soon as the call returns
 *    (inputs are copied or staged before return).
 *  - A map_handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef NERFMAP_H
#define NERFMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAP_OK 0
#define MAP_EINVAL (-1)   /* bad argument: null pointer, size or configuration */
#define MAP_ENOMEM (-2)   /* device memory or the map's HBM budget exhausted */
#define MAP_ENOKF (-3)    /* map_step before any keyframe was added */
#define MAP_ETIMEOUT (-4) /* a bounded device-side wait expired */
#define MAP_ECUDA (-5)    /* a CUDA runtime call failed */

#define MAP_MAX_LEVELS 32

#define MAP_MEM_HOST 0
#define MAP_MEM_DEVICE 1

/* MLP arithmetic.  Hash features, compositing, loss, gradients and Adam are FP32
 * in every mode; the MLP layers run on FP32 CUDA cores (plain form) or on the
 * tensor cores with FP16 / BF16 operands and FP32 accumulation. */
#define MAP_PREC_FP32 0
#define MAP_PREC_FP16 1
#define MAP_PREC_BF16 2

/* map_step flags */
#define MAP_STEP_NO_UPDATE 1u  /* compute loss and gradients, skip Adam, keep gradients */
#define MAP_STEP_POSE_GRAD 2u  /* also the gradient of L_M with respect to every keyframe pose */

/*
 * Field and step configuration (copied by map_create).
 *
 * Grid (Instant-NGP multiresolution hash encoding, the map of the paper's
 * Sec. 3.4): n_levels tables of 2^log2_table entries, n_features = 2 floats per
 * entry, level l at resolution level_res[l] (vertex coordinates 0..N_l).  A level
 * whose (N_l + 1)^3 vertices fit in its table is indexed densely, otherwise by the
 * spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861) mod 2^log2_table.
 * MLP widths are fixed: enc_width 32 (L * F zero padded), density_hidden 64,
 * geo_width 16, color_hidden 64.  Density sigma = exp(min(h_0, 15)) (an exponential
 * with its value capped: beyond h_0 = 15 a sample is opaque already; dsigma/dh_0 = 0
 * above the cap), colour = sigmoid of the colour MLP's output.
 *
 * Sampling (Sec. 3.2, sampling 3D positions along the pixel's ray): step i of a
 * ray is at t_i = near_t + i * step_t, i < n_steps, grid position
 * x = (o + t d - grid_origin) * grid_inv_size; it is kept when 0 <= x_a < box_max[a]
 * on every axis and, if occ_res > 0, its occupancy cell is set; the first
 * max_samples kept steps are the ray's samples, each with delta_i = step_t.
 *
 * Occupancy (occ_res > 0): cell density EMA d <- max(occ_decay * d,
 * sigma(x_cell)), bit = d > occ_thresh, refreshed every occ_every steps
 * (0 = only by map_refresh_occupancy).
 *
 * Loss (Eq. mapping_loss): per ray ||I - I*||^2 + lambda_d (D - D*)^2 / Sigma_D,
 * averaged over the rays of a step.  Adam: lr, beta1, beta2, eps, bias corrected.
 * render_t_min: a render stops a ray once its transmittance falls below it.
 */
typedef struct map_config {
    uint32_t n_levels;
    uint32_t n_features;
    uint32_t log2_table;
    uint32_t level_res[MAP_MAX_LEVELS];
    uint32_t enc_width;
    uint32_t density_hidden;
    uint32_t geo_width;
    uint32_t color_hidden;
    float near_t;
    float step_t;
    uint32_t n_steps;
    uint32_t max_samples;
    float grid_origin[3];
    float grid_inv_size;
    float box_max[3];
    uint32_t occ_res;
    uint32_t occ_every;
    float occ_decay;
    float occ_thresh;
    float lambda_d;
    float lr;
    float beta1;
    float beta2;
    float eps;
    float render_t_min;
    uint32_t precision;
    uint32_t reserved0;
    uint64_t seed;
} map_config;

typedef struct map_scene* map_handle;

/* Per-step counters of the last map_step / map_render (read back on request). */
typedef struct map_stats {
    uint64_t step;          /* completed optimisation steps (Adam t) */
    uint64_t n_samples;     /* retained samples of the last step or render */
    uint32_t n_rays;        /* rays of the last step or render */
    uint32_t n_keyframes;   /* keyframes in the store */
    uint64_t param_count;   /* FP32 parameters (tables then MLP weights) */
    uint64_t device_bytes;  /* device memory held by the map */
    uint64_t kernel_launches; /* kernels this map has launched since creation */
    uint64_t render_samples;  /* retained samples of the last map_render, all its chunks */
    uint64_t render_evaluated; /* of those, the samples whose field the render evaluated */
} map_stats;

/* Phases of a step or render, for map_profile_read. */
#define MAP_PH_RAYGEN 0     /* ray draw and casting (a1) */
#define MAP_PH_MARCH 1      /* march, occupancy test, count scan, emit (a2) */
#define MAP_PH_FIELD_FWD 2  /* encoding, SH and both MLPs forward (a3-a6) */
#define MAP_PH_COMPOSITE 3  /* compositing, loss and its per-sample gradient (a7-a9) */
#define MAP_PH_FIELD_BWD 4  /* MLP backward and hash-table scatter (a10-a11) */
#define MAP_PH_ADAM 5       /* Adam (a12) */
#define MAP_PH_OCC 6        /* occupancy refresh (a13) */
#define MAP_PH_OUTPUT 7     /* render output write */
#define MAP_PHASES 8

/*
 * map_config_init - a configuration holding the library's defaults and the level
 * table of the multiresolution grid (the Instant-NGP encoding that is the map of
 * Sec. 3.4): N_l = floor(n_min * b^l) for l < n_levels, b = growth when growth > 0,
 * else b = exp(ln(n_max / n_min) / (n_levels - 1)), evaluated in FP64 with a 1e-9
 * relative nudge so that products which are whole numbers in exact arithmetic
 * (e.g. 16 * 128) do not floor one below.  Also sets n_features = 2, log2_table,
 * the MLP widths (32, 64, 16, 64), lambda_d = 1, Adam lr = 1e-2, beta = (0.9, 0.99),
 * eps = 1e-15, occupancy decay 0.95 / threshold 0.01 / refresh every 16 steps,
 * render_t_min = 1e-4, max_samples = 128, precision MAP_PREC_FP16, seed 0.  The
 * scene fields (near_t, step_t, n_steps, grid_origin, grid_inv_size, box_max,
 * occ_res) are left zero for the caller to set.  Host only: no device is used.
 * Errors: MAP_EINVAL (message in map_last_error(NULL)) for a null cfg, n_levels
 * outside 1..16, log2_table outside 10..24, n_min < 2, growth <= 0 with
 * n_max <= n_min while n_levels > 1, or a level above 2^20.
 */
int map_config_init(map_config* cfg, uint32_t n_levels, uint32_t log2_table, uint32_t n_min, uint32_t n_max,
                    double growth);

/*
 * map_create - allocate a map on the current device.
 * cfg: configuration (validated: 1 <= n_levels <= 16 (n_levels * n_features <= 32),
 *   n_features == 2, 10 <= log2_table <= 24, level_res[l] >= 2, widths as above,
 *   occ_res a multiple of 8 (or 0) and <= 1024, precision a MAP_PREC_* value).
 * hbm_budget_bytes: upper bound on the device memory this map may hold, counting
 *   parameters, gradients, Adam moments, occupancy, keyframes and step workspace
 *   (0 = no bound).  Any allocation beyond it fails with MAP_ENOMEM.
 * out: receives the handle.  Parameters start seeded from cfg->seed: tables
 *   U(-1e-4, 1e-4), MLP weights N(0, 0.05).
 */
int map_create(const map_config* cfg, size_t hbm_budget_bytes, map_handle* out);

/* map_destroy - synchronise the device and free everything the map holds. */
int map_destroy(map_handle h);

/*
 * map_add_keyframe - hand a keyframe to the mapper (Sec. 3.3: the tracking
 * thread sends poses, images, depth maps and depth covariances of its window).
 * A kf_id already in the store is replaced in place (the window is re-sent with
 * refined poses and depths); a new id is appended.
 * c2w[12], K[4]: host memory.  rgb: H*W*3 floats in [0,1]; depth: H*W floats;
 * depth_var: H*W per-pixel variances Sigma_D (> 0).  depth_is_z != 0: depth and
 * variance are z-depth values and are converted to distance along the unit ray
 * (D * s and Sigma_D * s^2 with s = ||K^-1 [u+1/2, v+1/2, 1]||); 0: already ray
 * distances.  rgb, depth, depth_var live in mem_kind memory.
 */
int map_add_keyframe(map_handle h, uint32_t kf_id, const float c2w[12], const float K[4],
                     uint32_t W, uint32_t H, const float* rgb, const float* depth,
                     const float* depth_var, int depth_is_z, int mem_kind, void* stream);

/*
 * map_step - one mapping step (Sec. 3.2-3.3): draw n_rays rays uniformly over all
 * keyframes (with replacement, SplitMix64 counter generator keyed by seed and the
 * step counter), march, encode, evaluate the MLPs, composite colour and expected
 * depth, evaluate L_M, back-propagate to the tables and MLP weights and apply
 * Adam (unless MAP_STEP_NO_UPDATE).  The ray draw of the k-th call uses step
 * index k = map_stats.step before the call (NO_UPDATE calls do not advance it).
 * out_loss: host pointer or NULL; when set, the call waits for the step and stores
 * L_M there.  n_rays: 1 .. 2^24.
 */
int map_step(map_handle h, uint32_t n_rays, uint64_t seed, uint32_t flags, float* out_loss,
             void* stream);

/* map_loss_device - device address of the FP32 loss of the last step (valid until
 * the next step on the handle); lets a caller read it without a host wait. */
const float* map_loss_device(map_handle h);

/*
 * map_render - forward-only render of a W x H view (Sec. 3.3).  out_rgb: H*W*3
 * floats, out_depth: H*W floats (expected ray-termination distance along the unit
 * ray), both in mem_kind memory; either may be NULL.  out_acc (nullable, same
 * memory kind): H*W accumulated opacities.  Rays stop once transmittance drops
 * below cfg.render_t_min; with render_t_min > 0 the field is evaluated for the
 * first 32 samples of every ray and then only for the rays that have not stopped
 * (the image equals that of evaluating every sample, bit for bit;
 * map_stats.render_evaluated counts the evaluated samples).  Views of more than max(2^18, the map's current ray
 * capacity) pixels are rendered in chunks of that many pixels (map_get_samples and
 * map_get_ray_outputs then describe the last chunk).  With host outputs the call
 * waits for the stream; with device outputs it returns once the work is queued.
 */
int map_render(map_handle h, const float c2w[12], const float K[4], uint32_t W, uint32_t H,
               float* out_rgb, float* out_depth, float* out_acc, int mem_kind, void* stream);

/*
 * map_render_group - forward-only renders of n views of one or more maps in shared
 * launches (the serving pattern: render queries of several resident scenes and of
 * different resolutions batched together).  View i shows maps[i] (maps may repeat)
 * from c2w[12 i .. 12 i + 11] with intrinsics K[4 i .. 4 i + 3] at W[i] x H[i]
 * pixels; its colour goes to out_rgb[i] (device, H*W*3 floats) and its expected ray
 * distance to out_depth[i] (device, H*W floats); out_rgb / out_depth or an entry may
 * be NULL.  c2w, K, W, H, out_rgb and out_depth are host arrays of n entries.  The
 * views are cut into batches of up to 2^18 rays; each batch runs as one sequence of
 * launches (ray casting, march with each map's box and occupancy bitfield,
 * compaction, a persistent tensor-core field forward over 128-sample tiles that
 * never mix two views, switching weights where the map changes, compositing with
 * each map's render_t_min, output); as in map_render, with a threshold the field is
 * evaluated for the first 32 samples of every ray and then only for the rays still
 * above it.  Every pixel goes through the arithmetic of map_render of its view, and
 * the images equal map_render's bit for bit.  Every map
 * must use the FP16 or BF16 MLP (plain FP32 maps: map_render).  All work is queued
 * on `stream`; the caller orders it after any work that changes the maps.  Work
 * buffers are held by maps[0] (allocated on first use).  Errors: MAP_EINVAL
 * (message on maps[0]), MAP_ENOMEM, MAP_ECUDA.
 */
int map_render_group(const map_handle* maps, uint32_t n, const float* c2w, const float* K, const uint32_t* W,
                     const uint32_t* H, float* const* out_rgb, float* const* out_depth, void* stream);

/* Parameter I/O.  Layout (FP32): tables [L][2^log2_table][F], then W1 [64][32],
 * W2 [16][64], W3 [64][32], W4 [64][64], W5 [3][64], each (out, in) row-major.
 * n must equal map_stats.param_count.  get/set wait for the stream. */
int map_get_params(map_handle h, float* dst, size_t n, int mem_kind, void* stream);
int map_set_params(map_handle h, const float* src, size_t n, int mem_kind, void* stream);
/* Gradient of L_M from the last step (meaningful after MAP_STEP_NO_UPDATE). */
int map_get_grads(map_handle h, float* dst, size_t n, int mem_kind, void* stream);

/*
 * Joint pose refinement (Sec. 3.2: L_M is minimised over the keyframe poses T as
 * well as the map).  After a map_step with MAP_STEP_POSE_GRAD, map_get_pose_grads
 * writes, for each keyframe slot s < n_kf, dst[6 s .. 6 s + 5] = (dL/drho, dL/dphi):
 * the gradient of the step's L_M under the left world-frame perturbation
 * T <- exp(xi) T, xi = (rho, phi) (a point p moves to R(phi) p + rho), with the
 * step's sample list held fixed.  Keyframes that drew no ray get zeros.  Slots are
 * numbered in the order keyframes were first added (a replaced kf_id keeps its
 * slot; map_get_keyframe_ids lists the ids by slot).  n_kf must not exceed the
 * number of keyframes.  Waits for the stream with host memory.  MAP_EINVAL
 * without a preceding POSE_GRAD step.
 */
int map_get_pose_grads(map_handle h, float* dst, uint32_t n_kf, int mem_kind, void* stream);
/*
 * map_marginal_covariances - the per-pixel depth variances that weight the depth
 * loss, from the tracking frontend's dense bundle adjustment (Sec. 3.1, Eq. cov):
 * the BA Hessian has the cameras/depths arrow structure H = [[C, E], [E^T, P]]
 * (Eq. hessian); then H_T = C - E P^-1 E^T = L L^T, Sigma_T = (L L^T)^-1 and
 * Sigma_d = diag(P^-1 + P^-T E^T Sigma_T E P^-1).  Stateless (no map handle); FP64.
 * C: c x c row-major (its lower triangle is read), c = 6 x keyframes, 6..144.
 * P: p positive diagonal entries (one per pixel inverse depth).  E block-sparse:
 * blk [p][B] int32 pose index per block (< c/6, or -1 = unused), e [p][B][6] the
 * rows 6 blk .. 6 blk + 5 of column q of E; 1 <= B <= 8.  Outputs: sigma_T c x c
 * row-major, sigma_d [p].  All arrays in mem_kind memory; the call waits for the
 * stream.  Errors: MAP_EINVAL (sizes, a non-positive P entry, a reduced camera
 * matrix that is not positive definite; message in map_last_error(NULL)),
 * MAP_ENOMEM, MAP_ECUDA.  The paper computes these in its tracking frontend; here
 * they take synthetic Hessians.
 */
int map_marginal_covariances(const double* C, uint32_t c, const double* P, uint32_t p,
                             const int32_t* blk, const double* e, uint32_t B, double* sigma_T,
                             double* sigma_d, int mem_kind, void* stream);

/*
 * Keyframe streaming (the paper's memory mitigation, Sec. 6: inactive parts of the
 * map are streamed to the CPU and only a window around the region of interest is
 * kept on the GPU).  map_evict_keyframe copies a keyframe's images to pinned host
 * memory and frees its device memory; from then on map_step draws rays only from
 * the device-resident keyframes, the k-th of them in slot order taking the place of
 * keyframe k of the draw (the keyframe slots and ids are unchanged).
 * map_restore_keyframe brings the images back (bit-identical) and makes the
 * keyframe drawable again; map_add_keyframe with the id of a streamed-out keyframe
 * replaces it with the new images.  Both wait for the stream.  Already evicted /
 * resident: no-op.  MAP_EINVAL for an unknown kf_id; map_step returns MAP_ENOKF
 * while every keyframe is streamed out.  map_keyframe_resident: 1 resident, 0
 * streamed out, MAP_EINVAL unknown.
 */
int map_evict_keyframe(map_handle h, uint32_t kf_id, void* stream);
int map_restore_keyframe(map_handle h, uint32_t kf_id, void* stream);
int map_keyframe_resident(map_handle h, uint32_t kf_id);

/*
 * Checkpoint (the paper has none: a mapping run that is stopped and resumed later,
 * or moved to another process).  map_save writes the map's state to the file `path`:
 * its configuration, the parameters, the Adam moments and step count, the occupancy
 * bitfield and density EMA, the occupancy refresh counter and, with
 * MAP_SAVE_KEYFRAMES, every keyframe (id, pose, intrinsics, size, residency and its
 * images in the map's own texel format, depth already in ray units).  The gradient
 * buffer is not saved: it is zero after every step that updates the map.  It waits
 * for the stream first.  Little-endian file, versioned; MAP_EINVAL (with a message)
 * when the file cannot be written.
 * map_load creates a map from such a file, as map_create would with the saved
 * configuration and hbm_budget_bytes, and restores that state bit for bit: with the
 * keyframes saved, its next map_step (same n_rays, seed and flags) draws the same
 * rays and samples and returns the same loss as the saved map's next step would (the
 * table gradients then agree up to the order of their FP32 atomics); without them it
 * has no keyframes (map_step: MAP_ENOKF) until they are added again.
 * Streamed-out keyframes are restored streamed out.  MAP_EINVAL for a missing,
 * truncated or foreign file or a configuration this library does not accept;
 * MAP_ENOMEM as map_create.
 */
#define MAP_SAVE_KEYFRAMES 1u
int map_save(map_handle h, const char* path, uint32_t flags, void* stream);
int map_load(const char* path, size_t hbm_budget_bytes, map_handle* out);

/* The kf_id of each keyframe slot: ids[s] for s < min(n, number of keyframes);
 * returns the number of keyframes (host memory). */
int map_get_keyframe_ids(map_handle h, uint32_t* ids, uint32_t n);
/* Replace the pose of keyframe kf_id (c2w[12], host memory, the layout of
 * map_add_keyframe), keeping its images; stream ordered.  MAP_EINVAL if the id is
 * not in the store. */
int map_set_keyframe_pose(map_handle h, uint32_t kf_id, const float c2w[12], void* stream);
/* Adam moments m, v (either may be NULL) and a reset of the optimiser state. */
int map_get_adam(map_handle h, float* m, float* v, size_t n, int mem_kind, void* stream);
int map_reset_adam(map_handle h, void* stream);

/*
 * Occupancy.  bits: occ_res^3 / 8 bytes, cell (cx, cy, cz) at linear index
 * b = cx + occ_res * (cy + occ_res * cz) is bit (b & 7) of byte (b >> 3).
 * density: occ_res^3 floats (the EMA).  map_set_occupancy also sets the EMA of
 * set cells to 1 and of clear cells to 0.  map_refresh_occupancy runs one refresh
 * now (refresh index = number of refreshes so far).
 */
int map_set_occupancy(map_handle h, const uint8_t* bits, size_t n_bytes, int mem_kind,
                      void* stream);
int map_get_occupancy(map_handle h, uint8_t* bits, float* density, int mem_kind, void* stream);
int map_set_occupancy_density(map_handle h, const float* density, size_t n, int mem_kind,
                              void* stream);
int map_refresh_occupancy(map_handle h, void* stream);

/* Inspection of the last step or render (for tests and tools); waits for the
 * stream.  Copies min(cap, n_samples) samples: ray index and t of each retained
 * sample in ray-major order, and per ray the rendered colour (3), depth and
 * opacity.  Any pointer may be NULL. */
int map_get_samples(map_handle h, uint32_t* ray_id, float* t, size_t cap, void* stream);
int map_get_ray_outputs(map_handle h, float* rgb, float* depth, float* acc, size_t n_rays,
                        void* stream);

int map_get_stats(map_handle h, map_stats* out);

/* Phase timing with CUDA events recorded on the caller's stream around each phase
 * of every subsequent step / render.  map_profile_enable(h, 1) starts (and clears)
 * the record, (h, 0) stops it.  map_profile_read waits for the recorded events and
 * returns, per MAP_PH_* phase, the summed milliseconds and the number of phase
 * executions and kernel launches (arrays of MAP_PHASES entries, any may be NULL). */
int map_profile_enable(map_handle h, int enable);
int map_profile_read(map_handle h, double* ms, uint64_t* count, uint64_t* launches);

/*
 * map_march_noalloc - the march and sample compaction of a mapping step (sample
 * positions, box and occupancy tests, first max_samples kept per ray, compacted in
 * ray order) for callers that cannot allocate device memory.  The paper has no
 * counterpart: it is a deployment variant of the library's march kernel.
 *
 * Who needs it: a caller whose GPU memory belongs to another allocator (a
 * framework's caching allocator that has reserved the device, or a fixed memory
 * budget), or a latency-critical host loop for which a cudaMalloc, which may
 * synchronise the device, would stall.  map_step and map_render allocate their
 * work buffers in the map; this call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  Its only scratch (per-ray counts and
 * scan totals) is a static device array of about 4 MB that every GPU loading the
 * library holds until the process exits.
 *
 * cfg: the march fields are used (near_t, step_t, n_steps <= 65536, max_samples
 *   <= 1024, grid_origin, grid_inv_size, box_max, occ_res).  occ_bits: device
 *   bitfield (layout as map_set_occupancy), read as 32-bit words, so it must be
 *   4-byte aligned; required when occ_res > 0, ignored otherwise.  Every device
 *   array of this call must be 4-byte aligned (misaligned: MAP_EINVAL, no launch).
 * rays_o, rays_d: device arrays [n_rays][3] (origin, unit direction).
 * n_rays: 1 .. 1048576 (the scratch size); larger values fail with MAP_EINVAL.
 * offsets: device [n_rays + 1], receives the exclusive scan of the per-ray sample
 *   counts (offsets[n_rays] = total); ray_id, t: device [cap_samples], receive
 *   the samples in ray order; cap_samples >= n_rays * max_samples is required.
 * stream: all work is queued on it; the call returns without waiting.
 * The first call on a device looks up the scratch array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture.  All calls share the scratch array: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the caller.
 * Errors: MAP_EINVAL (argument), MAP_ECUDA (address lookup or launch); the message
 * is available from map_last_error(NULL) (see there).
 */
int map_march_noalloc(const map_config* cfg, const uint8_t* occ_bits, const float* rays_o,
                      const float* rays_d, uint32_t n_rays, uint32_t* offsets, uint32_t* ray_id,
                      float* t, size_t cap_samples, void* stream);

/*
 * Serving: several maps resident on one GPU (Sec. 3.3's mapping thread, which
 * optimises continuously while keyframes arrive and renders are requested, run for
 * several scenes at once).  A server owns a worker thread; each admitted scene gets
 * its own map and CUDA stream.  Requests of one scene run in submission order, up to
 * max_inflight of them on the GPU at a time; requests arriving meanwhile join
 * between them, and different scenes' work overlaps on the device.  A scene with
 * continuous mapping fills every gap in its queue with a mapping step of step_rays
 * rays.  Scenes are admitted while the device's free memory covers the scene's
 * estimated footprint (tables, gradients, Adam moments, occupancy, step workspace,
 * kf_reserve_bytes of keyframes) plus hbm_reserve_bytes; otherwise the call returns
 * MAP_ENOMEM and may be retried once scenes have been removed or memory freed.
 *
 * Grouped renders (group_renders = 1): in each round of the worker, the render
 * queries at the head of the queues of all scenes with a tensor-core MLP (per MLP
 * type) are evaluated together, whatever their resolutions: the views are cut into
 * batches of up to 2^18 rays, and each batch runs as one sequence of shared launches
 * (ray casting, march with each scene's box and bitfield, compaction, a persistent
 * tensor-core field forward whose 128-sample tiles never mix two views and which
 * switches weights where the scene changes, compositing, output).  Every pixel goes
 * through the arithmetic of a render of its view alone, so the results are the same
 * bit for bit.  A grouped render runs on one of the server's two render streams
 * (taken in turn) after the work each scene has already queued, and each scene's
 * later work waits for it.  Plain FP32 scenes render on their own streams.
 */
typedef struct map_server_s* map_server;

#define MAP_REQ_KEYFRAME 0
#define MAP_REQ_STEP 1
#define MAP_REQ_RENDER 2

typedef struct map_server_config {
    uint32_t max_scenes;        /* scene slots, 1..64 */
    uint32_t max_inflight;      /* requests per scene on the GPU at once (>= 1); with several scenes
                                   1 gives the lowest keyframe and render latency at the same
                                   mapping throughput (the other scenes keep the GPU busy) */
    uint32_t step_rays;         /* rays of a continuous-mapping step */
    uint32_t group_renders;     /* 1: render queries of the FP16 / BF16 scenes that are due together
                                   run as one grouped render (see below); 0: each on its own */
    size_t hbm_reserve_bytes;   /* device memory left free at admission */
    size_t kf_reserve_bytes;    /* keyframe memory budgeted per scene */
    uint64_t seed;              /* reserved (each scene draws its rays from its map_config seed) */
} map_server_config;

/* One finished request.  Times are seconds since map_server_create.  A keyframe
 * is done when the first mapping step that can draw from it has completed (its
 * insertion, if the scene has no continuous mapping); step_index is that step
 * (keyframe) or the step's own index; loss is the step's L_M when requested. */
typedef struct map_completion {
    uint64_t req_id;
    uint64_t step_index;
    uint32_t scene;
    uint32_t kind;
    int32_t status;
    float loss;
    double t_submit;
    double t_start;
    double t_done;
} map_completion;

typedef struct map_server_stats {
    double t_now;
    uint64_t rays_done;     /* rays of all completed mapping steps */
    uint64_t steps_done;
    uint64_t device_bytes;  /* admitted scenes' estimated footprints */
    uint32_t n_scenes;
    uint32_t pending;       /* requests submitted and not yet polled */
    uint64_t grouped_renders; /* render queries evaluated in grouped renders */
    uint64_t group_batches;   /* grouped renders issued (each one or more shared launch sequences) */
} map_server_stats;

int map_server_create(const map_server_config* cfg, map_server* out);
/* Stops the worker, waits for the device and frees every scene. */
int map_server_destroy(map_server s);
/* Admission by free HBM (see above); cfg as for map_create. */
int map_server_add_scene(map_server s, const map_config* cfg, int continuous_mapping, uint32_t* scene_id);
/* The scene's map, for parameter and occupancy I/O while no request of the scene
 * is pending (the worker thread owns it otherwise). */
int map_server_scene_handle(map_server s, uint32_t scene, map_handle* out);
/* Copies the keyframe (host memory) before returning; semantics of map_add_keyframe. */
int map_server_submit_keyframe(map_server s, uint32_t scene, uint32_t kf_id, const float c2w[12],
                               const float K[4], uint32_t W, uint32_t H, const float* rgb, const float* depth,
                               const float* depth_var, int depth_is_z, uint64_t* req_id);
/* One mapping step of n_rays rays; want_loss: report L_M in the completion. */
int map_server_submit_step(map_server s, uint32_t scene, uint32_t n_rays, int want_loss, uint64_t* req_id);
/* Render into host buffers out_rgb (H*W*3) and out_depth (H*W), either may be
 * NULL; they must stay valid until the request's completion has been polled (the
 * poll writes them). */
int map_server_submit_render(map_server s, uint32_t scene, const float c2w[12], const float K[4], uint32_t W,
                             uint32_t H, float* out_rgb, float* out_depth, uint64_t* req_id);
/* Up to cap finished requests, oldest first. */
int map_server_poll(map_server s, map_completion* out, uint32_t cap, uint32_t* n_out);
int map_server_get_stats(map_server s, map_server_stats* out);

/*
 * map_set_wait_polls - the poll limit of every bounded wait of this map's
 * tensor-core kernels for the completion of their MMAs (default 2^24 polls).  No
 * counterpart in the paper: it exists to test the timeout path.  When a wait runs
 * out, the kernel stops waiting, skips the rest of its work (results of that step
 * or render are garbage: gradients, renders and the loss), waits for the MMAs it
 * has issued, frees its tensor memory and sets a device flag; the next call that
 * waits for the stream (map_step with out_loss, map_render with host outputs)
 * returns MAP_ETIMEOUT and clears the flag, and the map stays usable.  polls = 0
 * makes every wait expire at once.  Takes effect for the following calls.
 */
int map_set_wait_polls(map_handle h, uint32_t polls);

/* sizeof(map_config) as compiled into the library, so a binding can check that its
 * own copy of the struct has the same layout. */
size_t map_abi_config_size(void);

/* Message of the last failure on h.  h = NULL: the message of this host thread's
 * most recent call that takes no map handle (map_create, map_march_noalloc,
 * map_marginal_covariances), or "" when that call succeeded. */
const char* map_last_error(map_handle h);

#ifdef __cplusplus
}
#endif

#endif /* NERFMAP_H */
