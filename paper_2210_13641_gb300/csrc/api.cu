// api.cu - the C ABI declared in include/nerfmap.h: map state in device memory,
// keyframe store, and the stream-ordered launch sequence of one mapping step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nerfmap.h"
#include "internal.h"

using namespace nm;

namespace {

thread_local std::string g_global_error;

struct Keyframe {
    uint32_t id, W, H;
    float4* texels;          // device texels (nullptr while streamed out)
    size_t bytes;
    float4* host = nullptr;  // pinned host copy while streamed out
};

struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
    uint32_t launches;
};

}  // namespace

struct map_scene {
    map_config cfg;
    DevCfg dc;
    int device = 0;
    int n_sm = 0;
    size_t budget = 0, held = 0;
    std::vector<std::pair<void*, size_t>> allocs;

    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    size_t n_params = 0, n_table = 0;
    uint32_t* occ_bits = nullptr;
    float* occ_density = nullptr;
    uint32_t n_cells = 0;

    std::vector<Keyframe> kfs;
    std::vector<KfDesc> kf_desc;
    KfDesc* d_kfs = nullptr;
    uint32_t d_kfs_cap = 0;
    float* staging = nullptr;       // keyframe upload staging (rgb, depth, var)
    size_t staging_floats = 0;

    StepBufs bufs{};
    std::vector<void*> buf_allocs;
    uint32_t* d_active = nullptr;   // slots of the device-resident keyframes (when some are streamed out)
    uint32_t d_active_cap = 0;
    uint32_t* h_active = nullptr;   // pinned staging of that list
    cudaEvent_t active_ev = nullptr;
    uint32_t n_active = 0;
    bool all_active = true;
    float4* pose_s = nullptr;       // per-sample pose terms (allocated on the first POSE_GRAD step)
    uint64_t pose_s_cap = 0;
    float* pose_g = nullptr;        // [pose_g_cap][8] per keyframe slot
    uint32_t pose_g_cap = 0;
    bool pose_valid = false;

    uint64_t step = 0, n_refresh = 0;
    bool grads_dirty = false;
    uint32_t last_rays = 0;
    cudaStream_t last_stream = nullptr;
    uint64_t launches = 0;
    bool prof_on = false;
    std::vector<PhaseRec> prof;
    std::string err;
    GroupBufs group{};              // work buffers of map_render_group calls led by this map
    uint32_t* render_off = nullptr; // [cap_rays + 1] scan of a two-pass render's selection
    uint32_t render_off_cap = 0;
};

namespace {

int fail(map_scene* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_global_error = msg;
    return code;
}

int cuda_fail(map_scene* h, cudaError_t e, const char* what) {
    return fail(h, MAP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NM_CUDA(h, call)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

int dalloc(map_scene* h, void** p, size_t bytes) {
    if (h->budget && h->held + bytes > h->budget)
        return fail(h, MAP_ENOMEM, "HBM budget exceeded (" + std::to_string(h->held + bytes) + " > " +
                                       std::to_string(h->budget) + " bytes)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, MAP_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->held += bytes;
    h->allocs.emplace_back(*p, bytes);
    return MAP_OK;
}

void dfree(map_scene* h, void* p) {
    if (!p) return;
    for (size_t i = 0; i < h->allocs.size(); ++i) {
        if (h->allocs[i].first == p) {
            h->held -= h->allocs[i].second;
            h->allocs.erase(h->allocs.begin() + i);
            break;
        }
    }
    cudaFree(p);
}

int validate(const map_config* c, std::string& why) {
    if (!c) return why = "null config", MAP_EINVAL;
    if (c->n_levels < 1 || c->n_levels > 16) return why = "n_levels must be 1..16", MAP_EINVAL;
    if (c->n_features != 2) return why = "n_features must be 2", MAP_EINVAL;
    if (c->log2_table < 10 || c->log2_table > 24) return why = "log2_table must be 10..24", MAP_EINVAL;
    for (uint32_t l = 0; l < c->n_levels; ++l)
        if (c->level_res[l] < 2 || c->level_res[l] > (1u << 20)) return why = "level_res out of range", MAP_EINVAL;
    if (c->enc_width != 32 || c->density_hidden != 64 || c->geo_width != 16 || c->color_hidden != 64)
        return why = "MLP widths must be 32/64/16/64", MAP_EINVAL;
    if (!(c->step_t > 0.f) || c->n_steps == 0 || c->n_steps > 65536) return why = "bad march", MAP_EINVAL;
    if (c->max_samples == 0 || c->max_samples > 1024) return why = "max_samples must be 1..1024", MAP_EINVAL;
    if (c->occ_res % 8 != 0 || c->occ_res > 1024) return why = "occ_res must be a multiple of 8, <= 1024", MAP_EINVAL;
    if (!(c->grid_inv_size > 0.f)) return why = "grid_inv_size must be > 0", MAP_EINVAL;
    if (c->precision > 2) return why = "precision must be 0, 1 or 2", MAP_EINVAL;
    return MAP_OK;
}

int ensure_step_bufs(map_scene* h, uint32_t n_rays) {
    const uint64_t need_samples = (uint64_t)n_rays * h->cfg.max_samples;
    const bool need_feat = true;
    if (h->bufs.cap_rays >= n_rays && h->bufs.cap_samples >= need_samples) return MAP_OK;
    cudaDeviceSynchronize();
    for (void* p : h->buf_allocs) dfree(h, p);
    h->buf_allocs.clear();
    StepBufs b{};
    const uint32_t cap = std::max<uint32_t>(n_rays, 1024);
    const uint64_t cs = (uint64_t)cap * h->cfg.max_samples;
    const uint32_t n_tiles = (cap + kScanTile - 1) / kScanTile;
    struct Req { void** p; size_t bytes; };
    std::vector<Req> reqs = {
        {(void**)&b.rays, sizeof(float) * kRayPlanes * cap},
        {(void**)&b.counts, sizeof(uint32_t) * cap},
        {(void**)&b.offsets, sizeof(uint32_t) * (cap + 1)},
        {(void**)&b.block_sums, sizeof(uint32_t) * (n_tiles + 1)},
        {(void**)&b.ray_id, sizeof(uint32_t) * cs},
        {(void**)&b.t, sizeof(float) * cs},
        {(void**)&b.sig_rgb, sizeof(float4) * cs},
        {(void**)&b.dsig_rgb, sizeof(float4) * cs},
        {(void**)&b.ray_out, sizeof(float) * 5 * cap},
        {(void**)&b.loss, 64},
        {(void**)&b.partials, sizeof(float) * 4 * kCompositeMaxBlocks},
        {(void**)&b.err, 64},
    };
    if (need_feat) reqs.push_back({(void**)&b.feat, sizeof(float) * kEnc * cs});
    for (auto& r : reqs) {
        int rc = dalloc(h, r.p, r.bytes);
        if (rc) {
            for (void* p : h->buf_allocs) dfree(h, p);
            h->buf_allocs.clear();
            h->bufs = StepBufs{};
            return rc;
        }
        h->buf_allocs.push_back(*r.p);
    }
    b.cap_rays = cap;
    b.cap_samples = cs;
    cudaMemset(b.loss, 0, 64);
    cudaMemset(b.err, 0, 64);
    h->bufs = b;
    return MAP_OK;
}

void fill_devcfg(map_scene* h) {
    const map_config& c = h->cfg;
    DevCfg& d = h->dc;
    std::memset(&d, 0, sizeof(d));
    d.L = c.n_levels;
    d.log2T = c.log2_table;
    d.T = 1u << c.log2_table;
    d.dense_mask = 0;
    for (uint32_t l = 0; l < c.n_levels; ++l) {
        d.res[l] = c.level_res[l];
        const uint64_t s = (uint64_t)c.level_res[l] + 1;
        if (s * s * s <= d.T) d.dense_mask |= 1u << l;
    }
    d.near_t = c.near_t;
    d.step_t = c.step_t;
    d.n_steps = c.n_steps;
    d.max_samples = c.max_samples;
    for (int a = 0; a < 3; ++a) {
        d.org[a] = c.grid_origin[a];
        d.box[a] = c.box_max[a];
    }
    d.inv_size = c.grid_inv_size;
    d.occ_res = c.occ_res;
    d.lambda_d = c.lambda_d;
    d.t_min = 0.f;
    d.wait_polls = kWaitPollsDefault;
}

int copy_in(map_scene* h, void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t s) {
    const cudaMemcpyKind k = mem_kind == MAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    NM_CUDA(h, cudaMemcpyAsync(dst, src, bytes, k, s));
    return MAP_OK;
}

int copy_out(map_scene* h, void* dst, const void* src, size_t bytes, int mem_kind, cudaStream_t s) {
    const cudaMemcpyKind k = mem_kind == MAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    NM_CUDA(h, cudaMemcpyAsync(dst, src, bytes, k, s));
    NM_CUDA(h, cudaStreamSynchronize(s));
    return MAP_OK;
}

// Error word the kernels set instead of trapping (a bounded wait that expired).
int check_device_flags(map_scene* h, cudaStream_t s) {
    uint32_t e = 0;
    NM_CUDA(h, cudaMemcpyAsync(&e, h->bufs.err, sizeof(e), cudaMemcpyDeviceToHost, s));
    NM_CUDA(h, cudaStreamSynchronize(s));
    if (e & kErrTimeout) {
        cudaMemsetAsync(h->bufs.err, 0, sizeof(uint32_t), s);
        return fail(h, MAP_ETIMEOUT, "a tensor-core wait expired on the device");
    }
    return MAP_OK;
}

int check_launch(map_scene* h, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    return MAP_OK;
}

constexpr uint32_t kRenderChunk = 1u << 18;

const char* const kPhaseName[MAP_PHASES] = {"ray_gen", "march", "field_fwd", "composite",
                                             "field_bwd", "adam", "occupancy", "output"};

// Runs one phase: optional CUDA events around it on the stream, launch check and
// launch accounting.
template <class F>
int phase(map_scene* h, int ph, uint32_t n_launch, cudaStream_t s, F&& f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (h->prof_on) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    nvtxRangePushA(kPhaseName[ph]);  // named host range around the phase's launches (profilers)
    f();
    nvtxRangePop();
    int rc = check_launch(h, kPhaseName[ph]);
    if (h->prof_on) {
        cudaEventRecord(b, s);
        h->prof.push_back(PhaseRec{ph, a, b, n_launch});
    }
    h->launches += n_launch;
    return rc;
}

void prof_clear(map_scene* h) {
    for (auto& r : h->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    h->prof.clear();
}

}  // namespace

namespace nm {
bool scene_view(const ::map_scene* h, SceneView* out) {
    if (!h || !out) return false;
    out->dc = h->dc;
    out->dc.t_min = h->cfg.render_t_min;
    out->params = h->params;
    out->occ = h->occ_bits;
    out->precision = h->cfg.precision;
    return true;
}

void clear_global_error() { g_global_error.clear(); }
void set_global_error(const char* msg) { g_global_error = msg; }
}  // namespace nm

extern "C" {

int map_config_init(map_config* cfg, uint32_t n_levels, uint32_t log2_table, uint32_t n_min, uint32_t n_max,
                    double growth) {
    g_global_error.clear();
    if (!cfg) return fail(nullptr, MAP_EINVAL, "map_config_init: null config");
    if (n_levels < 1 || n_levels > 16) return fail(nullptr, MAP_EINVAL, "map_config_init: n_levels must be 1..16");
    if (log2_table < 10 || log2_table > 24) return fail(nullptr, MAP_EINVAL, "map_config_init: log2_table must be 10..24");
    if (n_min < 2) return fail(nullptr, MAP_EINVAL, "map_config_init: n_min must be >= 2");
    double b = 1.0;
    if (growth > 0.0) b = growth;
    else if (n_levels > 1) {
        if (n_max <= n_min) return fail(nullptr, MAP_EINVAL, "map_config_init: need growth > 0 or n_max > n_min");
        b = std::exp(std::log((double)n_max / (double)n_min) / (double)(n_levels - 1));
    }
    std::memset(cfg, 0, sizeof(*cfg));
    for (uint32_t l = 0; l < n_levels; ++l) {
        const double N = std::floor((double)n_min * std::pow(b, (double)l) * (1.0 + 1e-9));
        if (N > (double)(1u << 20)) return fail(nullptr, MAP_EINVAL, "map_config_init: a level exceeds 2^20");
        cfg->level_res[l] = (uint32_t)N;
    }
    cfg->n_levels = n_levels;
    cfg->n_features = 2;
    cfg->log2_table = log2_table;
    cfg->enc_width = kEnc;
    cfg->density_hidden = kHid;
    cfg->geo_width = kGeo;
    cfg->color_hidden = kHid;
    cfg->max_samples = 128;
    cfg->occ_every = 16;
    cfg->occ_decay = 0.95f;
    cfg->occ_thresh = 0.01f;
    cfg->lambda_d = 1.f;
    cfg->lr = 1e-2f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.99f;
    cfg->eps = 1e-15f;
    cfg->render_t_min = 1e-4f;
    cfg->precision = MAP_PREC_FP16;
    return MAP_OK;
}

int map_create(const map_config* cfg, size_t hbm_budget_bytes, map_handle* out) {
    std::string why;
    g_global_error.clear();
    if (!out) return fail(nullptr, MAP_EINVAL, "null output handle");
    *out = nullptr;
    if (validate(cfg, why) != MAP_OK) return fail(nullptr, MAP_EINVAL, why);
    map_scene* h = new map_scene();
    h->cfg = *cfg;
    h->budget = hbm_budget_bytes;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    fill_devcfg(h);
    h->n_table = (size_t)cfg->n_levels * (1u << cfg->log2_table) * 2;
    h->n_params = h->n_table + kMlpParams;
    const size_t pb = h->n_params * sizeof(float);
    int rc = MAP_OK;
    if (!rc) rc = dalloc(h, (void**)&h->params, pb);
    if (!rc) rc = dalloc(h, (void**)&h->grads, pb);
    if (!rc) rc = dalloc(h, (void**)&h->adam_m, pb);
    if (!rc) rc = dalloc(h, (void**)&h->adam_v, pb);
    if (!rc && cfg->occ_res) {
        h->n_cells = cfg->occ_res * cfg->occ_res * cfg->occ_res;
        rc = dalloc(h, (void**)&h->occ_bits, h->n_cells / 8);
        if (!rc) rc = dalloc(h, (void**)&h->occ_density, h->n_cells * sizeof(float));
    }
    if (rc) {
        g_global_error = h->err;
        map_destroy(h);
        return rc;
    }
    cudaMemset(h->grads, 0, pb);
    cudaMemset(h->adam_m, 0, pb);
    cudaMemset(h->adam_v, 0, pb);
    if (h->occ_bits) {
        cudaMemset(h->occ_bits, 0xFF, h->n_cells / 8);  // all occupied until set or refreshed
        launch_occ_from_bits(h->occ_bits, h->occ_density, h->n_cells, nullptr);
    }
    launch_init_params(h->params, h->n_table, cfg->seed, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_global_error = std::string("init: ") + cudaGetErrorString(e);
        map_destroy(h);
        return MAP_ECUDA;
    }
    *out = h;
    return MAP_OK;
}

int map_destroy(map_handle h) {
    if (!h) return MAP_EINVAL;
    cudaDeviceSynchronize();
    prof_clear(h);
    for (auto& kf : h->kfs)
        if (kf.host) cudaFreeHost(kf.host);
    if (h->h_active) cudaFreeHost(h->h_active);
    if (h->active_ev) cudaEventDestroy(h->active_ev);
    for (auto& a : h->allocs) cudaFree(a.first);
    h->allocs.clear();
    if (h->group.items) group_bufs_free(h->group);
    delete h;
    return MAP_OK;
}

static int rebuild_active(map_scene* h, cudaStream_t s);

int map_add_keyframe(map_handle h, uint32_t kf_id, const float c2w[12], const float K[4], uint32_t W,
                     uint32_t H, const float* rgb, const float* depth, const float* depth_var,
                     int depth_is_z, int mem_kind, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!c2w || !K || !rgb || !depth || !depth_var) return fail(h, MAP_EINVAL, "null keyframe input");
    if (W == 0 || H == 0 || (uint64_t)W * H > (1ull << 26)) return fail(h, MAP_EINVAL, "bad keyframe size");
    if (!(K[0] > 0.f) || !(K[1] > 0.f)) return fail(h, MAP_EINVAL, "focal lengths must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const size_t npx = (size_t)W * H;
    size_t idx = h->kfs.size();
    for (size_t i = 0; i < h->kfs.size(); ++i)
        if (h->kfs[i].id == kf_id) idx = i;
    if (idx < h->kfs.size() && (h->kfs[idx].W != W || h->kfs[idx].H != H)) {
        cudaStreamSynchronize(s);
        dfree(h, h->kfs[idx].texels);
        h->kfs[idx].texels = nullptr;
    }
    if (idx == h->kfs.size()) h->kfs.push_back(Keyframe{kf_id, W, H, nullptr, 0});
    Keyframe& kf = h->kfs[idx];
    if (kf.host) {  // a streamed-out keyframe is replaced by the new images
        cudaFreeHost(kf.host);
        kf.host = nullptr;
    }
    kf.W = W;
    kf.H = H;
    if (!kf.texels) {
        int rc = dalloc(h, (void**)&kf.texels, npx * 2 * sizeof(float4));
        if (rc) {
            // drop the entry (new, or replaced at a new size) and republish the table
            h->kfs.erase(h->kfs.begin() + idx);
            if (idx < h->kf_desc.size()) h->kf_desc.erase(h->kf_desc.begin() + idx);
            if (h->d_kfs)
                for (size_t i = 0; i < h->kf_desc.size(); ++i)
                    launch_set_kf_desc(h->d_kfs, (uint32_t)i, h->kf_desc[i], s);
            if (!h->all_active) rebuild_active(h, s);
            return fail(h, rc, h->err);
        }
        kf.bytes = npx * 2 * sizeof(float4);
    }
    const float *d_rgb = rgb, *d_depth = depth, *d_var = depth_var;
    if (mem_kind != MAP_MEM_DEVICE) {
        if (h->staging_floats < npx * 5) {
            cudaStreamSynchronize(s);
            dfree(h, h->staging);
            h->staging = nullptr;
            int rc = dalloc(h, (void**)&h->staging, npx * 5 * sizeof(float));
            if (rc) return rc;
            h->staging_floats = npx * 5;
        }
        int rc = copy_in(h, h->staging, rgb, npx * 3 * sizeof(float), MAP_MEM_HOST, s);
        if (!rc) rc = copy_in(h, h->staging + npx * 3, depth, npx * sizeof(float), MAP_MEM_HOST, s);
        if (!rc) rc = copy_in(h, h->staging + npx * 4, depth_var, npx * sizeof(float), MAP_MEM_HOST, s);
        if (rc) return rc;
        d_rgb = h->staging;
        d_depth = h->staging + npx * 3;
        d_var = h->staging + npx * 4;
    }
    launch_keyframe_texels(d_rgb, d_depth, d_var, W, H, K, depth_is_z, kf.texels, s);
    int rc = check_launch(h, "keyframe texels");
    if (rc) return rc;
    // device keyframe table
    KfDesc dsc;
    std::memcpy(dsc.c2w, c2w, sizeof(dsc.c2w));
    std::memcpy(dsc.K, K, sizeof(dsc.K));
    dsc.W = W;
    dsc.H = H;
    dsc.texels = kf.texels;
    if (h->kf_desc.size() <= idx) h->kf_desc.resize(idx + 1);
    h->kf_desc[idx] = dsc;
    if (h->d_kfs_cap < h->kf_desc.size()) {
        // grow the device table: rewrite every descriptor into the new one
        cudaStreamSynchronize(s);
        dfree(h, h->d_kfs);
        h->d_kfs = nullptr;
        const uint32_t cap = std::max<uint32_t>(64, (uint32_t)h->kf_desc.size() * 2);
        rc = dalloc(h, (void**)&h->d_kfs, cap * sizeof(KfDesc));
        if (rc) return rc;
        h->d_kfs_cap = cap;
        for (size_t i = 0; i < h->kf_desc.size(); ++i) launch_set_kf_desc(h->d_kfs, (uint32_t)i, h->kf_desc[i], s);
    } else {
        launch_set_kf_desc(h->d_kfs, (uint32_t)idx, dsc, s);
    }
    rc = check_launch(h, "keyframe table");
    if (!rc && !h->all_active) rc = rebuild_active(h, s);  // the new or replaced slot is drawn again
    return rc;
}

static int run_forward(map_scene* h, uint32_t n_rays, bool train, cudaStream_t s) {
    const StepBufs& b = h->bufs;
    int rc = phase(h, MAP_PH_MARCH, 5, s, [&] { launch_march(h->dc, h->occ_bits, n_rays, b, s); });
    if (rc) return rc;
    return phase(h, MAP_PH_FIELD_FWD, 1, s, [&] {
        if (h->cfg.precision == MAP_PREC_FP32)
            launch_field_fwd_fp32(h->dc, h->params, n_rays, b, train, h->n_sm, s);
        else
            launch_field_fwd_tc(h->dc, h->params, n_rays, b, train, h->cfg.precision == MAP_PREC_BF16, h->n_sm, s);
    });
}

int map_step(map_handle h, uint32_t n_rays, uint64_t seed, uint32_t flags, float* out_loss, void* stream) {
    if (!h) return MAP_EINVAL;
    if (n_rays == 0 || n_rays > (1u << 24)) return fail(h, MAP_EINVAL, "n_rays must be 1..2^24");
    if (h->kfs.empty()) return fail(h, MAP_ENOKF, "no keyframes");
    if (!h->all_active && h->n_active == 0) return fail(h, MAP_ENOKF, "every keyframe is streamed out");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    int rc = ensure_step_bufs(h, n_rays);
    if (rc) return rc;
    if (h->grads_dirty) {
        NM_CUDA(h, cudaMemsetAsync(h->grads, 0, h->n_params * sizeof(float), s));
        h->grads_dirty = false;
    }
    const bool pose = (flags & MAP_STEP_POSE_GRAD) != 0;
    h->pose_valid = false;
    if (pose) {
        if (h->pose_s_cap < h->bufs.cap_samples) {
            cudaStreamSynchronize(s);
            dfree(h, h->pose_s);
            h->pose_s = nullptr;
            h->pose_s_cap = 0;
            rc = dalloc(h, (void**)&h->pose_s, h->bufs.cap_samples * 2 * sizeof(float4));
            if (rc) return rc;
            h->pose_s_cap = h->bufs.cap_samples;
        }
        if (h->pose_g_cap < h->kfs.size()) {
            cudaStreamSynchronize(s);
            dfree(h, h->pose_g);
            h->pose_g = nullptr;
            h->pose_g_cap = 0;
            const uint32_t cap = std::max<uint32_t>(64, (uint32_t)h->kfs.size() * 2);
            rc = dalloc(h, (void**)&h->pose_g, (size_t)cap * 8 * sizeof(float));
            if (rc) return rc;
            h->pose_g_cap = cap;
        }
        h->bufs.pose_s = h->pose_s;
        NM_CUDA(h, cudaMemsetAsync(h->pose_g, 0, h->kfs.size() * 8 * sizeof(float), s));
    }
    const StepBufs& b = h->bufs;
    rc = phase(h, MAP_PH_RAYGEN, 1, s,
               [&] {
                   launch_ray_gen(h->d_kfs, h->all_active ? nullptr : h->d_active,
                                  h->all_active ? (uint32_t)h->kfs.size() : h->n_active, seed, h->step, n_rays, b, s);
               });
    if (!rc) rc = run_forward(h, n_rays, true, s);
    if (!rc) rc = phase(h, MAP_PH_COMPOSITE, 1, s, [&] { launch_composite(h->dc, n_rays, true, b, s); });
    if (!rc)
        rc = phase(h, MAP_PH_FIELD_BWD, 1, s, [&] {
            if (h->cfg.precision == MAP_PREC_FP32)
                launch_field_bwd_fp32(h->dc, h->params, h->grads, n_rays, b, h->n_sm, s, pose);
            else
                launch_field_bwd_tc(h->dc, h->params, h->grads, n_rays, b, h->cfg.precision == MAP_PREC_BF16,
                                    h->n_sm, s, pose);
        });
    if (!rc && pose) {
        rc = phase(h, MAP_PH_FIELD_BWD, 1, s, [&] { launch_pose_reduce(h->dc, n_rays, b, h->pose_g, s); });
        if (!rc) h->pose_valid = true;
    }
    if (rc) return rc;
    h->last_rays = n_rays;
    if (!(flags & MAP_STEP_NO_UPDATE)) {
        const double t = (double)(h->step + 1);
        const float c1 = (float)(1.0 / (1.0 - std::pow((double)h->cfg.beta1, t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow((double)h->cfg.beta2, t)));
        rc = phase(h, MAP_PH_ADAM, 1, s, [&] {
            launch_adam(h->params, h->grads, h->adam_m, h->adam_v, h->n_params, h->cfg.lr, h->cfg.beta1,
                        h->cfg.beta2, h->cfg.eps, c1, c2, s);
        });
        if (rc) return rc;
        h->step += 1;
        if (h->occ_bits && h->cfg.occ_every && h->step % h->cfg.occ_every == 0) {
            rc = phase(h, MAP_PH_OCC, 1, s, [&] {
                launch_occ_refresh(h->dc, h->params, h->occ_density, h->occ_bits, h->cfg.seed, h->n_refresh,
                                   h->cfg.occ_decay, h->cfg.occ_thresh, s);
            });
            h->n_refresh += 1;
            if (rc) return rc;
        }
    } else {
        h->grads_dirty = true;
    }
    if (out_loss) {
        rc = copy_out(h, out_loss, b.loss, sizeof(float), MAP_MEM_HOST, s);
        if (rc) return rc;
        return check_device_flags(h, s);
    }
    return MAP_OK;
}

const float* map_loss_device(map_handle h) { return h ? h->bufs.loss : nullptr; }

// The list of device-resident keyframe slots the ray draw uses (in slot order);
// none while every keyframe is resident.  The pinned staging buffer is reused only
// after the previous upload from it has completed.
static int rebuild_active(map_scene* h, cudaStream_t s) {
    std::vector<uint32_t> act;
    for (size_t i = 0; i < h->kfs.size(); ++i)
        if (h->kfs[i].texels) act.push_back((uint32_t)i);
    h->all_active = act.size() == h->kfs.size();
    h->n_active = (uint32_t)act.size();
    if (h->all_active || act.empty()) return MAP_OK;
    if (h->d_active_cap < act.size()) {
        cudaStreamSynchronize(s);
        dfree(h, h->d_active);
        h->d_active = nullptr;
        if (h->h_active) cudaFreeHost(h->h_active);
        h->h_active = nullptr;
        const uint32_t cap = std::max<uint32_t>(64, (uint32_t)h->kfs.size() * 2);
        int rc = dalloc(h, (void**)&h->d_active, cap * sizeof(uint32_t));
        if (rc) return rc;
        NM_CUDA(h, cudaMallocHost((void**)&h->h_active, cap * sizeof(uint32_t)));
        h->d_active_cap = cap;
    }
    if (!h->active_ev) NM_CUDA(h, cudaEventCreateWithFlags(&h->active_ev, cudaEventDisableTiming));
    NM_CUDA(h, cudaEventSynchronize(h->active_ev));
    std::memcpy(h->h_active, act.data(), act.size() * sizeof(uint32_t));
    NM_CUDA(h, cudaMemcpyAsync(h->d_active, h->h_active, act.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    NM_CUDA(h, cudaEventRecord(h->active_ev, s));
    return MAP_OK;
}

int map_evict_keyframe(map_handle h, uint32_t kf_id, void* stream) {
    if (!h) return MAP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < h->kfs.size(); ++i) {
        Keyframe& kf = h->kfs[i];
        if (kf.id != kf_id) continue;
        if (!kf.texels) return MAP_OK;  // already streamed out
        NM_CUDA(h, cudaMallocHost((void**)&kf.host, kf.bytes));
        NM_CUDA(h, cudaMemcpyAsync(kf.host, kf.texels, kf.bytes, cudaMemcpyDeviceToHost, s));
        NM_CUDA(h, cudaStreamSynchronize(s));  // the copy and every step that read the texels are done
        dfree(h, kf.texels);
        kf.texels = nullptr;
        h->kf_desc[i].texels = nullptr;
        launch_set_kf_desc(h->d_kfs, (uint32_t)i, h->kf_desc[i], s);
        int rc = check_launch(h, "keyframe table");
        if (rc) return rc;
        return rebuild_active(h, s);
    }
    return fail(h, MAP_EINVAL, "unknown kf_id");
}

int map_restore_keyframe(map_handle h, uint32_t kf_id, void* stream) {
    if (!h) return MAP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < h->kfs.size(); ++i) {
        Keyframe& kf = h->kfs[i];
        if (kf.id != kf_id) continue;
        if (kf.texels) return MAP_OK;  // resident
        int rc = dalloc(h, (void**)&kf.texels, kf.bytes);
        if (rc) return rc;
        NM_CUDA(h, cudaMemcpyAsync(kf.texels, kf.host, kf.bytes, cudaMemcpyHostToDevice, s));
        NM_CUDA(h, cudaStreamSynchronize(s));
        cudaFreeHost(kf.host);
        kf.host = nullptr;
        h->kf_desc[i].texels = kf.texels;
        launch_set_kf_desc(h->d_kfs, (uint32_t)i, h->kf_desc[i], s);
        rc = check_launch(h, "keyframe table");
        if (rc) return rc;
        return rebuild_active(h, s);
    }
    return fail(h, MAP_EINVAL, "unknown kf_id");
}

int map_keyframe_resident(map_handle h, uint32_t kf_id) {
    if (!h) return MAP_EINVAL;
    for (const auto& kf : h->kfs)
        if (kf.id == kf_id) return kf.texels ? 1 : 0;
    return fail(h, MAP_EINVAL, "unknown kf_id");
}

// ------------------------------------------------------------------ checkpoint
// File layout (host byte order; both supported hosts are little-endian):
//   "NMAPCKPT", u32 version, u32 flags, u32 sizeof(map_config), map_config,
//   u64 step, u64 n_refresh, u64 n_params, f32 params / adam_m / adam_v [n_params],
//   u32 n_cells, u8 bits [n_cells / 8], f32 density [n_cells],
//   u32 n_kf, per keyframe: u32 id, W, H, resident, f32 c2w[12], K[4], u64 bytes, texels.
namespace {

constexpr char kCkptMagic[8] = {'N', 'M', 'A', 'P', 'C', 'K', 'P', 'T'};
constexpr uint32_t kCkptVersion = 1;
constexpr size_t kCkptChunk = size_t(64) << 20;

struct CkptFile {
    FILE* f = nullptr;
    ~CkptFile() {
        if (f) std::fclose(f);
    }
};

bool ck_write(FILE* f, const void* p, size_t n) { return std::fwrite(p, 1, n, f) == n; }
bool ck_read(FILE* f, void* p, size_t n) { return std::fread(p, 1, n, f) == n; }

// Device memory to the file (and back) through a host buffer, in chunks.
bool ck_write_dev(FILE* f, const void* d, size_t n, std::vector<uint8_t>& tmp) {
    for (size_t o = 0; o < n; o += kCkptChunk) {
        const size_t m = std::min(kCkptChunk, n - o);
        tmp.resize(m);
        if (cudaMemcpy(tmp.data(), static_cast<const uint8_t*>(d) + o, m, cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        if (!ck_write(f, tmp.data(), m)) return false;
    }
    return true;
}

bool ck_read_dev(FILE* f, void* d, size_t n, std::vector<uint8_t>& tmp) {
    for (size_t o = 0; o < n; o += kCkptChunk) {
        const size_t m = std::min(kCkptChunk, n - o);
        tmp.resize(m);
        if (!ck_read(f, tmp.data(), m)) return false;
        if (cudaMemcpy(static_cast<uint8_t*>(d) + o, tmp.data(), m, cudaMemcpyHostToDevice) != cudaSuccess)
            return false;
    }
    return true;
}

}  // namespace

int map_save(map_handle h, const char* path, uint32_t flags, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!path) return fail(h, MAP_EINVAL, "null path");
    if (flags & ~MAP_SAVE_KEYFRAMES) return fail(h, MAP_EINVAL, "unknown checkpoint flags");
    NM_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
    CkptFile F;
    F.f = std::fopen(path, "wb");
    if (!F.f) return fail(h, MAP_EINVAL, std::string("cannot open ") + path + " for writing");
    std::vector<uint8_t> tmp;
    const uint32_t cfg_size = sizeof(map_config);
    const uint64_t step = h->step, n_refresh = h->n_refresh, n_params = h->n_params;
    const uint32_t n_cells = h->n_cells;
    const uint32_t n_kf = (flags & MAP_SAVE_KEYFRAMES) ? (uint32_t)h->kfs.size() : 0u;
    const size_t pb = h->n_params * sizeof(float);
    bool ok = ck_write(F.f, kCkptMagic, sizeof(kCkptMagic)) && ck_write(F.f, &kCkptVersion, 4) &&
              ck_write(F.f, &flags, 4) && ck_write(F.f, &cfg_size, 4) && ck_write(F.f, &h->cfg, cfg_size) &&
              ck_write(F.f, &step, 8) && ck_write(F.f, &n_refresh, 8) && ck_write(F.f, &n_params, 8) &&
              ck_write_dev(F.f, h->params, pb, tmp) && ck_write_dev(F.f, h->adam_m, pb, tmp) &&
              ck_write_dev(F.f, h->adam_v, pb, tmp) && ck_write(F.f, &n_cells, 4);
    if (ok && n_cells)
        ok = ck_write_dev(F.f, h->occ_bits, n_cells / 8, tmp) &&
             ck_write_dev(F.f, h->occ_density, (size_t)n_cells * sizeof(float), tmp);
    ok = ok && ck_write(F.f, &n_kf, 4);
    for (uint32_t i = 0; ok && i < n_kf; ++i) {
        const Keyframe& kf = h->kfs[i];
        const KfDesc& d = h->kf_desc[i];
        const uint32_t rec[4] = {kf.id, kf.W, kf.H, kf.texels ? 1u : 0u};
        const uint64_t bytes = kf.bytes;
        ok = ck_write(F.f, rec, sizeof(rec)) && ck_write(F.f, d.c2w, sizeof(d.c2w)) &&
             ck_write(F.f, d.K, sizeof(d.K)) && ck_write(F.f, &bytes, 8) &&
             (kf.texels ? ck_write_dev(F.f, kf.texels, kf.bytes, tmp) : ck_write(F.f, kf.host, kf.bytes));
    }
    const bool closed = std::fclose(F.f) == 0;
    F.f = nullptr;
    if (!ok || !closed) return fail(h, MAP_EINVAL, std::string("writing ") + path + " failed");
    return MAP_OK;
}

int map_load(const char* path, size_t hbm_budget_bytes, map_handle* out) {
    g_global_error.clear();
    if (!out) return fail(nullptr, MAP_EINVAL, "null output handle");
    *out = nullptr;
    if (!path) return fail(nullptr, MAP_EINVAL, "null path");
    CkptFile F;
    F.f = std::fopen(path, "rb");
    if (!F.f) return fail(nullptr, MAP_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    uint32_t version = 0, flags = 0, cfg_size = 0;
    map_config cfg;
    if (!ck_read(F.f, magic, 8) || std::memcmp(magic, kCkptMagic, 8) != 0 || !ck_read(F.f, &version, 4) ||
        version != kCkptVersion || !ck_read(F.f, &flags, 4) || !ck_read(F.f, &cfg_size, 4) ||
        cfg_size != sizeof(map_config) || !ck_read(F.f, &cfg, sizeof(cfg)))
        return fail(nullptr, MAP_EINVAL, std::string(path) + ": not a checkpoint of this library version");
    uint64_t step = 0, n_refresh = 0, n_params = 0;
    if (!ck_read(F.f, &step, 8) || !ck_read(F.f, &n_refresh, 8) || !ck_read(F.f, &n_params, 8))
        return fail(nullptr, MAP_EINVAL, std::string(path) + ": truncated");
    map_handle h = nullptr;
    int rc = map_create(&cfg, hbm_budget_bytes, &h);
    if (rc) return rc;
    auto bad = [&](const std::string& what) {
        map_destroy(h);
        return fail(nullptr, MAP_EINVAL, std::string(path) + ": " + what);
    };
    if (n_params != h->n_params) return bad("parameter count does not match its configuration");
    std::vector<uint8_t> tmp;
    const size_t pb = h->n_params * sizeof(float);
    if (!ck_read_dev(F.f, h->params, pb, tmp) || !ck_read_dev(F.f, h->adam_m, pb, tmp) ||
        !ck_read_dev(F.f, h->adam_v, pb, tmp))
        return bad("truncated parameters");
    uint32_t n_cells = 0;
    if (!ck_read(F.f, &n_cells, 4) || n_cells != h->n_cells) return bad("occupancy grid does not match");
    if (n_cells && (!ck_read_dev(F.f, h->occ_bits, n_cells / 8, tmp) ||
                    !ck_read_dev(F.f, h->occ_density, (size_t)n_cells * sizeof(float), tmp)))
        return bad("truncated occupancy grid");
    h->step = step;
    h->n_refresh = n_refresh;
    uint32_t n_kf = 0;
    if (!ck_read(F.f, &n_kf, 4)) return bad("truncated keyframe table");
    for (uint32_t i = 0; i < n_kf; ++i) {
        uint32_t rec[4];
        KfDesc d{};
        uint64_t bytes = 0;
        if (!ck_read(F.f, rec, sizeof(rec)) || !ck_read(F.f, d.c2w, sizeof(d.c2w)) ||
            !ck_read(F.f, d.K, sizeof(d.K)) || !ck_read(F.f, &bytes, 8))
            return bad("truncated keyframe table");
        const uint32_t W = rec[1], H = rec[2];
        if (W == 0 || H == 0 || (uint64_t)W * H > (1ull << 26) || bytes != (uint64_t)W * H * 2 * sizeof(float4))
            return bad("bad keyframe record");
        // the map owns each buffer as soon as it exists (map_destroy frees it on failure)
        Keyframe kf{rec[0], W, H, nullptr, (size_t)bytes};
        if (rec[3]) {
            if (dalloc(h, (void**)&kf.texels, kf.bytes)) return bad("no device memory for the keyframes");
            h->kfs.push_back(kf);
            if (!ck_read_dev(F.f, kf.texels, kf.bytes, tmp)) return bad("truncated keyframe images");
        } else {
            if (cudaMallocHost((void**)&kf.host, kf.bytes) != cudaSuccess) return bad("no host memory");
            h->kfs.push_back(kf);
            if (!ck_read(F.f, kf.host, kf.bytes)) return bad("truncated keyframe images");
        }
        d.W = W;
        d.H = H;
        d.texels = kf.texels;
        h->kf_desc.push_back(d);
    }
    if (n_kf) {
        const uint32_t cap = std::max<uint32_t>(64, n_kf * 2);
        if (dalloc(h, (void**)&h->d_kfs, cap * sizeof(KfDesc))) return bad("no device memory for the keyframes");
        h->d_kfs_cap = cap;
        for (uint32_t i = 0; i < n_kf; ++i) launch_set_kf_desc(h->d_kfs, i, h->kf_desc[i], nullptr);
        if (rebuild_active(h, nullptr) != MAP_OK) return bad(h->err);
    }
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bad(std::string("restore: ") + cudaGetErrorString(e));
    *out = h;
    return MAP_OK;
}

int map_get_pose_grads(map_handle h, float* dst, uint32_t n_kf, int mem_kind, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!dst || n_kf > h->kfs.size()) return fail(h, MAP_EINVAL, "n_kf exceeds the number of keyframes");
    if (!h->pose_valid) return fail(h, MAP_EINVAL, "no pose gradient: run map_step with MAP_STEP_POSE_GRAD");
    if (n_kf == 0) return MAP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind kind = mem_kind == MAP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    // slot rows of 8 floats -> rows of 6
    NM_CUDA(h, cudaMemcpy2DAsync(dst, 6 * sizeof(float), h->pose_g, 8 * sizeof(float), 6 * sizeof(float), n_kf,
                                 kind, s));
    if (mem_kind != MAP_MEM_DEVICE) NM_CUDA(h, cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_get_keyframe_ids(map_handle h, uint32_t* ids, uint32_t n) {
    if (!h) return MAP_EINVAL;
    const uint32_t k = (uint32_t)h->kfs.size();
    if (ids)
        for (uint32_t i = 0; i < std::min(n, k); ++i) ids[i] = h->kfs[i].id;
    return (int)k;
}

int map_set_keyframe_pose(map_handle h, uint32_t kf_id, const float c2w[12], void* stream) {
    if (!h) return MAP_EINVAL;
    if (!c2w) return fail(h, MAP_EINVAL, "null pose");
    for (size_t i = 0; i < h->kfs.size(); ++i) {
        if (h->kfs[i].id != kf_id) continue;
        std::memcpy(h->kf_desc[i].c2w, c2w, sizeof(h->kf_desc[i].c2w));
        launch_set_kf_desc(h->d_kfs, (uint32_t)i, h->kf_desc[i], (cudaStream_t)stream);
        return check_launch(h, "keyframe pose");
    }
    return fail(h, MAP_EINVAL, "unknown kf_id");
}

int map_render(map_handle h, const float c2w[12], const float K[4], uint32_t W, uint32_t H, float* out_rgb,
               float* out_depth, float* out_acc, int mem_kind, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!c2w || !K) return fail(h, MAP_EINVAL, "null camera");
    if (W == 0 || H == 0 || (uint64_t)W * H > (1u << 24)) return fail(h, MAP_EINVAL, "bad view size");
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const uint32_t n = W * H;
    // views larger than the work buffers (or than 2^18 rays) are rendered in chunks
    const uint32_t chunk = std::min<uint32_t>(n, std::max<uint32_t>(h->bufs.cap_rays, kRenderChunk));
    int rc = ensure_step_bufs(h, chunk);
    if (rc) return rc;
    const StepBufs& b = h->bufs;
    DevCfg dc = h->dc;
    dc.t_min = h->cfg.render_t_min;
    float* tmp = b.feat;  // host outputs: staged here (unused by a render), then copied
    NM_CUDA(h, cudaMemsetAsync(render_sample_counter(b), 0, 2 * sizeof(unsigned long long), s));
    // Early termination saves field work: with a threshold the field is evaluated for
    // the first kRenderFirst samples of every ray, then only for the rays whose
    // transmittance is still above it (the images equal a single pass's bit for bit).
    const bool two_pass = dc.t_min > 0.f;
    if (two_pass && h->render_off_cap < b.cap_rays) {
        cudaStreamSynchronize(s);
        dfree(h, h->render_off);
        h->render_off = nullptr;
        h->render_off_cap = 0;
        rc = dalloc(h, (void**)&h->render_off, (b.cap_rays + 1) * sizeof(uint32_t));
        if (rc) return rc;
        h->render_off_cap = b.cap_rays;
    }
    uint32_t* sel = reinterpret_cast<uint32_t*>(b.dsig_rgb);  // unused by a render: the selections
    const bool fp32 = h->cfg.precision == MAP_PREC_FP32, bf16 = h->cfg.precision == MAP_PREC_BF16;
    auto fwd_sel = [&](const uint32_t* n_sel) {
        if (fp32) launch_field_fwd_fp32_sel(h->dc, h->params, sel, n_sel, b, h->n_sm, s);
        else launch_field_fwd_tc_sel(h->dc, h->params, sel, n_sel, b, bf16, h->n_sm, s);
    };
    for (uint32_t p0 = 0; p0 < n; p0 += chunk) {
        const uint32_t cnt = std::min(chunk, n - p0);
        rc = phase(h, MAP_PH_RAYGEN, 1, s, [&] { launch_ray_gen_view(c2w, K, W, p0, cnt, b, s); });
        if (!two_pass) {
            if (!rc) rc = run_forward(h, cnt, false, s);
            if (!rc) rc = phase(h, MAP_PH_COMPOSITE, 1, s, [&] { launch_composite(dc, cnt, false, b, s); });
        } else {
            uint32_t* off = h->render_off;  // off[cnt]: the pass's total, read by the forward
            if (!rc) rc = phase(h, MAP_PH_MARCH, 5, s, [&] { launch_march(h->dc, h->occ_bits, cnt, b, s); });
            for (int pass = 1; pass <= 2 && !rc; ++pass) {
                rc = phase(h, MAP_PH_FIELD_FWD, pass == 1 ? 6 : 5, s, [&] {
                    launch_render_select(cnt, b.offsets, b.counts, pass == 1, kRenderFirst, off, b.block_sums, sel,
                                         render_eval_counter(b), s);
                    fwd_sel(off + cnt);
                });
                if (!rc)
                    rc = phase(h, MAP_PH_COMPOSITE, 1, s,
                               [&] { launch_composite_split(dc, cnt, pass, b.counts, b, s); });
            }
        }
        if (rc) return rc;
        h->last_rays = cnt;
        if (mem_kind == MAP_MEM_DEVICE) {
            rc = phase(h, MAP_PH_OUTPUT, 1, s, [&] {
                launch_write_render(b, cnt, out_rgb ? out_rgb + 3 * (size_t)p0 : nullptr,
                                    out_depth ? out_depth + p0 : nullptr, out_acc ? out_acc + p0 : nullptr,
                                    !two_pass, s);
            });
            if (rc) return rc;
            continue;
        }
        rc = phase(h, MAP_PH_OUTPUT, 1, s,
                   [&] { launch_write_render(b, cnt, tmp, tmp + 3 * (size_t)cnt, tmp + 4 * (size_t)cnt, !two_pass, s); });
        if (rc) return rc;
        if (out_rgb)
            NM_CUDA(h, cudaMemcpyAsync(out_rgb + 3 * (size_t)p0, tmp, 3 * (size_t)cnt * sizeof(float),
                                       cudaMemcpyDeviceToHost, s));
        if (out_depth)
            NM_CUDA(h, cudaMemcpyAsync(out_depth + p0, tmp + 3 * (size_t)cnt, cnt * sizeof(float),
                                       cudaMemcpyDeviceToHost, s));
        if (out_acc)
            NM_CUDA(h, cudaMemcpyAsync(out_acc + p0, tmp + 4 * (size_t)cnt, cnt * sizeof(float),
                                       cudaMemcpyDeviceToHost, s));
        NM_CUDA(h, cudaStreamSynchronize(s));  // the staging buffer is reused by the next chunk
    }
    return mem_kind == MAP_MEM_DEVICE ? MAP_OK : check_device_flags(h, s);
}

int map_render_group(const map_handle* maps, uint32_t n, const float* c2w, const float* K, const uint32_t* W,
                     const uint32_t* H, float* const* out_rgb, float* const* out_depth, void* stream) {
    if (!maps || n == 0 || !maps[0] || !c2w || !K || !W || !H) return MAP_EINVAL;
    map_scene* lead = maps[0];
    std::vector<GroupView> views[2];  // FP16, BF16
    uint32_t stride = 0;
    for (uint32_t i = 0; i < n; ++i) {
        GroupView gv{};
        if (!maps[i] || !scene_view(maps[i], &gv.scene)) return fail(lead, MAP_EINVAL, "null map in the group");
        if (gv.scene.precision == MAP_PREC_FP32)
            return fail(lead, MAP_EINVAL, "map_render_group: plain FP32 maps render with map_render");
        if (W[i] == 0 || H[i] == 0 || (uint64_t)W[i] * H[i] > (1u << 24))
            return fail(lead, MAP_EINVAL, "map_render_group: bad view size");
        std::memcpy(gv.c2w, c2w + 12 * (size_t)i, sizeof(gv.c2w));
        std::memcpy(gv.K, K + 4 * (size_t)i, sizeof(gv.K));
        gv.W = W[i];
        gv.H = H[i];
        gv.out_rgb = out_rgb ? out_rgb[i] : nullptr;
        gv.out_depth = out_depth ? out_depth[i] : nullptr;
        stride = std::max(stride, gv.scene.dc.max_samples);
        views[gv.scene.precision == MAP_PREC_BF16 ? 1 : 0].push_back(gv);
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (lead->group.row_stride < stride) {
        if (lead->group.items) {
            cudaStreamSynchronize(s);
            group_bufs_free(lead->group);
        }
        if (group_bufs_alloc(lead->group, kRenderChunk, std::max<uint32_t>(stride, 128)) != MAP_OK)
            return fail(lead, MAP_ENOMEM, "map_render_group: work buffers");
    }
    for (int k = 0; k < 2; ++k) {
        if (views[k].empty()) continue;
        const int rc = render_group(views[k].data(), (uint32_t)views[k].size(), k == 1, lead->group, lead->n_sm, s,
                                    &lead->launches);
        if (rc) return fail(lead, rc, "map_render_group: launch failed");
    }
    return MAP_OK;
}

int map_get_params(map_handle h, float* dst, size_t n, int mem_kind, void* stream) {
    if (!h || !dst) return MAP_EINVAL;
    if (n != h->n_params) return fail(h, MAP_EINVAL, "parameter count mismatch");
    return copy_out(h, dst, h->params, n * sizeof(float), mem_kind, (cudaStream_t)stream);
}

int map_set_params(map_handle h, const float* src, size_t n, int mem_kind, void* stream) {
    if (!h || !src) return MAP_EINVAL;
    if (n != h->n_params) return fail(h, MAP_EINVAL, "parameter count mismatch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_in(h, h->params, src, n * sizeof(float), mem_kind, s);
    if (rc) return rc;
    NM_CUDA(h, cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_get_grads(map_handle h, float* dst, size_t n, int mem_kind, void* stream) {
    if (!h || !dst) return MAP_EINVAL;
    if (n != h->n_params) return fail(h, MAP_EINVAL, "parameter count mismatch");
    return copy_out(h, dst, h->grads, n * sizeof(float), mem_kind, (cudaStream_t)stream);
}

int map_get_adam(map_handle h, float* m, float* v, size_t n, int mem_kind, void* stream) {
    if (!h) return MAP_EINVAL;
    if (n != h->n_params) return fail(h, MAP_EINVAL, "parameter count mismatch");
    int rc = MAP_OK;
    if (m) rc = copy_out(h, m, h->adam_m, n * sizeof(float), mem_kind, (cudaStream_t)stream);
    if (!rc && v) rc = copy_out(h, v, h->adam_v, n * sizeof(float), mem_kind, (cudaStream_t)stream);
    return rc;
}

int map_reset_adam(map_handle h, void* stream) {
    if (!h) return MAP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    NM_CUDA(h, cudaMemsetAsync(h->adam_m, 0, h->n_params * sizeof(float), s));
    NM_CUDA(h, cudaMemsetAsync(h->adam_v, 0, h->n_params * sizeof(float), s));
    NM_CUDA(h, cudaMemsetAsync(h->grads, 0, h->n_params * sizeof(float), s));
    h->step = 0;
    h->grads_dirty = false;
    return MAP_OK;
}

int map_set_occupancy(map_handle h, const uint8_t* bits, size_t n_bytes, int mem_kind, void* stream) {
    if (!h || !bits) return MAP_EINVAL;
    if (!h->occ_bits) return fail(h, MAP_EINVAL, "map has no occupancy grid");
    if (n_bytes != h->n_cells / 8) return fail(h, MAP_EINVAL, "occupancy size mismatch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_in(h, h->occ_bits, bits, n_bytes, mem_kind, s);
    if (rc) return rc;
    launch_occ_from_bits(h->occ_bits, h->occ_density, h->n_cells, s);
    rc = check_launch(h, "occupancy");
    if (rc) return rc;
    NM_CUDA(h, cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_set_occupancy_density(map_handle h, const float* density, size_t n, int mem_kind, void* stream) {
    if (!h || !density) return MAP_EINVAL;
    if (!h->occ_bits) return fail(h, MAP_EINVAL, "map has no occupancy grid");
    if (n != h->n_cells) return fail(h, MAP_EINVAL, "occupancy size mismatch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_in(h, h->occ_density, density, n * sizeof(float), mem_kind, s);
    if (rc) return rc;
    NM_CUDA(h, cudaStreamSynchronize(s));
    return MAP_OK;
}

int map_get_occupancy(map_handle h, uint8_t* bits, float* density, int mem_kind, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!h->occ_bits) return fail(h, MAP_EINVAL, "map has no occupancy grid");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = MAP_OK;
    if (bits) rc = copy_out(h, bits, h->occ_bits, h->n_cells / 8, mem_kind, s);
    if (!rc && density) rc = copy_out(h, density, h->occ_density, h->n_cells * sizeof(float), mem_kind, s);
    return rc;
}

int map_refresh_occupancy(map_handle h, void* stream) {
    if (!h) return MAP_EINVAL;
    if (!h->occ_bits) return fail(h, MAP_EINVAL, "map has no occupancy grid");
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = phase(h, MAP_PH_OCC, 1, s, [&] {
        launch_occ_refresh(h->dc, h->params, h->occ_density, h->occ_bits, h->cfg.seed, h->n_refresh,
                           h->cfg.occ_decay, h->cfg.occ_thresh, s);
    });
    h->n_refresh += 1;
    return rc;
}

static int last_total(map_scene* h, uint64_t* total) {
    *total = 0;
    if (!h->last_rays) return MAP_OK;
    uint32_t t = 0;
    int rc = copy_out(h, &t, h->bufs.offsets + h->last_rays, sizeof(uint32_t), MAP_MEM_HOST, h->last_stream);
    *total = t;
    return rc;
}

int map_get_samples(map_handle h, uint32_t* ray_id, float* t, size_t cap, void* stream) {
    if (!h) return MAP_EINVAL;
    (void)stream;
    uint64_t total;
    int rc = last_total(h, &total);
    if (rc) return rc;
    const size_t n = std::min<size_t>(cap, total);
    if (ray_id && n) rc = copy_out(h, ray_id, h->bufs.ray_id, n * sizeof(uint32_t), MAP_MEM_HOST, h->last_stream);
    if (!rc && t && n) rc = copy_out(h, t, h->bufs.t, n * sizeof(float), MAP_MEM_HOST, h->last_stream);
    return rc;
}

int map_get_ray_outputs(map_handle h, float* rgb, float* depth, float* acc, size_t n_rays, void* stream) {
    if (!h) return MAP_EINVAL;
    (void)stream;
    if (n_rays > h->last_rays) return fail(h, MAP_EINVAL, "more rays than the last step");
    cudaStream_t s = h->last_stream;
    const uint32_t cap = h->bufs.cap_rays;
    int rc = MAP_OK;
    for (int c = 0; c < 3 && rgb && !rc; ++c) {
        std::vector<float> tmp(n_rays);
        rc = copy_out(h, tmp.data(), h->bufs.ray_out + (size_t)c * cap, n_rays * sizeof(float), MAP_MEM_HOST, s);
        for (size_t i = 0; i < n_rays; ++i) rgb[3 * i + c] = tmp[i];
    }
    if (!rc && depth) rc = copy_out(h, depth, h->bufs.ray_out + 3 * (size_t)cap, n_rays * sizeof(float), MAP_MEM_HOST, s);
    if (!rc && acc) rc = copy_out(h, acc, h->bufs.ray_out + 4 * (size_t)cap, n_rays * sizeof(float), MAP_MEM_HOST, s);
    return rc;
}

int map_get_stats(map_handle h, map_stats* out) {
    if (!h || !out) return MAP_EINVAL;
    uint64_t total;
    int rc = last_total(h, &total);
    if (rc) return rc;
    out->step = h->step;
    out->n_samples = total;
    out->n_rays = h->last_rays;
    out->n_keyframes = (uint32_t)h->kfs.size();
    out->param_count = h->n_params;
    out->device_bytes = h->held;
    out->kernel_launches = h->launches;
    unsigned long long rs[2] = {0, 0};
    if (h->bufs.loss) rc = copy_out(h, rs, render_sample_counter(h->bufs), sizeof(rs), MAP_MEM_HOST, h->last_stream);
    out->render_samples = rs[0];
    out->render_evaluated = rs[1];
    return rc;
}

int map_profile_enable(map_handle h, int enable) {
    if (!h) return MAP_EINVAL;
    if (enable) {
        cudaDeviceSynchronize();
        prof_clear(h);
    }
    h->prof_on = enable != 0;
    return MAP_OK;
}

int map_profile_read(map_handle h, double* ms, uint64_t* count, uint64_t* launches) {
    if (!h) return MAP_EINVAL;
    double acc[MAP_PHASES] = {0};
    uint64_t cnt[MAP_PHASES] = {0}, lch[MAP_PHASES] = {0};
    for (auto& r : h->prof) {
        NM_CUDA(h, cudaEventSynchronize(r.b));
        float t = 0.f;
        NM_CUDA(h, cudaEventElapsedTime(&t, r.a, r.b));
        acc[r.phase] += t;
        cnt[r.phase] += 1;
        lch[r.phase] += r.launches;
    }
    for (int p = 0; p < MAP_PHASES; ++p) {
        if (ms) ms[p] = acc[p];
        if (count) count[p] = cnt[p];
        if (launches) launches[p] = lch[p];
    }
    return MAP_OK;
}

int map_set_wait_polls(map_handle h, uint32_t polls) {
    if (!h) return MAP_EINVAL;
    h->dc.wait_polls = polls;
    return MAP_OK;
}

size_t map_abi_config_size(void) { return sizeof(map_config); }

const char* map_last_error(map_handle h) {
    return h ? h->err.c_str() : g_global_error.c_str();
}

}  // extern "C"
