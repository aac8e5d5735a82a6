// server.cu - multi-scene serving loop around the mapping library (host code).
//
// The paper runs mapping as a thread that continuously optimises the map while the
// tracking thread hands over keyframes and the viewer asks for renders (Sec. 3.3).
// A server keeps several such maps resident on one GPU: each admitted scene has its
// own map (tables, occupancy, Adam state, keyframes) and its own CUDA stream.  Host
// threads submit keyframe, step and render requests at any time; one worker thread
// issues each scene's requests in submission order, keeps up to max_inflight of
// them on the GPU at once, and - when a scene's queue is empty and continuous mapping
// is on - fills the gap with mapping steps.  Requests that arrive while others are on
// the GPU join between them (continuous batching), and the scenes' streams overlap
// on the device.  The worker never waits on the GPU: it records an event after each
// request and retires requests whose events have completed.
//
// Latencies: every request carries submit / start / done times (seconds since the
// server was created).  A keyframe is done when the first mapping step issued after
// its insertion completes (the first step that can draw rays from it); without
// continuous mapping, when the insertion completes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nerfmap.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct PinnedBuf {
    float* p = nullptr;
    size_t floats = 0;
    bool busy = false;
};

struct Request {
    uint64_t id = 0;
    uint32_t scene = 0;
    uint32_t kind = 0;  // MAP_REQ_*
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = MAP_OK;
    uint64_t step_index = 0;   // step: its index; keyframe: the first step that covers it
    bool auto_step = false;    // issued by continuous mapping (not reported)
    cudaEvent_t ev = nullptr;
    int pin = -1;
    float* pin_ptr = nullptr;  // keyframe: rgb | depth | var; render: rgb | depth; step: loss
    uint32_t kf_id = 0, W = 0, H = 0, n_rays = 0;
    int depth_is_z = 0;
    float c2w[12], K[4];
    float* out_rgb = nullptr;
    float* out_depth = nullptr;
    float loss = 0.f;
    bool grouped = false;      // render issued in a grouped launch with other scenes' renders
};

struct Scene {
    bool active = false;
    map_handle h = nullptr;
    cudaStream_t stream = nullptr;
    bool mapping = false;
    bool has_keyframe = false;
    uint32_t precision = 0;           // MAP_PREC_* of the scene's MLP
    uint32_t step_rays = 0;
    uint64_t seed = 0;
    uint64_t steps_issued = 0, steps_done = 0;
    std::deque<Request*> fifo;        // submitted, not yet issued
    std::deque<Request*> inflight;    // issued, in issue order
    std::vector<Request*> kf_waiting; // inserted, waiting for a covering step
    float* d_render = nullptr;
    size_t d_render_floats = 0;
    size_t footprint = 0;
};

}  // namespace

struct map_server_s {
    map_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> incoming;
    std::vector<Request*> done;
    std::vector<Scene> scenes;
    std::deque<PinnedBuf> pins;  // deque: element addresses stay valid as it grows
    std::vector<cudaEvent_t> event_pool;
    uint64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::atomic<uint64_t> rays_done{0};
    // grouped renders (cfg.group_renders): lanes of a stream, work buffers and an
    // output arena each, taken in turn, so that batches issued one after the other
    // (lone renders of different scenes, the usual case) still overlap on the device
    struct GroupLane {
        cudaStream_t stream = nullptr;
        nm::GroupBufs gbufs{};
        float* arena = nullptr;
        size_t arena_floats = 0;
    };
    static constexpr int kGroupLanes = 2;
    GroupLane lanes[kGroupLanes];
    int next_lane = 0;
    int n_sm = 0;
    std::atomic<uint64_t> grouped_renders{0}, group_batches{0};

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    cudaEvent_t get_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }

    // a free pinned buffer of at least n floats (created on demand); mu held
    int get_pin(size_t n) {
        for (size_t i = 0; i < pins.size(); ++i)
            if (!pins[i].busy && pins[i].floats >= n) {
                pins[i].busy = true;
                return (int)i;
            }
        PinnedBuf b;
        if (cudaMallocHost((void**)&b.p, n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        b.floats = n;
        b.busy = true;
        pins.push_back(b);
        return (int)pins.size() - 1;
    }
    void release_pin(Request* r) {
        if (r->pin < 0) return;
        std::lock_guard<std::mutex> lock(mu);
        pins[r->pin].busy = false;
        r->pin = -1;
        r->pin_ptr = nullptr;
    }
};

namespace {

void complete(map_server_s* s, Request* r, int status) {
    r->t_done = s->now();
    r->status = status;
    if (r->auto_step) {
        delete r;
        return;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    s->done.push_back(r);
}

// Queues request r of scene sc on the GPU; false if it failed at issue.
bool issue_one(map_server_s* s, Scene& sc, Request* r) {
    r->t_start = s->now();
    int rc = MAP_OK;
    if (r->kind == MAP_REQ_KEYFRAME) {
        const size_t n = (size_t)r->W * r->H;
        const float* b = r->pin_ptr;
        rc = map_add_keyframe(sc.h, r->kf_id, r->c2w, r->K, r->W, r->H, b, b + 3 * n, b + 4 * n, r->depth_is_z,
                              MAP_MEM_HOST, sc.stream);
        if (rc == MAP_OK) {
            sc.has_keyframe = true;
            r->step_index = sc.steps_issued;
        }
    } else if (r->kind == MAP_REQ_STEP) {
        if (!sc.has_keyframe) rc = MAP_ENOKF;
        else {
            rc = map_step(sc.h, r->n_rays, sc.seed, 0, nullptr, sc.stream);
            if (rc == MAP_OK) {
                r->step_index = sc.steps_issued++;
                if (r->pin_ptr)
                    cudaMemcpyAsync(r->pin_ptr, map_loss_device(sc.h), sizeof(float), cudaMemcpyDeviceToHost,
                                    sc.stream);
            }
        }
    } else {  // render
        const size_t n = (size_t)r->W * r->H;
        if (sc.d_render_floats < 4 * n) {
            cudaStreamSynchronize(sc.stream);
            cudaFree(sc.d_render);
            sc.d_render = nullptr;
            sc.d_render_floats = 0;
            if (cudaMalloc((void**)&sc.d_render, 4 * n * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                rc = MAP_ENOMEM;
            } else {
                sc.d_render_floats = 4 * n;
            }
        }
        if (rc == MAP_OK)
            rc = map_render(sc.h, r->c2w, r->K, r->W, r->H, sc.d_render, sc.d_render + 3 * n, nullptr,
                            MAP_MEM_DEVICE, sc.stream);
        if (rc == MAP_OK)
            cudaMemcpyAsync(r->pin_ptr, sc.d_render, 4 * n * sizeof(float), cudaMemcpyDeviceToHost, sc.stream);
    }
    if (rc != MAP_OK) {
        s->release_pin(r);
        complete(s, r, rc);
        return false;
    }
    r->ev = s->get_event();
    cudaEventRecord(r->ev, sc.stream);
    sc.inflight.push_back(r);
    return true;
}

constexpr uint32_t kGroupCapRays = 1u << 18;
constexpr size_t kGroupMaxPixels = (size_t)1 << 22;  // pixels of one grouped batch

// Renders at the head of the tensor-core scenes' queues, issued together: one grouped
// render (shared launches over all their views) per MLP type on the next group lane's
// stream, which first waits for the work each scene has already queued; each scene's
// later work waits for the grouped render (it reads the scene's parameters).  Returns
// whether anything was issued.
bool issue_group(map_server_s* s) {
    bool any = false;
    for (uint32_t prec : {(uint32_t)MAP_PREC_FP16, (uint32_t)MAP_PREC_BF16}) {
        std::vector<std::pair<Scene*, Request*>> batch;
        std::vector<nm::GroupView> views;
        size_t pixels = 0;
        uint32_t stride = 0;
        const size_t cap = std::max<uint32_t>(1, s->cfg.max_inflight);
        for (auto& sc : s->scenes) {
            if (!sc.active) continue;
            nm::SceneView sv;
            if (!nm::scene_view(sc.h, &sv) || sv.precision != prec) continue;
            size_t taken = 0;
            // a view larger than the batch budget goes alone
            while (!sc.fifo.empty() && sc.fifo.front()->kind == MAP_REQ_RENDER && sc.inflight.size() + taken < cap &&
                   (batch.empty() || pixels + (size_t)sc.fifo.front()->W * sc.fifo.front()->H <= kGroupMaxPixels)) {
                Request* r = sc.fifo.front();
                sc.fifo.pop_front();
                batch.emplace_back(&sc, r);
                nm::GroupView gv{};
                gv.scene = sv;
                std::memcpy(gv.c2w, r->c2w, sizeof(gv.c2w));
                std::memcpy(gv.K, r->K, sizeof(gv.K));
                gv.W = r->W;
                gv.H = r->H;
                views.push_back(gv);
                pixels += (size_t)r->W * r->H;
                stride = std::max(stride, sv.dc.max_samples);
                ++taken;
            }
        }
        if (batch.empty()) continue;
        any = true;
        map_server_s::GroupLane& L = s->lanes[s->next_lane];
        s->next_lane = (s->next_lane + 1) % map_server_s::kGroupLanes;
        int rc = MAP_OK;
        if (!L.stream && cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess)
            rc = MAP_ECUDA;
        if (rc == MAP_OK && L.gbufs.row_stride < stride) {
            if (L.gbufs.items) {
                cudaStreamSynchronize(L.stream);
                nm::group_bufs_free(L.gbufs);
            }
            rc = nm::group_bufs_alloc(L.gbufs, kGroupCapRays, std::max<uint32_t>(stride, 128));
        }
        if (rc == MAP_OK && L.arena_floats < 4 * pixels) {
            cudaStreamSynchronize(L.stream);
            cudaFree(L.arena);
            L.arena = nullptr;
            L.arena_floats = 0;
            if (cudaMalloc((void**)&L.arena, 4 * pixels * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                rc = MAP_ENOMEM;
            } else {
                L.arena_floats = 4 * pixels;
            }
        }
        std::vector<Scene*> scenes;
        for (auto& br : batch)
            if (std::find(scenes.begin(), scenes.end(), br.first) == scenes.end()) scenes.push_back(br.first);
        if (rc == MAP_OK) {
            for (Scene* sc : scenes) {  // the render sees each scene as its queue left it
                cudaEvent_t e = s->get_event();
                cudaEventRecord(e, sc->stream);
                cudaStreamWaitEvent(L.stream, e, 0);
                s->event_pool.push_back(e);
            }
            size_t off = 0;
            for (size_t k = 0; k < views.size(); ++k) {
                const size_t n = (size_t)views[k].W * views[k].H;
                views[k].out_rgb = L.arena + off;
                views[k].out_depth = L.arena + off + 3 * n;
                off += 4 * n;
            }
            const double t = s->now();
            rc = nm::render_group(views.data(), (uint32_t)views.size(), prec == MAP_PREC_BF16, L.gbufs, s->n_sm,
                                  L.stream, nullptr);
            for (size_t k = 0; k < batch.size() && rc == MAP_OK; ++k) {
                Request* r = batch[k].second;
                const size_t n = (size_t)r->W * r->H;
                cudaMemcpyAsync(r->pin_ptr, views[k].out_rgb, 4 * n * sizeof(float), cudaMemcpyDeviceToHost,
                                L.stream);
                r->t_start = t;
                r->grouped = true;
            }
        }
        if (L.stream) {
            // the scenes' later steps wait for the grouped render (whatever of it was
            // queued, also when a launch failed part way: it still reads the parameters)
            cudaEvent_t done = s->get_event();
            cudaEventRecord(done, L.stream);
            for (Scene* sc : scenes) cudaStreamWaitEvent(sc->stream, done, 0);
            s->event_pool.push_back(done);
        }
        if (rc != MAP_OK) {
            for (auto& br : batch) {
                s->release_pin(br.second);
                complete(s, br.second, rc);
            }
            continue;
        }
        for (auto& br : batch) {
            Request* r = br.second;
            r->ev = s->get_event();
            cudaEventRecord(r->ev, L.stream);
            br.first->inflight.push_back(r);
        }
        s->grouped_renders += batch.size();
        s->group_batches += 1;
    }
    return any;
}

bool issue(map_server_s* s, Scene& sc) {
    bool any = false;
    const size_t cap = std::max<uint32_t>(1, s->cfg.max_inflight);
    while (!sc.fifo.empty() && sc.inflight.size() < cap) {
        Request* r = sc.fifo.front();
        // a tensor-core scene's render waits at the head of its queue for the next
        // grouped render (issue_group), which keeps the scene's request order
        if (s->cfg.group_renders && r->kind == MAP_REQ_RENDER && sc.precision != MAP_PREC_FP32) break;
        sc.fifo.pop_front();
        issue_one(s, sc, r);
        any = true;
    }
    if (sc.fifo.empty() && sc.mapping && sc.has_keyframe && sc.inflight.size() < cap) {
        Request* r = new Request();
        r->kind = MAP_REQ_STEP;
        r->scene = (uint32_t)(&sc - &s->scenes[0]);
        r->auto_step = true;
        r->n_rays = sc.step_rays;
        r->t_submit = s->now();
        issue_one(s, sc, r);
        any = true;
    }
    return any;
}

bool retire(map_server_s* s, Scene& sc) {
    bool any = false;
    while (!sc.inflight.empty() && cudaEventQuery(sc.inflight.front()->ev) == cudaSuccess) {
        Request* r = sc.inflight.front();
        sc.inflight.pop_front();
        s->event_pool.push_back(r->ev);
        r->ev = nullptr;
        any = true;
        if (r->kind == MAP_REQ_STEP) {
            sc.steps_done = r->step_index + 1;
            s->rays_done += r->n_rays;
            if (r->pin_ptr) r->loss = *r->pin_ptr;
            s->release_pin(r);
            complete(s, r, MAP_OK);
        } else if (r->kind == MAP_REQ_KEYFRAME) {
            s->release_pin(r);  // the texels are on the device
            if (sc.mapping) sc.kf_waiting.push_back(r);
            else complete(s, r, MAP_OK);
        } else {
            complete(s, r, MAP_OK);  // map_server_poll copies the pinned render out
        }
    }
    for (size_t i = 0; i < sc.kf_waiting.size();) {
        Request* r = sc.kf_waiting[i];
        if (sc.steps_done > r->step_index || !sc.mapping) {
            sc.kf_waiting.erase(sc.kf_waiting.begin() + i);
            complete(s, r, MAP_OK);
            any = true;
        } else {
            ++i;
        }
    }
    return any;
}

void worker_main(map_server_s* s) {
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            while (!s->incoming.empty()) {
                Request* r = s->incoming.front();
                s->incoming.pop_front();
                s->scenes[r->scene].fifo.push_back(r);
            }
        }
        bool progress = false;
        for (auto& sc : s->scenes)
            if (sc.active) progress |= retire(s, sc);
        if (s->cfg.group_renders) progress |= issue_group(s);
        for (auto& sc : s->scenes)
            if (sc.active) progress |= issue(s, sc);
        if (!progress) {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->incoming.empty()) s->cv.wait_for(lock, std::chrono::microseconds(50));
        }
    }
}

size_t scene_footprint(const map_config* c, uint32_t step_rays, size_t kf_reserve) {
    const size_t P = (size_t)c->n_levels * ((size_t)1 << c->log2_table) * 2 + 9408;
    const size_t cells = (size_t)c->occ_res * c->occ_res * c->occ_res;
    const size_t rays = std::max<size_t>(step_rays, (size_t)1 << 18);
    const size_t samples = rays * c->max_samples;
    return 16 * P + cells * 4 + cells / 8 + rays * 80 + samples * 168 + kf_reserve + (64u << 20);
}

Request* new_request(map_server_s* s, uint32_t scene, uint32_t kind) {
    Request* r = new Request();
    r->scene = scene;
    r->kind = kind;
    r->t_submit = s->now();
    return r;
}

int enqueue(map_server_s* s, Request* r, uint64_t* req_id) {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    if (req_id) *req_id = r->id;
    s->incoming.push_back(r);
    s->cv.notify_all();
    return MAP_OK;
}

bool scene_ok(map_server_s* s, uint32_t scene) {
    std::lock_guard<std::mutex> lock(s->mu);
    return scene < s->scenes.size() && s->scenes[scene].active;
}

}  // namespace

extern "C" {

int map_server_create(const map_server_config* cfg, map_server* out) {
    if (!cfg || !out || cfg->max_scenes == 0 || cfg->max_scenes > 64 || cfg->step_rays == 0 ||
        cfg->step_rays > (1u << 24))
        return MAP_EINVAL;
    map_server_s* s = new map_server_s();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
    s->t0 = Clock::now();
    s->scenes.resize(cfg->max_scenes);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return MAP_OK;
}

int map_server_destroy(map_server s) {
    if (!s) return MAP_EINVAL;
    s->stop = true;
    s->cv.notify_all();
    s->worker.join();
    cudaDeviceSynchronize();
    for (auto& sc : s->scenes) {
        if (!sc.active) continue;
        for (Request* r : sc.fifo) delete r;
        for (Request* r : sc.inflight) {
            if (r->ev) cudaEventDestroy(r->ev);
            delete r;
        }
        for (Request* r : sc.kf_waiting) delete r;
        map_destroy(sc.h);
        cudaStreamDestroy(sc.stream);
        cudaFree(sc.d_render);
    }
    for (auto& L : s->lanes) {
        if (L.gbufs.items) nm::group_bufs_free(L.gbufs);
        cudaFree(L.arena);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    for (Request* r : s->incoming) delete r;
    for (Request* r : s->done) delete r;
    for (auto& b : s->pins) cudaFreeHost(b.p);
    for (auto e : s->event_pool) cudaEventDestroy(e);
    delete s;
    return MAP_OK;
}

int map_server_add_scene(map_server s, const map_config* cfg, int continuous_mapping, uint32_t* scene_id) {
    if (!s || !cfg || !scene_id) return MAP_EINVAL;
    const size_t need = scene_footprint(cfg, s->cfg.step_rays, s->cfg.kf_reserve_bytes);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MAP_ECUDA;
    if (free_b < need + s->cfg.hbm_reserve_bytes) return MAP_ENOMEM;  // not admitted now: retry later
    uint32_t slot = UINT32_MAX;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (uint32_t i = 0; i < s->scenes.size(); ++i)
            if (!s->scenes[i].active) {
                slot = i;
                break;
            }
    }
    if (slot == UINT32_MAX) return MAP_ENOMEM;  // every slot taken
    map_handle h = nullptr;
    int rc = map_create(cfg, need, &h);
    if (rc != MAP_OK) return rc;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        map_destroy(h);
        return MAP_ECUDA;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    Scene& sc = s->scenes[slot];
    sc = Scene();
    sc.h = h;
    sc.stream = st;
    sc.step_rays = s->cfg.step_rays;
    sc.seed = cfg->seed;  // the scene's own draws, whatever slot it lands in
    sc.mapping = continuous_mapping != 0;
    sc.precision = cfg->precision;
    sc.footprint = need;
    sc.active = true;
    *scene_id = slot;
    return MAP_OK;
}

int map_server_scene_handle(map_server s, uint32_t scene, map_handle* out) {
    if (!s || !out || !scene_ok(s, scene)) return MAP_EINVAL;
    *out = s->scenes[scene].h;
    return MAP_OK;
}

int map_server_submit_keyframe(map_server s, uint32_t scene, uint32_t kf_id, const float c2w[12],
                               const float K[4], uint32_t W, uint32_t H, const float* rgb, const float* depth,
                               const float* depth_var, int depth_is_z, uint64_t* req_id) {
    if (!s || !c2w || !K || !rgb || !depth || !depth_var || W == 0 || H == 0 || (uint64_t)W * H > (1ull << 26))
        return MAP_EINVAL;
    if (!scene_ok(s, scene)) return MAP_EINVAL;
    const size_t n = (size_t)W * H;
    Request* r = new_request(s, scene, MAP_REQ_KEYFRAME);
    r->kf_id = kf_id;
    r->W = W;
    r->H = H;
    r->depth_is_z = depth_is_z;
    std::memcpy(r->c2w, c2w, sizeof(r->c2w));
    std::memcpy(r->K, K, sizeof(r->K));
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->pin = s->get_pin(5 * n);
        if (r->pin >= 0) r->pin_ptr = s->pins[r->pin].p;
    }
    if (r->pin < 0) {
        delete r;
        return MAP_ENOMEM;
    }
    std::memcpy(r->pin_ptr, rgb, 3 * n * sizeof(float));
    std::memcpy(r->pin_ptr + 3 * n, depth, n * sizeof(float));
    std::memcpy(r->pin_ptr + 4 * n, depth_var, n * sizeof(float));
    return enqueue(s, r, req_id);
}

int map_server_submit_step(map_server s, uint32_t scene, uint32_t n_rays, int want_loss, uint64_t* req_id) {
    if (!s || n_rays == 0 || n_rays > (1u << 24) || !scene_ok(s, scene)) return MAP_EINVAL;
    Request* r = new_request(s, scene, MAP_REQ_STEP);
    r->n_rays = n_rays;
    if (want_loss) {
        std::lock_guard<std::mutex> lock(s->mu);
        r->pin = s->get_pin(1);
        if (r->pin < 0) {
            delete r;
            return MAP_ENOMEM;
        }
        r->pin_ptr = s->pins[r->pin].p;
    }
    return enqueue(s, r, req_id);
}

int map_server_submit_render(map_server s, uint32_t scene, const float c2w[12], const float K[4], uint32_t W,
                             uint32_t H, float* out_rgb, float* out_depth, uint64_t* req_id) {
    if (!s || !c2w || !K || W == 0 || H == 0 || (uint64_t)W * H > (1u << 24)) return MAP_EINVAL;
    if (!scene_ok(s, scene)) return MAP_EINVAL;
    Request* r = new_request(s, scene, MAP_REQ_RENDER);
    r->W = W;
    r->H = H;
    r->out_rgb = out_rgb;
    r->out_depth = out_depth;
    std::memcpy(r->c2w, c2w, sizeof(r->c2w));
    std::memcpy(r->K, K, sizeof(r->K));
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->pin = s->get_pin(4 * (size_t)W * H);
        if (r->pin >= 0) r->pin_ptr = s->pins[r->pin].p;
    }
    if (r->pin < 0) {
        delete r;
        return MAP_ENOMEM;
    }
    return enqueue(s, r, req_id);
}

int map_server_poll(map_server s, map_completion* out, uint32_t cap, uint32_t* n_out) {
    if (!s || (!out && cap) || !n_out) return MAP_EINVAL;
    std::vector<Request*> take;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const size_t k = std::min<size_t>(cap, s->done.size());
        take.assign(s->done.begin(), s->done.begin() + k);
        s->done.erase(s->done.begin(), s->done.begin() + k);
    }
    for (size_t i = 0; i < take.size(); ++i) {
        Request* r = take[i];
        if (r->kind == MAP_REQ_RENDER && r->status == MAP_OK && r->pin_ptr) {
            const size_t n = (size_t)r->W * r->H;
            if (r->out_rgb) std::memcpy(r->out_rgb, r->pin_ptr, 3 * n * sizeof(float));
            if (r->out_depth) std::memcpy(r->out_depth, r->pin_ptr + 3 * n, n * sizeof(float));
        }
        s->release_pin(r);
        map_completion& c = out[i];
        c.req_id = r->id;
        c.scene = r->scene;
        c.kind = r->kind;
        c.status = r->status;
        c.step_index = r->step_index;
        c.loss = r->loss;
        c.t_submit = r->t_submit;
        c.t_start = r->t_start;
        c.t_done = r->t_done;
        delete r;
    }
    *n_out = (uint32_t)take.size();
    return MAP_OK;
}

int map_server_get_stats(map_server s, map_server_stats* out) {
    if (!s || !out) return MAP_EINVAL;
    std::memset(out, 0, sizeof(*out));
    std::lock_guard<std::mutex> lock(s->mu);
    out->t_now = s->now();
    out->rays_done = s->rays_done.load();
    for (const auto& sc : s->scenes) {
        if (!sc.active) continue;
        out->n_scenes += 1;
        out->steps_done += sc.steps_done;
        out->device_bytes += sc.footprint;
    }
    out->pending = (uint32_t)(s->incoming.size() + s->done.size());
    out->grouped_renders = s->grouped_renders.load();
    out->group_batches = s->group_batches.load();
    return MAP_OK;
}

}  // extern "C"
