// Serving: resident scenes, admission by device memory, continuous batching of camera
// requests of mixed resolutions (declared in trisplat.h, tri_serve_*).
//
// A dispatcher thread owns `slots` pipelines, each with its own context, stream and
// completion event. Whenever a slot is free it takes the scene of the oldest queued
// request and up to max_batch queued requests of that scene (any resolutions) and
// launches one batched preprocess, one sort and one persistent render over all
// (request, tile) work items. Requests that arrive while batches run wait in the queue
// and join the next free slot, so work of different batches overlaps on the device.
// Each slot replays a CUDA graph per batch composition (scene and per-view
// resolutions), after rewriting its context's pinned camera and output tables; the
// first batch of a composition runs eagerly and is then captured. The batch also
// copies the context's counters back, so an overflowing pair list is detected when the
// batch completes and the batch re-runs with a larger list.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "ctx.h"

using namespace ts;

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() { return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count(); }

struct SrvScene {
    void *mem = nullptr;
    tri_scene desc{};
    size_t bytes = 0;
    int inflight = 0;
    bool removing = false;
};

struct Req {
    uint64_t ticket;
    int32_t scene;
    tri_camera cam;
    float *out;
    double t_submit;
    double deadline;   // <= 0: none
    double t_launch;
};

struct Slot {
    tri_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Ctl *h_ctl = nullptr;              // pinned copy of the context's counters after a batch
    std::vector<Req> batch;
    bool busy = false;
    int32_t scene = -1;
    int attempts = 0;
    std::map<std::vector<int>, cudaGraphExec_t> graphs;
    std::map<std::vector<int>, int> eager_runs;   // eager runs per composition (capture policy)
    uint64_t graph_gen = 0;             // context realloc generation the graphs were captured at
    int64_t graph_cap = 0;              // pair capacity the graphs were captured at
};

std::vector<int> graph_key(int32_t scene, const std::vector<Req> &reqs) {
    std::vector<int> k;
    k.reserve(1 + 2 * reqs.size());
    k.push_back(scene);
    for (const Req &r : reqs) {
        k.push_back(r.cam.width);
        k.push_back(r.cam.height);
    }
    return k;
}

// What one launch did, folded into the server's counters under its lock.
struct LaunchInfo {
    bool replayed = false, captured = false;
    double eager_ms = 0.0, capture_ms = 0.0;
    uint64_t reallocs = 0;
};

}  // namespace

struct tri_serve {
    tri_serve_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Req> queue;
    std::map<int32_t, SrvScene> scenes;
    int32_t next_scene = 0;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::thread th;
    bool stop = false;
    std::deque<std::pair<uint64_t, int32_t>> done_q;
    std::unordered_map<uint64_t, int32_t> done_map;
    std::vector<double> lat_ms, queue_ms;
    std::vector<int32_t> drop_requests;   // scenes whose graphs the dispatcher must drop
    uint64_t drops_done = 0;              // drop requests served so far
    uint64_t submitted = 0, completed = 0, rejected = 0, timed_out = 0, batches = 0, views = 0;
    uint64_t graph_replays = 0, graph_captures = 0, eager_batches = 0, reruns = 0, reallocs = 0;
    double eager_ms = 0.0, capture_ms = 0.0;
    double t_first = -1.0, t_last = 0.0;
    size_t bytes_resident = 0;
};

namespace {

size_t slot_bytes(const Slot &s) {
    size_t b = 0;
    for (TsDevBuf *d : s.ctx->all()) b += d->bytes;
    return b;
}

// Drop the slot's graphs and stamp the cache with the context's current buffers.
// Only the dispatcher thread calls this, never while the slot's work is in flight.
void drop_graphs(Slot &s) {
    for (auto &kv : s.graphs) cudaGraphExecDestroy(kv.second);
    s.graphs.clear();
    s.graph_gen = s.ctx->realloc_gen;
    s.graph_cap = s.ctx->pair_cap;
}

void drop_scene_graphs(Slot &s, int32_t scene) {
    for (auto it = s.graphs.begin(); it != s.graphs.end();) {
        if (it->first[0] == scene) {
            cudaGraphExecDestroy(it->second);
            it = s.graphs.erase(it);
        } else {
            ++it;
        }
    }
}

void finish(tri_serve *S, const Req &r, int32_t status, double t) {
    S->done_q.emplace_back(r.ticket, status);
    S->done_map[r.ticket] = status;
    if (status == TRI_OK) {
        S->lat_ms.push_back(t - r.t_submit);
        S->queue_ms.push_back(r.t_launch - r.t_submit);
        ++S->completed;
        S->t_last = std::max(S->t_last, t);
    } else if (status == TRI_ERR_TIMEOUT) {
        ++S->timed_out;
    } else {
        ++S->rejected;
    }
}

// The three pipeline calls of one batch (eager or under capture).
tri_status batch_calls(Slot &sl, const tri_scene &sc, const std::vector<tri_camera> &cams,
                       const std::vector<float *> &outs) {
    tri_status st = tri_preprocess(sl.ctx, &sc, cams.data(), (int)cams.size(), sl.stream);
    if (st != TRI_OK) return st;
    if ((st = tri_bin_sort(sl.ctx, nullptr, sl.stream)) != TRI_OK) return st;
    return tri_render_fwd(sl.ctx, outs.data(), nullptr, nullptr, sl.stream);
}

// Launch the slot's batch: replay its composition's graph, or run eagerly and capture.
tri_status launch(tri_serve *S, Slot &sl, const tri_scene &sc, LaunchInfo &li) {
    const uint64_t gen0 = sl.ctx->realloc_gen;
    struct Count {
        const tri_ctx *c;
        uint64_t g0;
        LaunchInfo &li;
        ~Count() { li.reallocs += c->realloc_gen - g0; }
    } count{sl.ctx, gen0, li};
    std::vector<tri_camera> cams;
    std::vector<float *> outs;
    for (const Req &r : sl.batch) {
        cams.push_back(r.cam);
        outs.push_back(r.out);
    }
    if (sl.graph_gen != sl.ctx->realloc_gen || sl.graph_cap != sl.ctx->pair_cap) drop_graphs(sl);
    const std::vector<int> key = graph_key(sl.scene, sl.batch);
    auto it = S->opts.use_graphs ? sl.graphs.find(key) : sl.graphs.end();
    if (it != sl.graphs.end()) {
        std::vector<ViewDev> views;
        int tiles = 0;
        int64_t pix = 0;
        tri_status st = ts_build_views(sl.ctx, cams.data(), (int)cams.size(), views, tiles, pix);
        if (st != TRI_OK) return st;
        memcpy(sl.ctx->h_views, views.data(), sizeof(ViewDev) * views.size());
        for (size_t v = 0; v < outs.size(); ++v) sl.ctx->h_outs_fwd[v] = ViewOut{outs[v], nullptr};
        if (cudaGraphLaunch(it->second, sl.stream) != cudaSuccess) {
            cudaGetLastError();
            return TRI_ERR_CUDA;
        }
        li.replayed = true;
    } else {
        const double t0 = now_ms();
        tri_status st = batch_calls(sl, sc, cams, outs);
        const double t1 = now_ms();
        li.eager_ms += t1 - t0;
        if (st != TRI_OK) return st;
        // the eager run may have grown a buffer: every graph captured before it would
        // replay into freed memory
        if (sl.graph_gen != sl.ctx->realloc_gen || sl.graph_cap != sl.ctx->pair_cap) drop_graphs(sl);
        if (sl.eager_runs.size() > 4096) sl.eager_runs.clear();
        const int runs = S->opts.use_graphs ? ++sl.eager_runs[key] : 0;
        if (S->opts.use_graphs && sl.ctx->pair_cap > 0 && runs >= std::max(1, S->opts.graph_after)) {
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                tri_status cs = batch_calls(sl, sc, cams, outs);
                ok = cudaStreamEndCapture(sl.stream, &g) == cudaSuccess && cs == TRI_OK;
            }
            cudaGraphExec_t ex = nullptr;
            // capture allocates nothing, so the generation checked above still holds
            if (ok && sl.graph_gen == sl.ctx->realloc_gen && sl.graph_cap == sl.ctx->pair_cap &&
                cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                if (sl.graphs.size() >= 64) drop_graphs(sl);
                sl.graphs[key] = ex;
            }
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            li.captured = ex != nullptr;
            li.capture_ms += now_ms() - t1;
        }
    }
    if (cudaMemcpyAsync(sl.h_ctl, sl.ctx->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaEventRecord(sl.done, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_CUDA;
    }
    return TRI_OK;
}

void fold(tri_serve *S, const LaunchInfo &li) {
    S->graph_replays += li.replayed;
    S->graph_captures += li.captured;
    S->eager_batches += !li.replayed;
    S->reallocs += li.reallocs;
    S->eager_ms += li.eager_ms;
    S->capture_ms += li.capture_ms;
}

// Take the next batch for slot `sl` from the queue (lock held). Returns false if none.
bool take_batch(tri_serve *S, Slot &sl, double t) {
    // expire requests whose deadline has passed
    for (auto q = S->queue.begin(); q != S->queue.end();) {
        if (q->deadline > 0 && t > q->deadline) {
            finish(S, *q, TRI_ERR_TIMEOUT, t);
            q = S->queue.erase(q);
        } else {
            ++q;
        }
    }
    if (S->queue.empty()) return false;
    const int32_t sid = S->queue.front().scene;
    auto sc = S->scenes.find(sid);
    if (sc == S->scenes.end()) {
        finish(S, S->queue.front(), TRI_ERR_INVALID_ARG, t);
        S->queue.pop_front();
        return false;
    }
    std::vector<Req> reqs;
    for (auto q = S->queue.begin(); q != S->queue.end() && (int)reqs.size() < S->opts.max_batch;) {
        if (q->scene == sid) {
            reqs.push_back(*q);
            q = S->queue.erase(q);
        } else {
            ++q;
        }
    }
    // admission by memory: shrink the batch until its workspace fits the budget
    size_t others = S->bytes_resident;
    for (const Slot &o : S->slots)
        if (&o != &sl) others += slot_bytes(o);
    while (!reqs.empty()) {
        std::vector<tri_camera> cams;
        for (const Req &r : reqs) cams.push_back(r.cam);
        size_t need = 0;
        tri_workspace_query(&sc->second.desc, cams.data(), (int)cams.size(),
                            sl.ctx->pair_cap > 0 ? sl.ctx->pair_cap : 0, &need);
        need = std::max(need, slot_bytes(sl));
        if (others + need <= S->opts.mem_budget_bytes) break;
        S->queue.push_front(reqs.back());
        reqs.pop_back();
    }
    if (reqs.empty()) {
        bool any_busy = false;
        for (const Slot &o : S->slots) any_busy |= o.busy;
        if (!any_busy) {   // even a single request can never fit
            finish(S, S->queue.front(), TRI_ERR_CAPACITY, t);
            S->queue.pop_front();
        }
        return false;
    }
    // order by resolution, so that the graph cache keys on the multiset of resolutions
    std::sort(reqs.begin(), reqs.end(), [](const Req &a, const Req &b) {
        if (a.cam.width != b.cam.width) return a.cam.width < b.cam.width;
        if (a.cam.height != b.cam.height) return a.cam.height < b.cam.height;
        return a.ticket < b.ticket;
    });
    for (Req &r : reqs) r.t_launch = t;
    sl.batch = std::move(reqs);
    sl.scene = sid;
    sl.attempts = 0;
    sc->second.inflight += (int)sl.batch.size();
    return true;
}

void dispatcher(tri_serve *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool any_busy = false;
        if (!S->drop_requests.empty()) {
            for (int32_t sid : S->drop_requests)
                for (Slot &sl : S->slots) drop_scene_graphs(sl, sid);
            S->drops_done += S->drop_requests.size();
            S->drop_requests.clear();
            S->done_cv.notify_all();
        }
        const double t = now_ms();
        // 1. completions
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            if (cudaEventQuery(sl.done) != cudaSuccess) {
                cudaGetLastError();
                any_busy = true;
                continue;
            }
            SrvScene &sc = S->scenes[sl.scene];
            const Ctl &h = *sl.h_ctl;
            if (h.overflow && sl.attempts < 3) {
                // pair list too small: grow it and run the batch again
                ++sl.attempts;
                const int64_t want = (int64_t)h.n_pairs + (int64_t)h.n_pairs / 4 + 1024;
                const tri_scene desc = sc.desc;
                LaunchInfo li;
                lk.unlock();
                const uint64_t g0 = sl.ctx->realloc_gen;
                tri_status st = tri_reserve(sl.ctx, want);
                li.reallocs += sl.ctx->realloc_gen - g0;
                if (st == TRI_OK) st = launch(S, sl, desc, li);
                lk.lock();
                fold(S, li);
                ++S->reruns;
                if (st == TRI_OK) {
                    any_busy = true;
                    continue;
                }
            }
            const int32_t status = h.error ? ((h.error & ERR_SPIN) ? TRI_ERR_TIMEOUT : TRI_ERR_DEVICE_CHECK)
                                           : (h.overflow ? TRI_ERR_CAPACITY : TRI_OK);
            const double tc = now_ms();
            for (const Req &r : sl.batch) finish(S, r, status, tc);
            sc.inflight -= (int)sl.batch.size();
            ++S->batches;
            S->views += sl.batch.size();
            sl.batch.clear();
            sl.busy = false;
            S->done_cv.notify_all();
        }
        // 2. launches
        for (Slot &sl : S->slots) {
            if (sl.busy || S->queue.empty()) continue;
            if (S->opts.batch_window_us > 0 && (int)S->queue.size() < S->opts.max_batch &&
                now_ms() - S->queue.front().t_submit < S->opts.batch_window_us * 1e-3)
                break;
            if (!take_batch(S, sl, now_ms())) {
                S->done_cv.notify_all();
                continue;
            }
            sl.busy = true;
            any_busy = true;
            const tri_scene desc = S->scenes[sl.scene].desc;
            LaunchInfo li;
            lk.unlock();
            tri_status st = launch(S, sl, desc, li);
            lk.lock();
            fold(S, li);
            if (st != TRI_OK) {
                const double tc = now_ms();
                for (const Req &r : sl.batch) finish(S, r, st, tc);
                S->scenes[sl.scene].inflight -= (int)sl.batch.size();
                sl.batch.clear();
                sl.busy = false;
                S->done_cv.notify_all();
            }
        }
        if (S->stop && S->queue.empty() && !any_busy) break;
        if (any_busy || !S->queue.empty()) {
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

tri_status tri_serve_create(tri_serve **out, const tri_serve_opts *opts, int device) {
    if (!out || !opts) return TRI_ERR_INVALID_ARG;
    *out = nullptr;
    if (opts->max_batch < 1 || opts->max_batch > MAX_VIEWS || opts->slots < 1 || opts->slots > 16 ||
        opts->max_width < 1 || opts->max_height < 1 || opts->max_width > 65535 || opts->max_height > 65535)
        return TRI_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_CUDA;
    }
    tri_serve *S = new tri_serve();
    S->opts = *opts;
    S->device = device;
    if (S->opts.mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->opts.mem_budget_bytes = fr / 10 * 8;
    }
    S->slots.resize(opts->slots);
    // serving streams take the device's highest priority: their blocks are scheduled
    // ahead of pending blocks of other work (a training job) sharing the GPU
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        cudaGetLastError();
        prio_hi = 0;
    }
    for (Slot &sl : S->slots) {
        if (tri_ctx_create(&sl.ctx, device) != TRI_OK ||
            cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&sl.h_ctl, sizeof(Ctl)) != cudaSuccess) {
            cudaGetLastError();
            tri_serve_destroy(S);
            if (prev >= 0) cudaSetDevice(prev);
            return TRI_ERR_CUDA;
        }
        memset(sl.h_ctl, 0, sizeof(Ctl));
    }
    S->th = std::thread(dispatcher, S);
    if (prev >= 0) cudaSetDevice(prev);
    *out = S;
    return TRI_OK;
}

tri_status tri_serve_add_scene(tri_serve *S, const tri_scene *scene, int32_t *scene_id) {
    if (!S || !scene || !scene_id || scene->n <= 0 || scene->sh_degree < 0 || scene->sh_degree > 3 ||
        !scene->verts || !scene->sh || !scene->opacity || !scene->sigma)
        return TRI_ERR_INVALID_ARG;
    const size_t n = (size_t)scene->n, nk = (size_t)(scene->sh_degree + 1) * (scene->sh_degree + 1);
    const size_t bv = (n * 9 * 4 + 255) & ~(size_t)255, bs = (n * nk * 3 * 4 + 255) & ~(size_t)255;
    const size_t bo = (n * 4 + 255) & ~(size_t)255;
    const size_t bytes = bv + bs + 2 * bo;
    std::lock_guard<std::mutex> lk(S->mu);
    size_t ws = 0;
    for (const Slot &sl : S->slots) ws += slot_bytes(sl);
    if (S->bytes_resident + ws + bytes > S->opts.mem_budget_bytes) return TRI_ERR_CAPACITY;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};
    SrvScene sc;
    if (cudaMalloc(&sc.mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_OOM;
    }
    char *m = (char *)sc.mem;
    // cudaMemcpyDefault: the source may be host or device memory
    if (cudaMemcpy(m, scene->verts, n * 9 * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(m + bv, scene->sh, n * nk * 3 * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(m + bv + bs, scene->opacity, n * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(m + bv + bs + bo, scene->sigma, n * 4, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sc.mem);
        return TRI_ERR_CUDA;
    }
    sc.desc.verts = (const float *)m;
    sc.desc.sh = (const float *)(m + bv);
    sc.desc.opacity = (const float *)(m + bv + bs);
    sc.desc.sigma = (const float *)(m + bv + bs + bo);
    sc.desc.n = scene->n;
    sc.desc.sh_degree = scene->sh_degree;
    sc.bytes = bytes;
    const int32_t id = S->next_scene++;
    S->scenes[id] = sc;
    S->bytes_resident += bytes;
    *scene_id = id;
    return TRI_OK;
}

tri_status tri_serve_remove_scene(tri_serve *S, int32_t scene_id) {
    if (!S) return TRI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->scenes.find(scene_id);
    if (it == S->scenes.end()) return TRI_ERR_INVALID_ARG;
    it->second.removing = true;
    const double t0 = now_ms();
    // wait until no queued or running request uses it
    for (;;) {
        bool queued = false;
        for (const Req &r : S->queue) queued |= r.scene == scene_id;
        if (!queued && it->second.inflight == 0) break;
        if (now_ms() - t0 > 60000) return TRI_ERR_TIMEOUT;
        S->done_cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    // graphs may reference the scene's memory: the dispatcher drops them
    const uint64_t want = S->drops_done + S->drop_requests.size() + 1;
    S->drop_requests.push_back(scene_id);
    S->cv.notify_all();
    while (S->drops_done < want) {
        if (now_ms() - t0 > 60000) return TRI_ERR_TIMEOUT;
        S->done_cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    cudaSetDevice(S->device);
    cudaFree(it->second.mem);
    S->bytes_resident -= it->second.bytes;
    S->scenes.erase(it);
    return TRI_OK;
}

tri_status tri_serve_submit(tri_serve *S, int32_t scene_id, const tri_camera *cam, float *out_image,
                            uint64_t *ticket) {
    if (!S || !cam || !out_image || !ticket) return TRI_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0) return TRI_ERR_INVALID_ARG;
    if (cam->width > S->opts.max_width || cam->height > S->opts.max_height) return TRI_ERR_CAPACITY;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->scenes.find(scene_id);
    if (it == S->scenes.end() || it->second.removing) return TRI_ERR_INVALID_ARG;
    Req r;
    r.ticket = S->next_ticket++;
    r.scene = scene_id;
    r.cam = *cam;
    r.out = out_image;
    r.t_submit = now_ms();
    r.t_launch = r.t_submit;
    r.deadline = S->opts.timeout_ms > 0 ? r.t_submit + S->opts.timeout_ms : 0.0;
    if (S->t_first < 0) S->t_first = r.t_submit;
    S->queue.push_back(r);
    ++S->submitted;
    *ticket = r.ticket;
    S->cv.notify_one();
    return TRI_OK;
}

tri_status tri_serve_poll(tri_serve *S, uint64_t *done, int32_t *status, int32_t max, int32_t *ndone) {
    if (!S || !ndone || (max > 0 && !done)) return TRI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int32_t k = 0;
    while (k < max && !S->done_q.empty()) {
        done[k] = S->done_q.front().first;
        if (status) status[k] = S->done_q.front().second;
        S->done_q.pop_front();
        ++k;
    }
    *ndone = k;
    return TRI_OK;
}

tri_status tri_serve_wait(tri_serve *S, uint64_t ticket, int32_t timeout_ms) {
    if (!S) return TRI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return TRI_ERR_INVALID_ARG;
    const bool ok = S->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return S->done_map.count(ticket) > 0; });
    if (!ok) return TRI_ERR_TIMEOUT;
    return (tri_status)S->done_map[ticket];
}

tri_status tri_serve_stats(tri_serve *S, tri_serve_stats_t *out) {
    if (!S || !out) return TRI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->timed_out = S->timed_out;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->views / (double)S->batches : 0.0;
    out->bytes_resident = S->bytes_resident;
    out->graph_replays = S->graph_replays;
    out->graph_captures = S->graph_captures;
    out->eager_batches = S->eager_batches;
    out->reruns = S->reruns;
    out->reallocs = S->reallocs;
    out->eager_ms = S->eager_ms;
    out->capture_ms = S->capture_ms;
    for (const Slot &sl : S->slots) out->bytes_workspace += slot_bytes(sl);
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double pos = p * (double)(v.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        out->p50_ms = pct(0.50);
        std::vector<double> q = S->queue_ms;
        std::sort(q.begin(), q.end());
        if (!q.empty()) out->queue_p99_ms = q[(size_t)(0.99 * (double)(q.size() - 1))];
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / (double)v.size();
        const double span = S->t_last - S->t_first;
        out->fps = span > 0 ? (double)S->completed / (span * 1e-3) : 0.0;
    }
    return TRI_OK;
}

tri_status tri_serve_reset_stats(tri_serve *S) {
    if (!S) return TRI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_ms.clear();
    S->queue_ms.clear();
    S->submitted = S->completed = S->rejected = S->timed_out = S->batches = S->views = 0;
    S->graph_replays = S->graph_captures = S->eager_batches = S->reruns = S->reallocs = 0;
    S->eager_ms = S->capture_ms = 0.0;
    S->t_first = -1.0;
    S->t_last = 0.0;
    return TRI_OK;
}

void tri_serve_destroy(tri_serve *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        drop_graphs(sl);
        if (sl.ctx) tri_ctx_destroy(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_ctl) cudaFreeHost(sl.h_ctl);
    }
    for (auto &kv : S->scenes) cudaFree(kv.second.mem);
    delete S;
}

}  // extern "C"
