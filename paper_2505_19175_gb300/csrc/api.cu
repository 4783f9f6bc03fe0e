// C ABI of the triangle-splat renderer: contexts, workspace, pipeline sequencing.
// Declarations and contracts: include/trisplat.h.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"
#include "trisplat.h"

using namespace ts;

#include "ctx.h"

namespace {

// NVTX range over one API call (host timeline of profilers; free without one attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

constexpr int64_t MAX_PAIRS = (int64_t)LB_MASK;  // pair slots and item ids stay below 2^30

tri_status fail(tri_ctx *c, tri_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

tri_status cuda_fail(tri_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? TRI_ERR_OOM : TRI_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

// Record the stream of a call (see ensure).
void begin_call(tri_ctx *c, cudaStream_t st) {
    c->prev_stream = c->last_stream;
    c->last_stream = st;
}

// Grow `b` to at least `bytes` (never shrinks; a regrowth keeps 50 % headroom). Before
// freeing the old allocation it waits for the streams of this call and of the previous
// one, the only work of this context that can still use it. Allocation and release are
// stream-ordered (the device's memory pool) on this call's stream, so a growth never
// waits for other work on the device (cudaFree / cudaMalloc would synchronise it all);
// the stream is then synchronised so that the new buffer is usable from any stream.
tri_status ensure(tri_ctx *c, TsDevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return TRI_OK;
    cudaStream_t st = c->last_stream;
    size_t want = b.p ? bytes + bytes / 2 : bytes + bytes / 8;
    want = (want + 255) & ~(size_t)255;
    if (b.p) {
        CK(cudaStreamSynchronize(c->prev_stream));
        if (c->last_stream != c->prev_stream) CK(cudaStreamSynchronize(c->last_stream));
        CK(cudaFreeAsync(b.p, st));
        b.p = nullptr;
        b.bytes = 0;
    }
    if (c->fault_alloc > 0 && ++c->n_allocs == c->fault_alloc)
        return fail(c, TRI_ERR_OOM, "injected allocation failure (TRI_FAULT)");
    cudaError_t e = cudaMallocAsync(&b.p, want, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return cuda_fail(c, e, "cudaMallocAsync");
    }
    CK(cudaStreamSynchronize(st));
    b.bytes = want;
    ++c->realloc_gen;
    return TRI_OK;
}

#define ENSURE(buf, n)                          \
    do {                                        \
        tri_status s_ = ensure(c, (buf), (n));  \
        if (s_ != TRI_OK) return s_;            \
    } while (0)

// ensure() for buffers that must hold zeros when a kernel first sees them (look-back
// status words, which the kernels clear again after use): zeroed when (re)allocated.
static tri_status ensure_zeroed(tri_ctx *c, TsDevBuf &b, size_t bytes, cudaStream_t st) {
    void *old = b.p;
    const size_t old_bytes = b.bytes;
    const tri_status s = ensure(c, b, bytes);
    if (s != TRI_OK) return s;
    if (b.p != old || b.bytes != old_bytes) CK(cudaMemsetAsync(b.p, 0, b.bytes, st));
    return TRI_OK;
}

template <class T>
T *P(TsDevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

Ctl *ctl_of(tri_ctx *c) { return P<Ctl>(c->ctl); }

tri_status set_device(tri_ctx *c) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != c->device) CK(cudaSetDevice(c->device));
    return TRI_OK;
}

int64_t default_pair_cap(int64_t n_items) {
    int64_t cap = 4 * n_items;
    if (cap < (1 << 20)) cap = 1 << 20;
    if (cap > MAX_PAIRS) cap = MAX_PAIRS;
    return cap;
}

tri_status validate_scene(tri_ctx *c, const tri_scene *s) {
    if (!s) return fail(c, TRI_ERR_INVALID_ARG, "scene is null");
    if (s->n < 0) return fail(c, TRI_ERR_INVALID_ARG, "scene n < 0");
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(c, TRI_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (s->n > 0 && (!s->verts || !s->sh || !s->opacity || !s->sigma))
        return fail(c, TRI_ERR_INVALID_ARG, "scene pointer is null");
    // vertices and SH are staged with 16-byte vector loads
    if (((uintptr_t)s->verts & 15) || ((uintptr_t)s->sh & 15) || ((uintptr_t)s->opacity & 3) ||
        ((uintptr_t)s->sigma & 3))
        return fail(c, TRI_ERR_INVALID_ARG, "verts and sh must be 16-byte aligned");
    return TRI_OK;
}

}  // namespace

tri_status ts_build_views(tri_ctx *c, const tri_camera *cams, int nviews, std::vector<ViewDev> &out, int &tiles,
                          int64_t &pix) {
    if (!cams || nviews <= 0 || nviews > MAX_VIEWS)
        return fail(c, TRI_ERR_INVALID_ARG, "need 1.." + std::to_string(MAX_VIEWS) + " cameras");
    out.resize(nviews);
    int64_t tb = 0, pb = 0;
    for (int v = 0; v < nviews; ++v) {
        const tri_camera &k = cams[v];
        if (k.width <= 0 || k.height <= 0 || k.width > 65535 || k.height > 65535)
            return fail(c, TRI_ERR_INVALID_ARG, "camera width/height out of range");
        ViewDev &d = out[v];
        memcpy(d.R, k.R, sizeof d.R);
        memcpy(d.t, k.t, sizeof d.t);
        d.fx = k.fx; d.fy = k.fy; d.cx = k.cx; d.cy = k.cy;
        memcpy(d.bg, k.bg, sizeof d.bg);
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) acc -= (double)k.R[i * 3 + j] * (double)k.t[i];
            d.campos[j] = (float)acc;
        }
        d.W = k.width; d.H = k.height;
        d.tiles_x = (k.width + TILE - 1) / TILE;
        d.tiles_y = (k.height + TILE - 1) / TILE;
        d.tile_base = (int)tb;
        d.pix_base = (int)pb;
        tb += (int64_t)d.tiles_x * d.tiles_y;
        pb += (int64_t)k.width * k.height;
        if (tb > (1ll << 30) || pb > (1ll << 31) - 1) return fail(c, TRI_ERR_INVALID_ARG, "views too large");
    }
    tiles = (int)tb;
    pix = pb;
    return TRI_OK;
}

namespace {


// Host -> device copy of a small per-call table. Outside stream capture the driver
// stages the pageable source, so the caller may reuse it at once. Under capture the
// copy node must read memory that outlives the call: the context's pinned buffer,
// which a replay re-reads (the tables of the most recent captured call of this kind).
// The per-view output pointers of a render call: by value in the launch for a few views
// (no copy), through the page-locked host copy while the stream is captured (a replay
// reads what was written there before it), else copied to the device table.
static tri_status set_outs(tri_ctx *c, RenderArgs &r, const std::vector<ViewOut> &outs, TsDevBuf &dev, ViewOut *pinned,
                           cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    const int n = (int)outs.size();
    if (cs == cudaStreamCaptureStatusActive) {
        memcpy(pinned, outs.data(), sizeof(ViewOut) * n);
        r.outs = pinned;
        r.outs_by_value = 0;
    } else if (n <= OUTS_INLINE) {
        for (int v = 0; v < n; ++v) r.outs_inline[v] = outs[v];
        r.outs_by_value = 1;
    } else {
        CK(cudaMemcpyAsync(dev.p, outs.data(), sizeof(ViewOut) * n, cudaMemcpyHostToDevice, st));
        r.outs = P<ViewOut>(dev);
        r.outs_by_value = 0;
    }
    return TRI_OK;
}

// Pair buffers for the context's capacity: binned (depth key, item) words, the merge
// buffer of long tile ranges, and the sorted item ids.
tri_status ensure_pairs(tri_ctx *c) {
    ENSURE(c->kv, 8 * (size_t)c->pair_cap);
    ENSURE(c->kv_tmp, 8 * (size_t)c->pair_cap);
    ENSURE(c->items, 4 * (size_t)c->pair_cap);
    ENSURE(c->kmask, 4 * KM_WORDS * (size_t)c->pair_cap);
    return TRI_OK;
}

BinArgs bin_args(tri_ctx *c) {
    BinArgs b;
    b.views = P<ViewDev>(c->views_d);
    b.nviews = c->nviews;
    b.n = c->scene.n;
    b.n_items = c->n_items;
    b.vislist = P<uint4>(c->vislist);
    b.vis_cap = (uint32_t)c->n_items;
    b.tile_count = P<uint32_t>(c->tile_count);
    b.tile_cursor = P<uint32_t>(c->tile_cursor);
    b.ranges = P<uint2>(c->ranges);
    b.kv = P<unsigned long long>(c->kv);
    b.kv_tmp = P<unsigned long long>(c->kv_tmp);
    b.items = P<uint32_t>(c->items);
    b.big_tiles = P<uint32_t>(c->big_tiles);
    b.tile_order = P<uint32_t>(c->tile_order);
    b.scan_status = P<uint64_t>(c->scan_status);
    b.scan_ticket = &ctl_of(c)->cta_counter[3];
    b.cap = (uint32_t)c->pair_cap;
    b.total_tiles = c->total_tiles;
    b.ctl = ctl_of(c);
    return b;
}

tri_status launch_check(tri_ctx *c, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    return TRI_OK;
}

}  // namespace

extern "C" {

tri_status tri_ctx_create(tri_ctx **out, int device) {
    if (!out) return TRI_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TRI_ERR_CUDA;
    }
    tri_ctx *c = new tri_ctx();
    c->device = device;
    // host-side fault injection for tests: TRI_FAULT="alloc:N" fails the N-th device
    // allocation of the context, "slow:MS" delays every tri_bin_sort by MS ms
    if (const char *f = std::getenv("TRI_FAULT")) {
        if (!strncmp(f, "alloc:", 6)) c->fault_alloc = atol(f + 6);
        else if (!strncmp(f, "slow:", 5)) c->fault_slow_ms = atol(f + 5);
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    {
        // workspace growth releases memory to the device's default pool (cudaFreeAsync);
        // keep it there for the next growth instead of returning it at every sync
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    bool ok = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
              cudaMallocHost((void **)&c->h_views, sizeof(ViewDev) * MAX_VIEWS) == cudaSuccess &&
              cudaMallocHost((void **)&c->h_outs_fwd, sizeof(ViewOut) * MAX_VIEWS) == cudaSuccess &&
              cudaMallocHost((void **)&c->h_outs_bwd, sizeof(ViewOut) * MAX_VIEWS) == cudaSuccess;
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
    if (!ok) {
        cudaGetLastError();
        if (c->h_views) cudaFreeHost(c->h_views);
        if (c->h_outs_fwd) cudaFreeHost(c->h_outs_fwd);
        if (c->h_outs_bwd) cudaFreeHost(c->h_outs_bwd);
        delete c;
        return TRI_ERR_CUDA;
    }
    *out = c;
    return TRI_OK;
}

void tri_ctx_destroy(tri_ctx *c) {
    if (!c) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != c->device) cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (TsDevBuf *b : c->all())
        if (b->p) cudaFreeAsync(b->p, 0);   // pool allocations (see ensure)
    cudaStreamSynchronize(0);
    if (c->h_views) cudaFreeHost(c->h_views);
    if (c->h_outs_fwd) cudaFreeHost(c->h_outs_fwd);
    if (c->h_outs_bwd) cudaFreeHost(c->h_outs_bwd);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    delete c;
}

const char *tri_last_error(const tri_ctx *c) { return c ? c->err.c_str() : "null context"; }

tri_status tri_workspace_query(const tri_scene *scene, const tri_camera *cams, int nviews, int64_t pair_capacity,
                               size_t *bytes) {
    if (!bytes) return TRI_ERR_INVALID_ARG;
    tri_status s = validate_scene(nullptr, scene);
    if (s != TRI_OK) return s;
    std::vector<ViewDev> v;
    int tiles = 0;
    int64_t pix = 0;
    s = ts_build_views(nullptr, cams, nviews, v, tiles, pix);
    if (s != TRI_OK) return s;
    const int64_t M = scene->n * nviews;
    const int64_t cap = pair_capacity > 0 ? pair_capacity : default_pair_cap(M);
    size_t b = 0;
    b += (size_t)M * (sizeof(Rec) + 4 + 8 + 4 + GRAD_FIELDS * 4);    // records, counts, rects, keys, grads
    b += (size_t)cap * (8 + 8 + 4 + 2);                               // binned pairs, merge buffer, items, masks
    b += (size_t)tiles * (4 + 4 + 4 + 4 + 8 + 64) + (size_t)pix * 8;  // counts, cursors, queue, order, ranges, maxima
    b += sizeof(Ctl) + nviews * (sizeof(ViewDev) + 2 * sizeof(ViewOut));
    b += 256 * 18;                                                    // allocation rounding
    *bytes = b;
    return TRI_OK;
}

tri_status tri_reserve(tri_ctx *c, int64_t pair_capacity) {
    if (!c) return TRI_ERR_INVALID_ARG;
    if (pair_capacity <= 0 || pair_capacity > MAX_PAIRS)
        return fail(c, TRI_ERR_INVALID_ARG, "pair_capacity out of range");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    if (pair_capacity > c->pair_cap) c->pair_cap = pair_capacity;
    return ensure_pairs(c);
}

static tri_status preprocess_impl(tri_ctx *c, const tri_scene *scene, const tri_camera *cams, int nviews,
                                  bool solid, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    NvtxRange nv("tri_preprocess");
    tri_status s = validate_scene(c, scene);
    if (s != TRI_OK) return s;
    if ((s = set_device(c)) != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    begin_call(c, st);
    std::vector<ViewDev> views;
    int tiles = 0;
    int64_t pix = 0;
    if ((s = ts_build_views(c, cams, nviews, views, tiles, pix)) != TRI_OK) return s;
    const int64_t M = scene->n * (int64_t)nviews;
    if (M > (int64_t)LB_MASK) return fail(c, TRI_ERR_INVALID_ARG, "too many (view, triangle) items");
    c->scene = *scene;
    c->nviews = nviews;
    c->views = views;
    c->n_items = M;
    c->total_tiles = tiles;
    c->total_pix = pix;
    c->stage = 0;
    ENSURE(c->ctl, sizeof(Ctl));
    ENSURE(c->views_d, sizeof(ViewDev) * nviews);
    ENSURE(c->outs_fwd, sizeof(ViewOut) * nviews);
    ENSURE(c->outs_bwd, sizeof(ViewOut) * nviews);
    ENSURE(c->recs, sizeof(Rec) * (size_t)M);
    ENSURE(c->rects, 8 * (size_t)M);
    ENSURE(c->vislist, 16 * (size_t)M);
    ENSURE(c->vmask, 8 * (size_t)scene->n);
    ENSURE(c->tile_count, 4 * (size_t)tiles);
    ENSURE(c->tile_cursor, 4 * (size_t)tiles);
    ENSURE(c->big_tiles, 4 * (size_t)tiles);
    ENSURE(c->tile_order, 4 * (size_t)tiles);
    if ((s = ensure_zeroed(c, c->scan_status, 8 * bin_scan_status_words(tiles), st)) != TRI_OK) return s;
    ENSURE(c->ranges, sizeof(uint2) * (size_t)tiles);
    ENSURE(c->tile_max, 4 * GROUPS_PER_TILE * (size_t)tiles);
    ENSURE(c->Tfin, 4 * (size_t)pix);
    ENSURE(c->ncontrib, 4 * (size_t)pix);
    {
        // the view table: by value, or, while the stream is captured, through the pinned
        // copy that a replay reads at run time
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cs));
        const ViewDev *pinned = nullptr;
        if (cs == cudaStreamCaptureStatusActive) {
            memcpy(c->h_views, views.data(), sizeof(ViewDev) * nviews);
            pinned = c->h_views;
        }
        launch_step_init(views.data(), pinned, nviews, P<ViewDev>(c->views_d), ctl_of(c), P<uint32_t>(c->tile_count),
                         tiles, st);
        if ((s = launch_check(c, "step_init_kernel")) != TRI_OK) return s;
    }
    if (M > 0) {
        PreArgs a;
        a.verts = scene->verts;
        a.sh = scene->sh;
        a.opacity = scene->opacity;
        a.sigma = scene->sigma;
        a.n = scene->n;
        a.sh_degree = scene->sh_degree;
        a.views = P<ViewDev>(c->views_d);
        a.nviews = nviews;
        a.recs = P<Rec>(c->recs);
        a.rects = P<ushort4>(c->rects);
        a.vislist = P<uint4>(c->vislist);
        a.vmask = P<uint64_t>(c->vmask);
        a.vis_cap = (uint32_t)M;
        a.ctl = ctl_of(c);
        a.tile_count = P<uint32_t>(c->tile_count);
        a.solid = solid ? 1 : 0;
        a.window = c->window;
        if (!solid && c->sort == TRI_SORT_PIXEL) {
            ENSURE(c->zplane, sizeof(float4) * (size_t)M);
            a.zplane = P<float4>(c->zplane);
        }
        launch_preprocess_fwd(a, st);
        if ((s = launch_check(c, "preprocess_fwd_kernel")) != TRI_OK) return s;
    }
    c->stage = 1;
    c->solid = solid;
    c->rec_window = c->window;
    c->rec_sort = solid ? TRI_SORT_TILE : c->sort;
    return TRI_OK;
}

tri_status tri_preprocess(tri_ctx *c, const tri_scene *scene, const tri_camera *cams, int nviews, void *stream) {
    return preprocess_impl(c, scene, cams, nviews, false, stream);
}

tri_status tri_bin_sort(tri_ctx *c, int64_t *num_pairs_out, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    NvtxRange nv("tri_bin_sort");
    if (c->fault_slow_ms > 0) std::this_thread::sleep_for(std::chrono::milliseconds(c->fault_slow_ms));
    if (c->stage < 1) return fail(c, TRI_ERR_STATE, "tri_bin_sort before tri_preprocess");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    begin_call(c, st);
    Ctl *ctl = ctl_of(c);
    if (c->pair_cap <= 0) c->pair_cap = default_pair_cap(c->n_items);
    if ((s = ensure_pairs(c)) != TRI_OK) return s;
    // the scan and the sort leave their tickets, queues and look-back words at zero
    // (last_cta_done), and the scan assigns the pair totals
    BinArgs b = bin_args(c);
    if (c->test_withhold) {
        b.withhold = c->test_withhold;
        if (c->test_wait_ns) b.wait_ns = c->test_wait_ns;
        c->test_withhold = 0;
        c->test_wait_ns = 0;
    }
    // 1. per-tile counts (from tri_preprocess), 2. ranges
    launch_bin_scan(b, st);
    if ((s = launch_check(c, "bin_scan")) != TRI_OK) return s;
    if (num_pairs_out) {
        uint32_t np = 0;
        CK(cudaMemcpyAsync(&np, &ctl->n_pairs, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if ((int64_t)np > c->pair_cap) {
            // grow the pair buffers and redo the scan with the new capacity
            if ((int64_t)np > MAX_PAIRS) return fail(c, TRI_ERR_CAPACITY, "more than 2^30 pairs");
            int64_t cap = (int64_t)np + (int64_t)np / 4;
            if (cap > MAX_PAIRS) cap = MAX_PAIRS;
            c->pair_cap = cap;
            if ((s = ensure_pairs(c)) != TRI_OK) return s;
            b = bin_args(c);
            CK(cudaMemsetAsync(&ctl_of(c)->big_count, 0, 4, st));   // queued and counted by the first scan
            CK(cudaMemsetAsync(ctl_of(c)->ord_hist, 0, sizeof(ctl_of(c)->ord_hist), st));
            launch_bin_scan(b, st);
            if ((s = launch_check(c, "bin_scan")) != TRI_OK) return s;
        }
        *num_pairs_out = np;
    }
    // 3. scatter into the tile ranges, 4. per-tile depth order
    launch_bin_scatter(b, c->sms, st);
    launch_tile_sort(b, c->sms, st);
    if ((s = launch_check(c, "bin_scatter / tile_sort")) != TRI_OK) return s;
    c->stage = 2;
    return TRI_OK;
}

static RenderArgs render_args(tri_ctx *c, TsDevBuf &outs) {
    RenderArgs r;
    r.views = P<ViewDev>(c->views_d);
    r.outs = P<ViewOut>(outs);
    r.nviews = c->nviews;
    r.total_tiles = c->total_tiles;
    r.ranges = P<uint2>(c->ranges);
    r.tile_order = P<uint32_t>(c->tile_order);
    r.items = P<uint32_t>(c->items);
    r.recs = P<Rec>(c->recs);
    r.rects = P<ushort4>(c->rects);
    r.T_final = P<float>(c->Tfin);
    r.n_contrib = P<int32_t>(c->ncontrib);
    r.tile_max = P<uint32_t>(c->tile_max);
    r.grad2d = P<float>(c->grad2d);
    r.kmask = P<uint32_t>(c->kmask);
    r.stat_w = r.stat_n = nullptr;
    r.n_per_view = c->scene.n;
    r.window = c->rec_window;
    r.count_frags = c->count_frags;
    r.n_items = (uint32_t)c->n_items;
    r.ctl = ctl_of(c);
    return r;
}

// Forward of the per-pixel sort: candidate counts, their scan, then (outside stream
// capture) the total read back to size the candidate buffer; under capture the buffer
// must already hold them (overflow is reported by tri_ctx_check as an index error).
static tri_status render_fwd_pps(tri_ctx *c, RenderArgs &r, cudaStream_t st) {
    Ctl *ctl = ctl_of(c);
    const int64_t pix = c->total_pix;
    ENSURE(c->pcount, 4 * (size_t)pix);
    ENSURE(c->poff, 8 * (size_t)pix);
    tri_status s;
    if ((s = ensure_zeroed(c, c->pscan_status, 8 * pps_scan_status_words(pix), st)) != TRI_OK) return s;
    r.zplane = P<float4>(c->zplane);
    r.pcount = P<uint32_t>(c->pcount);
    r.poff = P<unsigned long long>(c->poff);
    r.pscan_status = P<unsigned long long>(c->pscan_status);
    r.total_pix = pix;
    launch_pps_count(r, c->sms, st);
    launch_pps_scan(r, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
        unsigned long long total = 0;
        CK(cudaMemcpyAsync(&total, &ctl->pps_total, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (total > c->cand_cap) {
            c->cand_cap = total + total / 4 + 1024;
            ENSURE(c->cand, 8 * (size_t)c->cand_cap);
        }
    } else if (c->cand_cap == 0) {
        return fail(c, TRI_ERR_STATE, "per-pixel sort captured before an uncaptured forward sized its buffer");
    }
    r.cand = P<unsigned long long>(c->cand);
    r.cand_cap = c->cand_cap;
    launch_pps_fwd(r, c->sms, st);
    return TRI_OK;
}

static tri_status render_fwd_impl(tri_ctx *c, float *const *images, float *const *T_final,
                                  int32_t *const *n_contrib, float *max_weight, int32_t *n_pixels, void *stream,
                                  int32_t *const *ids = nullptr, const float *const *targets = nullptr,
                                  float *const *grads = nullptr, float *loss = nullptr) {
    if (!c) return TRI_ERR_INVALID_ARG;
    NvtxRange nv("tri_render_fwd");
    if (c->stage < 2) return fail(c, TRI_ERR_STATE, "tri_render_fwd before tri_bin_sort");
    if (!images) return fail(c, TRI_ERR_INVALID_ARG, "images is null");
    for (int v = 0; v < c->nviews; ++v)
        if (!images[v]) return fail(c, TRI_ERR_INVALID_ARG, "image pointer is null");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    begin_call(c, st);
    std::vector<ViewOut> outs(c->nviews);
    int64_t n_loss = 0;
    for (int v = 0; v < c->nviews; ++v) {
        outs[v] = ViewOut{images[v], nullptr};
        if (targets) {
            outs[v].target = targets[v];
            outs[v].grad = grads[v];
            n_loss += 3 * (int64_t)c->views[v].W * c->views[v].H;
        }
    }
    RenderArgs r = render_args(c, c->outs_fwd);
    if ((s = set_outs(c, r, outs, c->outs_fwd, c->h_outs_fwd, st)) != TRI_OK) return s;
    if (targets) {
        r.loss = loss;
        r.loss_scale = 1.0f / (float)n_loss;
        if (loss) CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
    }
    if (c->solid) {
        r.kmask = nullptr;
        if (ids) {
            ENSURE(c->ids, 4 * (size_t)c->total_pix);
            r.ids = P<int32_t>(c->ids);
        }
    }
    if (max_weight && n_pixels) {
        CK(cudaMemsetAsync(max_weight, 0, 4 * (size_t)c->n_items, st));
        CK(cudaMemsetAsync(n_pixels, 0, 4 * (size_t)c->n_items, st));
        r.stat_w = reinterpret_cast<uint32_t *>(max_weight);
        r.stat_n = reinterpret_cast<uint32_t *>(n_pixels);
    }
    if (c->rec_sort == TRI_SORT_PIXEL) {
        if (r.stat_w) return fail(c, TRI_ERR_INVALID_ARG, "pruning statistics need the tile sort");
        if ((s = render_fwd_pps(c, r, st)) != TRI_OK) return s;
    } else {
        launch_render_fwd(r, c->sms, st, c->solid);
    }
    if ((s = launch_check(c, "render_fwd_kernel")) != TRI_OK) return s;
    for (int v = 0; v < c->nviews; ++v) {
        const ViewDev &V = c->views[v];
        const size_t np = (size_t)V.W * V.H;
        if (T_final && T_final[v])
            CK(cudaMemcpyAsync(T_final[v], P<float>(c->Tfin) + V.pix_base, 4 * np, cudaMemcpyDeviceToDevice, st));
        if (n_contrib && n_contrib[v])
            CK(cudaMemcpyAsync(n_contrib[v], P<int32_t>(c->ncontrib) + V.pix_base, 4 * np, cudaMemcpyDeviceToDevice,
                               st));
        if (r.ids && ids[v])
            CK(cudaMemcpyAsync(ids[v], P<int32_t>(c->ids) + V.pix_base, 4 * np, cudaMemcpyDeviceToDevice, st));
    }
    c->stage = 3;
    return TRI_OK;
}

tri_status tri_render_fwd(tri_ctx *c, float *const *images, float *const *T_final, int32_t *const *n_contrib,
                          void *stream) {
    return render_fwd_impl(c, images, T_final, n_contrib, nullptr, nullptr, stream);
}

tri_status tri_render_fwd_l1(tri_ctx *c, float *const *images, const float *const *targets, float *const *dL_dimages,
                             float *loss, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    if (!targets || !dL_dimages) return fail(c, TRI_ERR_INVALID_ARG, "targets or dL_dimages is null");
    for (int v = 0; v < c->nviews; ++v)
        if (!targets[v] || !dL_dimages[v]) return fail(c, TRI_ERR_INVALID_ARG, "target or dL_dimage pointer is null");
    if (c->solid) return fail(c, TRI_ERR_STATE, "the L1 forward after tri_render_solid");
    if (c->rec_sort == TRI_SORT_PIXEL)
        return fail(c, TRI_ERR_INVALID_ARG, "the fused L1 loss needs the tile sort (use tri_loss_l1)");
    return render_fwd_impl(c, images, nullptr, nullptr, nullptr, nullptr, stream, nullptr, targets, dL_dimages, loss);
}

tri_status tri_render_solid(tri_ctx *c, const tri_scene *scene, const tri_camera *cams, int nviews,
                            float *const *images, int32_t *const *ids, int64_t *num_pairs_out, void *stream) {
    tri_status s = preprocess_impl(c, scene, cams, nviews, true, stream);
    if (s != TRI_OK) return s;
    if ((s = tri_bin_sort(c, num_pairs_out, stream)) != TRI_OK) return s;
    return render_fwd_impl(c, images, nullptr, nullptr, nullptr, nullptr, stream, ids);
}

tri_status tri_set_window(tri_ctx *c, int window) {
    if (!c) return TRI_ERR_INVALID_ARG;
    if (window != TRI_WINDOW_POWER && window != TRI_WINDOW_SIGMOID)
        return fail(c, TRI_ERR_INVALID_ARG, "unknown window kind");
    c->window = window;
    c->stage = 0;   // records of the other kind are stale
    return TRI_OK;
}

tri_status tri_set_fragment_counting(tri_ctx *c, int on) {
    if (!c) return TRI_ERR_INVALID_ARG;
    c->count_frags = on ? 1 : 0;
    return TRI_OK;
}

tri_status tri_set_sort(tri_ctx *c, int sort) {
    if (!c) return TRI_ERR_INVALID_ARG;
    if (sort != TRI_SORT_TILE && sort != TRI_SORT_PIXEL) return fail(c, TRI_ERR_INVALID_ARG, "unknown sort kind");
    c->sort = sort;
    c->stage = 0;   // records of the other kind are stale
    return TRI_OK;
}

tri_status tri_densify(tri_ctx *c, float *verts, float *sh, float *opacity, float *sigma, int sh_degree, int64_t n,
                       int64_t capacity, const int32_t *sel, int64_t k, const float *noise, float noise_scale,
                       float tau_small, int64_t *n_out, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    if (!verts || !sh || !opacity || !sigma || !n_out || n < 0 || k < 0 || (k > 0 && (!sel || !noise)) ||
        sh_degree < 0 || sh_degree > 3)
        return fail(c, TRI_ERR_INVALID_ARG, "tri_densify: bad arguments");
    if (k > n) return fail(c, TRI_ERR_INVALID_ARG, "tri_densify: more selections than triangles");
    if (n + 3 * k > capacity) return fail(c, TRI_ERR_CAPACITY, "tri_densify: capacity below n + 3 k");
    if (3 * k > (int64_t)LB_MASK) return fail(c, TRI_ERR_CAPACITY, "tri_densify: too many selections");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    begin_call(c, st);
    ENSURE(c->ctl, sizeof(Ctl));
    if (k == 0) {
        CK(cudaMemcpyAsync(n_out, &n, sizeof n, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));   // the source is a host stack variable
        return TRI_OK;
    }
    const size_t words = (size_t)((k + 255) / 256) + 1;
    ENSURE(c->dens_status, 4 * words);
    CK(cudaMemsetAsync(c->dens_status.p, 0, 4 * words, st));
    CK(cudaMemsetAsync(&ctl_of(c)->cta_counter[2], 0, 4, st));
    DensifyArgs a;
    a.verts = verts;
    a.sh = sh;
    a.opacity = opacity;
    a.sigma = sigma;
    a.nk = (sh_degree + 1) * (sh_degree + 1);
    a.n = n;
    a.k = k;
    a.sel = sel;
    a.noise = noise;
    a.noise_scale = noise_scale;
    a.tau_small = tau_small;
    a.n_out = n_out;
    a.ticket = &ctl_of(c)->cta_counter[2];
    a.lb_status = P<uint32_t>(c->dens_status);
    a.err = &ctl_of(c)->error;
    launch_densify(a, st);
    return launch_check(c, "densify_kernel");
}

tri_status tri_size_reg(const float *verts, int64_t n, float weight, float *loss, float *dverts, void *stream) {
    if (!verts || n < 0 || (!loss && !dverts)) return TRI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_CUDA;
    }
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return TRI_ERR_CUDA;
    launch_size_reg(verts, n, weight, loss, dverts, sms, st);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

static tri_status current_sms(int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_CUDA;
    }
    return TRI_OK;
}

tri_status tri_prune_fold(const float *max_weight, const int32_t *n_pixels, int nviews, int64_t n, int min_pixels,
                          float *best, int32_t *views, void *stream) {
    if (n < 0 || nviews < 0) return TRI_ERR_INVALID_ARG;
    if (n == 0 || nviews == 0) return TRI_OK;
    if (!max_weight || !n_pixels || !best || !views) return TRI_ERR_INVALID_ARG;
    int sms = 1;
    if (current_sms(&sms) != TRI_OK) return TRI_ERR_CUDA;
    launch_prune_fold(max_weight, n_pixels, nviews, n, min_pixels, best, views, sms, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

tri_status tri_prune_mask(const float *best, const int32_t *views, int64_t n, float tau_prune, int min_views,
                          uint8_t *keep, void *stream) {
    if (n < 0 || (n > 0 && (!best || !views || !keep))) return TRI_ERR_INVALID_ARG;
    if (n == 0) return TRI_OK;
    int sms = 1;
    if (current_sms(&sms) != TRI_OK) return TRI_ERR_CUDA;
    launch_prune_mask(best, views, n, tau_prune, min_views, keep, sms, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

tri_status tri_render_fwd_stats(tri_ctx *c, float *const *images, float *const *T_final,
                                int32_t *const *n_contrib, float *max_weight, int32_t *n_pixels, void *stream) {
    if (c && (!max_weight || !n_pixels)) return fail(c, TRI_ERR_INVALID_ARG, "statistics outputs are null");
    return render_fwd_impl(c, images, T_final, n_contrib, max_weight, n_pixels, stream);
}

tri_status tri_render_bwd(tri_ctx *c, const float *const *dL, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    NvtxRange nv("tri_render_bwd");
    if (c->stage < 3) return fail(c, TRI_ERR_STATE, "tri_render_bwd before tri_render_fwd");
    if (c->solid) return fail(c, TRI_ERR_STATE, "tri_render_bwd after tri_render_solid (no backward)");
    if (!dL) return fail(c, TRI_ERR_INVALID_ARG, "dL_dimages is null");
    for (int v = 0; v < c->nviews; ++v)
        if (!dL[v]) return fail(c, TRI_ERR_INVALID_ARG, "dL_dimage pointer is null");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    begin_call(c, st);
    std::vector<ViewOut> outs(c->nviews);
    for (int v = 0; v < c->nviews; ++v) outs[v] = ViewOut{nullptr, dL[v]};
    ENSURE(c->grad2d, sizeof(float) * GRAD_FIELDS * (size_t)c->n_items);
    CK(cudaMemsetAsync(c->grad2d.p, 0, sizeof(float) * GRAD_FIELDS * (size_t)c->n_items, st));
    RenderArgs r = render_args(c, c->outs_bwd);
    if ((s = set_outs(c, r, outs, c->outs_bwd, c->h_outs_bwd, st)) != TRI_OK) return s;
    if (c->rec_sort == TRI_SORT_PIXEL) {
        r.poff = P<unsigned long long>(c->poff);
        r.pcount = P<uint32_t>(c->pcount);
        r.cand = P<unsigned long long>(c->cand);
        r.cand_cap = c->cand_cap;
        r.total_pix = c->total_pix;
        launch_pps_bwd(r, st);
    } else {
        launch_render_bwd(r, c->sms, st);
    }
    if ((s = launch_check(c, "render_bwd_kernel")) != TRI_OK) return s;
    c->stage = 4;
    return TRI_OK;
}

tri_status tri_preprocess_bwd(tri_ctx *c, float *dverts, float *dsh, float *dopacity, float *dsigma, int accumulate,
                              void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    NvtxRange nv("tri_preprocess_bwd");
    if (c->stage < 4) return fail(c, TRI_ERR_STATE, "tri_preprocess_bwd before tri_render_bwd");
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    PreBwdArgs a;
    a.verts = c->scene.verts;
    a.sh = c->scene.sh;
    a.sigma = c->scene.sigma;
    a.window = c->rec_window;
    a.n = c->scene.n;
    a.sh_degree = c->scene.sh_degree;
    a.views = P<ViewDev>(c->views_d);
    a.nviews = c->nviews;
    a.ntiles = nullptr;
    a.vmask = P<uint64_t>(c->vmask);
    a.grad2d = P<float>(c->grad2d);
    a.dverts = dverts;
    a.dsh = dsh;
    a.dopacity = dopacity;
    a.dsigma = dsigma;
    a.accumulate = accumulate;
    launch_preprocess_bwd(a, st);
    return launch_check(c, "preprocess_bwd_kernel");
}

tri_status tri_ctx_check(tri_ctx *c, tri_ctx_info *info, void *stream) {
    if (!c) return TRI_ERR_INVALID_ARG;
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    Ctl h;
    memset(&h, 0, sizeof h);
    if (c->ctl.p) CK(cudaMemcpy(&h, c->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (info) {
        info->n_items = c->n_items;
        info->n_visible = h.n_visible;
        info->n_pairs = h.n_pairs;
        info->pair_capacity = c->pair_cap;
        info->overflow = (int32_t)h.overflow;
        info->device_error = (int32_t)h.error;
        info->n_views = c->nviews;
        info->total_tiles = c->total_tiles;
        info->frag_evaluated = (int64_t)h.frag_eval;
        info->frag_composited = (int64_t)h.frag_kept;
    }
    if (h.error & ERR_SPIN) return fail(c, TRI_ERR_TIMEOUT, "a bounded device wait gave up");
    if (h.error) return fail(c, TRI_ERR_DEVICE_CHECK, "device-side check failed");
    if (h.overflow) return fail(c, TRI_ERR_CAPACITY, "pair buffer overflow");
    return TRI_OK;
}

tri_status tri_debug_withhold_scan(tri_ctx *c, int32_t cta, uint64_t wait_ns) {
    if (!c || cta < 0) return TRI_ERR_INVALID_ARG;
    c->test_withhold = (uint32_t)cta + 1u;
    c->test_wait_ns = wait_ns;
    return TRI_OK;
}

tri_status tri_debug_copy(tri_ctx *c, int which, void *dst, size_t max_bytes, size_t *bytes) {
    if (!c || !dst) return TRI_ERR_INVALID_ARG;
    tri_status s = set_device(c);
    if (s != TRI_OK) return s;
    CK(cudaDeviceSynchronize());
    Ctl h;
    memset(&h, 0, sizeof h);
    if (c->ctl.p) CK(cudaMemcpy(&h, c->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost));
    const void *src = nullptr;
    size_t n = 0;
    const size_t M = (size_t)c->n_items;
    const size_t np = (size_t)(h.n_pairs_used);
    switch (which) {
        case 0: {
            // tile id of every sorted pair, expanded from the tile ranges
            n = 4 * np;
            if (n > max_bytes) return fail(c, TRI_ERR_CAPACITY, "destination too small");
            std::vector<uint2> rg((size_t)c->total_tiles);
            if (!rg.empty()) CK(cudaMemcpy(rg.data(), c->ranges.p, sizeof(uint2) * rg.size(), cudaMemcpyDeviceToHost));
            uint32_t *out = (uint32_t *)dst;
            for (size_t t = 0; t < rg.size(); ++t)
                for (uint32_t k = rg[t].x; k < rg[t].y && k < np; ++k) out[k] = (uint32_t)t;
            if (bytes) *bytes = n;
            return TRI_OK;
        }
        case 1: src = c->items.p; n = 4 * np; break;
        case 2: src = c->ranges.p; n = sizeof(uint2) * (size_t)c->total_tiles; break;
        case 3:
        case 5: {
            // per-item depth keys / tile counts, from the visible-item list (items without
            // an entry: key 0xffffffff, count 0)
            n = 4 * M;
            if (n > max_bytes) return fail(c, TRI_ERR_CAPACITY, "destination too small");
            std::vector<uint4> L(std::min((size_t)h.vis_count, M));
            if (!L.empty()) CK(cudaMemcpy(L.data(), c->vislist.p, sizeof(uint4) * L.size(), cudaMemcpyDeviceToHost));
            uint32_t *out = (uint32_t *)dst;
            for (size_t k = 0; k < M; ++k) out[k] = which == 3 ? 0xffffffffu : 0u;
            for (const uint4 &e : L) {
                if (e.x == VIS_HOLE || e.x >= M) continue;
                const uint32_t tw = (e.w & 0xffffu) / TILE - (e.z & 0xffffu) / TILE + 1;
                const uint32_t th = (e.w >> 16) / TILE - (e.z >> 16) / TILE + 1;
                out[e.x] = which == 3 ? e.y : tw * th;
            }
            if (bytes) *bytes = n;
            return TRI_OK;
        }
        case 4: src = c->rects.p; n = 8 * M; break;
        case 6: src = c->kv.p; n = 8 * np; break;
        case 7: src = c->recs.p; n = sizeof(Rec) * M; break;
        case 8: src = c->grad2d.p; n = sizeof(float) * GRAD_FIELDS * M; break;
        case 9: src = c->tile_order.p; n = 4 * (size_t)c->total_tiles; break;
        default: return fail(c, TRI_ERR_INVALID_ARG, "unknown buffer");
    }
    if (n > max_bytes) return fail(c, TRI_ERR_CAPACITY, "destination too small");
    if (bytes) *bytes = n;
    if (n == 0) return TRI_OK;
    if (!src) return fail(c, TRI_ERR_STATE, "buffer not allocated");
    CK(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost));
    return TRI_OK;
}

tri_status tri_loss_l1(const float *image, const float *target, int64_t n, float *dL_dimage, float *loss,
                       void *stream) {
    if (!image || !target || !dL_dimage || n < 0) return TRI_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return TRI_ERR_CUDA;
    launch_loss_l1(image, target, n, dL_dimage, loss, st);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

}  // extern "C"
