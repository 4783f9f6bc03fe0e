// Internal definition of the renderer context (shared by api.cu, serve.cu).
#pragma once

#include <string>
#include <vector>

#include "kernels.h"
#include "trisplat.h"

struct TsDevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct tri_ctx {
    int device = 0;
    int sms = 0;
    std::string err;
    tri_scene scene{};
    int nviews = 0;
    std::vector<ts::ViewDev> views;
    int64_t n_items = 0;
    int total_tiles = 0;
    int64_t total_pix = 0;
    int64_t pair_cap = 0;
    int stage = 0;  // 1 preprocessed, 2 sorted, 3 rendered, 4 backward rendered
    bool solid = false;  // records of the opaque-triangle render (no backward)
    int window = 0;      // window kind for the next tri_preprocess (tri_set_window)
    int rec_window = 0;  // window kind of the current records
    int sort = 0;        // compositing order for the next tri_preprocess (tri_set_sort)
    int count_frags = 0; // forwards count their fragments (tri_set_fragment_counting)
    int rec_sort = 0;    // compositing order of the current records
    uint64_t cand_cap = 0;   // per-pixel sort: candidate capacity
    long fault_alloc = 0, fault_slow_ms = 0, n_allocs = 0;   // TRI_FAULT injection (tests)
    uint32_t test_withhold = 0;     // tri_debug_withhold_scan: CTA + 1 (0: none), next tri_bin_sort only
    uint64_t test_wait_ns = 0;      // and the scan's wait limit (0: the default)
    uint64_t realloc_gen = 0;   // bumped whenever a device buffer is reallocated
    // streams of the previous and the current call: a reallocation waits for both,
    // not for the whole device
    cudaStream_t prev_stream = nullptr, last_stream = nullptr;
    // pinned copies of the small per-call tables, used while the stream is captured
    ts::ViewDev *h_views = nullptr;
    ts::ViewOut *h_outs_fwd = nullptr, *h_outs_bwd = nullptr;
    TsDevBuf views_d, outs_fwd, outs_bwd, ctl, recs, rects, tile_count, tile_cursor, big_tiles, tile_order,
        kv, kv_tmp, items, kmask, ids, dens_status, scan_status, ranges, tile_max, Tfin, ncontrib, grad2d, zplane, pcount,
        poff, cand, pscan_status, vislist, vmask;
    std::vector<TsDevBuf *> all() {
        return {&views_d, &outs_fwd, &outs_bwd, &ctl, &recs, &rects, &tile_count, &tile_cursor,
                &big_tiles, &tile_order, &kv, &kv_tmp, &items, &kmask, &ids, &dens_status, &scan_status, &ranges, &tile_max, &Tfin, &ncontrib, &grad2d,
                &zplane, &pcount, &poff, &cand, &pscan_status, &vislist, &vmask};
    }
};

// Device view table of `cams` (validated); tiles / pixels of all views.
tri_status ts_build_views(tri_ctx *c, const tri_camera *cams, int nviews, std::vector<ts::ViewDev> &out, int &tiles,
                          int64_t &pix);
