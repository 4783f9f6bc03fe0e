// Launch interfaces between the host-side API (api.cu) and the kernels.
#pragma once

#include "common.cuh"

namespace ts {

// Entry of the visible-item list, written by the preprocess for each item that passes
// its view's frustum test (CTA by CTA, in no particular order): (item id, depth key,
// x0 | y0 << 16, x1 | y1 << 16), the inclusive pixel rectangle; item id VIS_HOLE for an
// item that then touches no tile.
constexpr uint32_t VIS_HOLE = 0xffffffffu;
struct PreArgs {
    const float *verts, *sh, *opacity, *sigma;
    int64_t n;
    int sh_degree;
    const ViewDev *views;
    int nviews;
    Rec *recs;
    uint32_t *ntiles;
    ushort4 *rects;            // pixel rectangle (x0, y0, x1, y1), inclusive
    uint32_t *dkeys;           // depth key per item; 0xffffffff for items with no tile
    Ctl *ctl;
    int depth_hist = 0;        // also accumulate the 4 digit histograms of the depth keys
    uint32_t *tile_count = nullptr;  // if set (zeroed): pairs per tile, for the binning
    int solid = 0;                   // opaque-triangle records: full triangle, o = 1
    int window = WIN_POWER;          // window kind of the records
    float4 *zplane = nullptr;        // if set: [items] (a, b, c, 0), 1/z(p) = a (p.x - cx) + b (p.y - cy) + c
    uint4 *vislist = nullptr;        // if set: the visible-item list (entries as above)
    uint32_t vis_cap = 0;
    // if set: [triangles] bit v = the triangle's item of view v touches a tile; the
    // per-item ntiles and dkeys are then not written
    uint64_t *vmask = nullptr;
};

struct PreBwdArgs {
    const float *verts, *sh;
    const float *sigma = nullptr;   // read by the sigmoid window's chain rule
    int64_t n;
    int sh_degree;
    const ViewDev *views;
    int nviews;
    const uint32_t *ntiles;
    const uint64_t *vmask = nullptr;   // if set: read instead of ntiles (see PreArgs)
    const float *grad2d;       // [items][16]
    float *dverts, *dsh, *dopacity, *dsigma;
    int accumulate;
    int window = WIN_POWER;
};

// Start of a pipeline run in one kernel: the view table into views_d, the control
// block and the per-tile counts to zero. The table is passed by value, or, with
// `pinned`, read at run time from that page-locked host copy (what a captured graph
// does, so that its replays pick up the cameras written there before each launch).
void launch_step_init(const ViewDev *views, const ViewDev *pinned, int nviews, ViewDev *views_d, Ctl *ctl,
                      uint32_t *tile_count, int tiles, cudaStream_t st);
void launch_preprocess_fwd(const PreArgs &a, cudaStream_t st);
void launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t st);

// ---- sorting ----
constexpr int SORT_THREADS = 256;
constexpr int SORT_IPT_MAX = 15;                      // keys per thread, large sorts

// Keys per CTA tile used for a sort of at most `cap` keys: 256 x {4, 8, 15}, so that
// small sorts still spread over every SM.
int onesweep_tile(uint32_t cap, int sm_count);

// One stable 8-bit LSD pass over (key, value) pairs. `count` lives on the device and
// is clamped to `cap` (null: `cap` keys); `vin` null means value = index;
// `hist` is this digit's 256-bin histogram over all keys;
// `status` has room for ceil(cap / tile) x 256 words and is zeroed.
void launch_onesweep_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                          const uint32_t *count, uint32_t cap, const uint32_t *hist, uint32_t *status,
                          uint32_t *tile_counter, int shift, uint32_t *err, int tile, int sm_count,
                          cudaStream_t st);

struct EmitArgs {
    const uint32_t *sorted_items;   // depth-sorted visible items
    const uint32_t *ntiles;
    const ushort4 *rects;
    const ViewDev *views;
    int nviews;
    int64_t n;                      // triangles per view
    uint32_t *pkeys, *pvals;        // pair output
    uint32_t cap;
    int tile_passes;                // digits of the tile key
    uint32_t *lb_status;            // one word per CTA, zeroed
    Ctl *ctl;
};
void launch_emit(const EmitArgs &a, int64_t max_items, cudaStream_t st);

void launch_ranges(const uint32_t *keys, const uint32_t *count, uint2 *ranges, uint32_t total_tiles, uint32_t *err,
                   int grid, cudaStream_t st);

// ---- tile binning (binning.cu) ----
struct BinArgs {
    const ViewDev *views;
    int nviews;
    int64_t n;                      // triangles per view
    int64_t n_items;                // views x triangles
    uint32_t *tile_count;           // [total_tiles] pairs per tile (counted by the preprocess)
    uint32_t *tile_cursor;          // [total_tiles]
    uint2 *ranges;                  // [total_tiles]
    unsigned long long *kv;         // [cap] (depth key << 32 | item), unsorted within tiles
    unsigned long long *kv_tmp;     // [cap] merge buffer for ranges longer than one chunk
    uint32_t *items;                // [cap] sorted item ids
    uint32_t *big_tiles;            // [total_tiles] tiles whose range one warp cannot sort
    uint32_t *tile_order = nullptr; // [total_tiles] if set: tiles by descending pair count
    uint32_t cap;
    int total_tiles;
    const uint4 *vislist;           // [min(ctl->vis_count, vis_cap)] visible-item list (see PreArgs)
    uint32_t vis_cap;
    uint64_t *scan_status;          // [bin_scan_status_words] zeroed look-back words
    uint32_t *scan_ticket;          // zeroed CTA ticket of the scan
    Ctl *ctl;                       // n_pairs / n_pairs_used / overflow, work_counter[2], big_*
    uint64_t wait_ns = WAIT_NS;     // limit of the scan's look-back waits
    uint32_t withhold = 0;          // test: CTA withhold - 1 of the scan publishes no status
};
void launch_bin_scan(const BinArgs &a, cudaStream_t st);
size_t bin_scan_status_words(int total_tiles);
void launch_bin_scatter(const BinArgs &a, int sms, cudaStream_t st);
void launch_tile_sort(const BinArgs &a, int sms, cudaStream_t st);

// ---- densification (densify.cu) ----
struct DensifyArgs {
    float *verts, *sh, *opacity, *sigma;   // capacity >= n + 3 k triangles
    int nk;                                 // SH coefficients per channel
    int64_t n, k;
    const int32_t *sel;                     // [k] distinct triangle indices
    const float *noise;                     // [k][2] standard normal draws
    float noise_scale, tau_small;
    int64_t *n_out;                         // device: triangle count afterwards
    uint32_t *ticket;                       // zeroed CTA ticket
    uint32_t *lb_status;                    // [ceil(k / 256)] zeroed look-back words
    uint32_t *err;
};
void launch_densify(const DensifyArgs &a, cudaStream_t st);
void launch_prune_fold(const float *max_weight, const int32_t *n_pixels, int nviews, int64_t n, int min_pixels,
                       float *best, int32_t *views, int sms, cudaStream_t st);
void launch_prune_mask(const float *best, const int32_t *views, int64_t n, float tau_prune, int min_views,
                       uint8_t *keep, int sms, cudaStream_t st);
void launch_size_reg(const float *verts, int64_t n, float weight, float *loss, float *dverts, int sms,
                     cudaStream_t st);

// ---- rendering ----
// Render groups: the lanes of a warp that walk one backward list together (2x1 pixels
// for 2, 2x2 for 4, 2x4 for 8); the forward marks per pair which groups composited it,
// as KM_WORDS 32-bit words per pair (bit (32 / GROUP) b + g: group g of 8x4 block b).
#ifndef KM_GROUP
#define KM_GROUP 4
#endif
constexpr int GROUP = KM_GROUP;
constexpr int GROUPS_PER_TILE = TILE_PIX / GROUP;
constexpr int KM_WORDS = GROUPS_PER_TILE / 32;

constexpr int OUTS_INLINE = 4;   // views whose output pointers a launch can carry by value

struct RenderArgs {
    const ViewDev *views;
    const ViewOut *outs;            // device table, or a page-locked host copy (captured graphs)
    ViewOut outs_inline[OUTS_INLINE];   // used instead of `outs` when outs_by_value
    int outs_by_value = 0;
    int nviews;
    int total_tiles;
    const uint2 *ranges;
    const uint32_t *tile_order = nullptr;   // if set: the forward's tile visiting order
    const uint32_t *items;          // sorted pair item ids
    const Rec *recs;
    const ushort4 *rects;           // per-item pixel rectangles
    float *T_final;                 // [total pixels]
    int32_t *n_contrib;             // [total pixels]
    uint32_t *tile_max;             // [total tiles][GROUPS_PER_TILE]: largest n_contrib of each group
    uint32_t *stat_w;               // [items] largest T o as float bits (null: no statistics)
    uint32_t *stat_n;               // [items] pixels where the item was composited
    int32_t *ids = nullptr;         // solid render: [total pixels] triangle id of the winner, -1
    int64_t n_per_view = 0;         // triangles per view (item m = view * n_per_view + triangle)
    int window = WIN_POWER;         // window kind of the records
    int count_frags = 0;            // forward: count evaluated / composited fragments into the control block
    uint32_t *kmask;                // [pairs][KM_WORDS]: bit (32 / GROUP) w + g = group g of warp w composited the pair (forward
                                    // writes it when set; the backward requires it)
    float *grad2d;                  // backward: [items][16]
    uint32_t n_items;               // bound of the item ids in `items`
    Ctl *ctl;
    // per-pixel sort: the items' inverse-depth planes, per-pixel candidate counts and
    // offsets, and the candidates (depth bits << 32 | item), sorted per pixel
    const float4 *zplane = nullptr;
    uint32_t *pcount = nullptr;
    unsigned long long *poff = nullptr;
    unsigned long long *cand = nullptr;
    unsigned long long cand_cap = 0;
    unsigned long long *pscan_status = nullptr;
    int64_t total_pix = 0;
    // forward with the L1 loss (views with a target): *loss += loss_scale sum |image - target|
    float *loss = nullptr;
    float loss_scale = 0.0f;
};
__device__ __forceinline__ ViewOut view_out(const RenderArgs &a, int vw) {
    return a.outs_by_value ? a.outs_inline[vw] : a.outs[vw];
}
void launch_render_fwd(const RenderArgs &a, int grid, cudaStream_t st, bool solid = false);
void launch_render_bwd(const RenderArgs &a, int grid, cudaStream_t st);
// per-pixel sort: count the candidates (alpha >= 1/255) of every pixel; scan the counts
// into offsets (total into ctl->pps_total); fill, sort per pixel and composite; backward.
void launch_pps_count(const RenderArgs &a, int grid, cudaStream_t st);
void launch_pps_scan(const RenderArgs &a, cudaStream_t st);
__host__ __device__ size_t pps_scan_status_words(int64_t total_pix);
void launch_pps_fwd(const RenderArgs &a, int grid, cudaStream_t st);
void launch_pps_bwd(const RenderArgs &a, cudaStream_t st);

void launch_loss_l1(const float *img, const float *tgt, int64_t n, float *grad, float *loss, cudaStream_t st);

}  // namespace ts
