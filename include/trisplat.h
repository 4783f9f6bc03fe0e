/*
 * trisplat.h — C ABI of the GB300 (sm_103a) differentiable triangle-splat rasterizer.
 *
 * The renderer follows "Triangle Splatting for Real-Time Radiance Field Rendering"
 * (arXiv 2505.19175). A scene is a soup of 3D triangles, each with three vertices
 * v_i, a spherical-harmonic colour c (degree <= 3, 48 floats at degree 3), a
 * smoothness sigma > 0 and an opacity o (Sec. 3.1 "Differentiable rasterization";
 * Sec. 4 counts 59 parameters per triangle). A pinhole camera K, R, t maps it to an
 * image; image gradients map back to parameter gradients (Sec. 3.3 "Optimization").
 *
 * Pipeline (one call each, all stream-ordered, none synchronises unless stated):
 *   tri_preprocess      project, build the signed-distance window, colour, depth and
 *                       tight tile rectangle of every (view, triangle) item
 *                       (Sec. 3.1, Eq. indicator1; Supp. "Tile assignment");
 *   tri_bin_sort        duplication of visible items into the tiles they touch,
 *                       binned by tile into per-tile ranges, each range ordered by
 *                       centroid depth (Supp. "Tile assignment", "Depth sorting");
 *   tri_render_fwd      per-pixel front-to-back compositing with alpha = o I (Sec. 3.1:
 *                       the rendering equation of prior splatting work);
 *   tri_render_bwd      back-to-front recomputation and per-item gradients;
 *   tri_preprocess_bwd  chain rule to vertices, SH, opacity and sigma.
 *
 * Conventions.
 *   Alignment: verts and sh must start on a 16-byte boundary (they are read with
 *     16-byte vector loads); any fresh cudaMalloc / torch allocation satisfies this.
 *   Device pointers: every float / int pointer below, unless marked host, is device
 *     memory of the context's device, fp32 / int32, contiguous, caller-owned. The
 *     library never frees caller memory.
 *   Workspace: each context owns its device workspace (cudaMalloc'd on demand, grown
 *     as needed, freed by tri_ctx_destroy). tri_workspace_query reports its size.
 *   Layouts: verts [n][3][3] (vertex-major xyz), sh [n][(deg+1)^2][3] (coefficient
 *     k = l*l + l + m, m = -l..l; channel innermost), opacity [n], sigma [n]; images
 *     [3][H][W] planar per view; per-pixel buffers [H][W].
 *   Camera: R row-major world->camera, t, OpenCV axes (+x right, +y down, +z
 *     forward); pixel (x, y) is sampled at (x + 0.5, y + 0.5).
 *   Errors: every call returns a tri_status and never aborts; tri_last_error gives a
 *     message. Device-side checks (bounded spins, capacity) set a status word that
 *     tri_ctx_check reads back (that call synchronises the stream).
 *   Threads: a context is not thread-safe; use one per host thread.
 *   Tracing: each pipeline call is an NVTX range (tri_preprocess, tri_bin_sort, ...).
 *   Fault injection (tests, host side only): the environment variable TRI_FAULT read at
 *     tri_ctx_create: "alloc:N" makes the context's N-th device allocation fail with
 *     TRI_ERR_OOM; "slow:MS" delays every tri_bin_sort by MS milliseconds on the host.
 *   Streams: cudaStream_t values are passed as void* (0 = legacy default stream).
 *   CUDA graphs: tri_preprocess, tri_bin_sort (with num_pairs_out = NULL),
 *     tri_render_fwd, tri_render_fwd_l1, tri_render_bwd, tri_preprocess_bwd and
 *     tri_loss_l1 may be
 *     captured once the context's buffers are sized by an eager run of the same
 *     workload (a capture allocates nothing). A replay's kernels read the context's
 *     page-locked copies of its camera and output-pointer tables at run time, as written
 *     by its most recent captured call of each kind (eager calls pass the tables by
 *     value, or copy them to the device, and do not touch these copies). A step makes no
 *     other host copies; its queues and look-back words are reset by the kernels.
 */
#ifndef TRISPLAT_H
#define TRISPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRI_OK = 0,
    TRI_ERR_INVALID_ARG = 1,   /* null pointer, n < 0, sh_degree not in 0..3, W/H <= 0, ... */
    TRI_ERR_OOM = 2,           /* cudaMalloc failed */
    TRI_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in tri_last_error) */
    TRI_ERR_CAPACITY = 4,      /* pair list or memory budget exceeded */
    TRI_ERR_TIMEOUT = 5,       /* a bounded device wait or a request deadline ran out */
    TRI_ERR_DEVICE_CHECK = 6,  /* a device-side check set the status word */
    TRI_ERR_STATE = 7          /* calls out of order (e.g. render before bin_sort) */
} tri_status;

/* Pinhole camera of one view (Sec. 3.1: q = K(R v + t) with the perspective divide). */
typedef struct {
    float R[9];        /* world -> camera rotation, row-major */
    float t[3];        /* world -> camera translation */
    float fx, fy;      /* focal lengths in pixels */
    float cx, cy;      /* principal point in pixels */
    int32_t width, height;  /* 1..65535 */
    float bg[3];       /* background colour added with the final transmittance */
} tri_camera;

/* Triangle soup (Sec. 3.1; 59 floats per triangle at SH degree 3, Sec. 4).
 * opacity is the activated o in (0, 1], sigma the activated sigma > 0. */
typedef struct {
    const float *verts;    /* [n][3][3] */
    const float *sh;       /* [n][(sh_degree+1)^2][3] */
    const float *opacity;  /* [n] */
    const float *sigma;    /* [n] */
    int64_t n;
    int32_t sh_degree;     /* 0..3 */
} tri_scene;

typedef struct tri_ctx tri_ctx;

/* Counters of the last pipeline run (tri_ctx_check fills them). */
typedef struct {
    int64_t n_items;       /* views x triangles */
    int64_t n_visible;     /* items with a non-empty tile rectangle */
    int64_t n_pairs;       /* (tile, item) pairs, may exceed pair_capacity */
    int64_t pair_capacity;
    int32_t overflow;      /* 1 when n_pairs > pair_capacity (pairs were dropped) */
    int32_t device_error;  /* bit 0: a bounded spin gave up; bit 1: index check failed */
    int32_t n_views, total_tiles;
    int64_t frag_evaluated;   /* counted forwards since the last tri_preprocess: (pixel, list entry) window
                                 evaluations (0 unless tri_set_fragment_counting is on) */
    int64_t frag_composited;  /* the same: fragments composited */
} tri_ctx_info;

/* Create a context on CUDA device `device`. Allocates nothing until first use.
 * Returns TRI_ERR_INVALID_ARG for a null `out`, TRI_ERR_CUDA for a bad device. */
tri_status tri_ctx_create(tri_ctx **out, int device);

/* Free the context and all its device workspace. Null is ignored. */
void tri_ctx_destroy(tri_ctx *ctx);

/* Message of the last failed call on this context ("" if none). Never null. */
const char *tri_last_error(const tri_ctx *ctx);

/* Device bytes a context holds to render `nviews` views of an n-triangle scene with
 * room for `pair_capacity` (tile, item) pairs (<= 0: the library's default estimate).
 * Pure host arithmetic; `cams` is a host array of nviews cameras. */
tri_status tri_workspace_query(const tri_scene *scene, const tri_camera *cams, int nviews,
                               int64_t pair_capacity, size_t *bytes);

/* Reserve room for at least `pair_capacity` pairs now (optional; bin_sort grows it
 * when it synchronises). Allocates with cudaMalloc. */
tri_status tri_reserve(tri_ctx *ctx, int64_t pair_capacity);

/* Step 1 (Sec. 3.1; Supp. "Tile assignment"): for every (view, triangle) item, project
 * the vertices (vertex 0 in double-float precision, the others relative to it), cull
 * items with a vertex nearer than z = 0.2 or an inradius below 1e-4 px, build the three
 * normalised edge lines (m_i = 1 at the incenter, 0 on edge i), the SH colour for the
 * direction camera -> centroid, the centroid depth and the tile rectangle of the
 * triangle shrunk about its incenter by f = 1 - (1/255 / o)^(1/sigma); and compact the
 * visible items in index order. `scene` device pointers must stay valid until
 * tri_preprocess_bwd. `cams` is a host array of `nviews` cameras (views may differ in
 * resolution). */
tri_status tri_preprocess(tri_ctx *ctx, const tri_scene *scene, const tri_camera *cams,
                          int nviews, void *stream);

/* Step 2 (Supp. "Depth sorting", "Tile assignment"): duplication of every visible item
 * into the tiles of its rectangle, binned by tile (per-tile counts, their scan into
 * [start, end) ranges, a scatter of the preprocess's list of visible items into the
 * ranges), then each tile's range sorted by
 * (32-bit centroid-depth key, item id). The result equals a stable sort of the 64-bit
 * keys (tile << 32 | depth bits) emitted in item order.
 * If `num_pairs_out` is non-null the call synchronises after the counts, returns the
 * pair count there, and grows the pair buffers before the scatter when they are too
 * small. If null,
 * nothing synchronises; an overflow drops pairs, sets the status word, and
 * tri_ctx_check reports TRI_ERR_CAPACITY. */
tri_status tri_bin_sort(tri_ctx *ctx, int64_t *num_pairs_out, void *stream);

/* Step 3 (Sec. 3.1): per pixel, in sorted order: ratio = min_i m_i(p); skip if ratio <= 0;
 * I = ratio^sigma; alpha = o I; skip if alpha < 1/255; alpha = min(alpha, 0.99); stop
 * before a fragment that would take the transmittance T below 1e-4; C += rgb alpha T;
 * T *= 1 - alpha. Output C + T bg.
 * `images` is a host array of nviews device pointers, each [3][H_v][W_v].
 * `T_final` / `n_contrib` (host arrays of nviews device pointers to [H_v][W_v], or null
 * arrays) receive the final transmittance and the 1-based index, within the tile's
 * list, of the last composited entry; the context keeps its own copies for the
 * backward pass either way. */
tri_status tri_render_fwd(tri_ctx *ctx, float *const *images, float *const *T_final,
                          int32_t *const *n_contrib, void *stream);

/* Step 3 fused with the L1 photometric loss (Sec. 3.3 lists L1 among the loss terms):
 * as tri_render_fwd (images only), and in the same kernel, per view v,
 * dL_dimages[v] = sign(image - targets[v]) / n and, when `loss` is not null,
 * *loss = sum over views of |image - target| / n, with n = sum_v 3 W_v H_v: the values
 * tri_loss_l1 gives over the views' images as one array (the gradient bit for bit, the
 * loss up to summation order), without a second pass over the images. targets and
 * dL_dimages: nviews device pointers [3][H_v][W_v] (caller-owned); loss: a device
 * float. TRI_ERR_INVALID_ARG for null pointers or with TRI_SORT_PIXEL (use
 * tri_loss_l1 there); TRI_ERR_STATE after tri_render_solid. Graph-capturable. */
tri_status tri_render_fwd_l1(tri_ctx *ctx, float *const *images, const float *const *targets,
                             float *const *dL_dimages, float *loss, void *stream);

/* Step 3 with the pruning statistics of Sec. 3.3 ("Pruning"): as tri_render_fwd, and
 * for every (view, triangle) item m = v n + i, max_weight[m] = the largest blending
 * weight T o over the pixels where the item was composited (T = transmittance in
 * front of the fragment, o its opacity; 0 if none) and n_pixels[m] = the number of
 * those pixels. Both are device arrays of n_items = nviews x n entries (float /
 * int32), overwritten (zeroed first, on the stream). The pruning decisions across
 * views (largest weight below tau_prune; fewer than two views with more than one
 * pixel) are device reductions of these arrays (tri_prune_fold, tri_prune_mask). Same errors as tri_render_fwd;
 * TRI_ERR_INVALID_ARG for a null output. */
tri_status tri_render_fwd_stats(tri_ctx *ctx, float *const *images, float *const *T_final,
                                int32_t *const *n_contrib, float *max_weight, int32_t *n_pixels,
                                void *stream);

/* Opaque-triangle render (Sec. 5 turns the optimised soup into solid triangles for
 * game engines; this is the CUDA counterpart, the sigma -> 0, o = 1 limit of the splat
 * render): tri_preprocess with every triangle taken whole and opaque (opacity and
 * sigma ignored; near-plane and degenerate triangles culled), tri_bin_sort, then each
 * pixel takes the colour of the nearest triangle by centroid depth (ties: lower
 * index) whose window ratio at the pixel centre is positive, else the background.
 * images [nviews] -> [3][H][W]; ids (nullable; entries nullable) -> [H][W] int32
 * winning triangle index, -1 for background. num_pairs_out as in tri_bin_sort (null:
 * no synchronisation). The context then holds no backward state: tri_render_bwd
 * returns TRI_ERR_STATE until the next tri_preprocess. */
tri_status tri_render_solid(tri_ctx *ctx, const tri_scene *scene, const tri_camera *cams, int nviews,
                            float *const *images, int32_t *const *ids, int64_t *num_pairs_out,
                            void *stream);

/* Step 4 (gradient of step 3): per pixel, back to front from its last composited
 * entry, recompute alpha and T_k = T_{k+1} / (1 - alpha_k), and accumulate per item
 * the gradients of the incenter, the six edge-line slopes, o, sigma and rgb (warp
 * reduction, then one vector atomic per item and tile). `dL_dimages` is a host array of
 * nviews device pointers [3][H_v][W_v]. Requires tri_render_fwd on the same context. */
tri_status tri_render_bwd(tri_ctx *ctx, const float *const *dL_dimages, void *stream);

/* Step 5 (chain rule of step 1): gradients of the loss with respect to the scene,
 * summed over views: dverts [n][3][3], dsh [n][(deg+1)^2][3], dopacity [n],
 * dsigma [n]. With accumulate = 0 the outputs are overwritten, else added to. Any
 * output pointer may be null to skip it. */
tri_status tri_preprocess_bwd(tri_ctx *ctx, float *dverts, float *dsh, float *dopacity,
                              float *dsigma, int accumulate, void *stream);

/* Synchronise `stream`, read the context's counters and device status word.
 * Returns TRI_ERR_CAPACITY on a pair overflow, TRI_ERR_DEVICE_CHECK / TRI_ERR_TIMEOUT on
 * a device-side check, else TRI_OK. `info` may be null. */
tri_status tri_ctx_check(tri_ctx *ctx, tri_ctx_info *info, void *stream);

/* Internal buffers, for tests and diagnostics: copies buffer `which` to host memory
 * `dst` (at most `max_bytes`), synchronously; `*bytes` receives the byte count used.
 *   0: sorted pair tile keys (uint32 [n_pairs])   1: sorted pair item ids (uint32)
 *   2: tile ranges (uint32 [total_tiles][2])       3: item depth keys (uint32 [n_items];
 *      0xffffffff for items that touch no tile; assembled from the visible-item list)
 *   4: item pixel rectangles (uint16 [n_items][4]: x0, y0, x1, y1 inclusive; written
 *      only for items with a non-zero tile count, as are the records of 7)
 *   5: item tile counts (uint32 [n_items]; assembled from the visible-item list)
 *   6: binned pairs (uint64 [n_pairs]: depth key << 32 | item id), grouped by tile;
 *      within a tile in scatter order, except tiles of more than 2048 pairs, whose
 *      ranges hold the sort's intermediate runs
 *   7: per-item render records (float [n_items][16])
 *   8: per-item 2D gradients (float [n_items][16])
 *   9: the forward's tile visiting order (uint32 [total_tiles]): a permutation of the
 *      tiles by descending half-octave bucket of their pair count */
tri_status tri_debug_copy(tri_ctx *ctx, int which, void *dst, size_t max_bytes, size_t *bytes);

/* Failure-detection test hook (the paper has no counterpart). Every wait of a kernel on
 * another CTA (the look-back of the single-pass scans) is bounded: after a limit of
 * device time (1 s) or a cap on its polls it sets the control block's error bit, the
 * kernel finishes with an invalid result (every access stays within its buffers) and
 * tri_ctx_check returns TRI_ERR_TIMEOUT. This call makes the next tri_bin_sort's
 * tile-count scan leave the look-back status word of its CTA `cta` (0-based, 1024
 * tiles each) unset, so that the CTA after it waits on a word nothing sets, and limits
 * that scan's waits to `wait_ns` nanoseconds (0: the default). It applies to one
 * tri_bin_sort; the next tri_preprocess clears the error bit. TRI_ERR_INVALID_ARG for
 * a null context or a negative cta. */
tri_status tri_debug_withhold_scan(tri_ctx *ctx, int32_t cta, uint64_t wait_ns);

/* Window function of the context's next tri_preprocess and of the renders that use its
 * records. TRI_WINDOW_POWER (default) is the paper's Eq. indicator1, I =
 * ReLU(phi(p)/phi(s))^sigma; TRI_WINDOW_SIGMOID is Eq. indicator2, the variant the
 * paper compares against, I = sigmoid(-phi(p)/sigma) with phi the signed distance
 * field in pixels: 1/2 on the triangle's edges and support beyond them (the tight
 * rectangle is the triangle dilated about its incenter until o I falls below 1/255).
 * The backward pass differentiates the chosen window. Resets the context's stage
 * (the next call must be tri_preprocess). TRI_ERR_INVALID_ARG for another value. */
#define TRI_WINDOW_POWER 0
#define TRI_WINDOW_SIGMOID 1
tri_status tri_set_window(tri_ctx *ctx, int window);

/* Compositing order of the context's next tri_preprocess and of the renders that use
 * its records. TRI_SORT_TILE (default) is the paper's: each tile's entries by the
 * camera depth of the triangle's centroid (Supp. "Tile assignment", "depth sorting").
 * TRI_SORT_PIXEL is the per-pixel sort the paper leaves to future work: each pixel's
 * fragments (alpha >= 1/255) by the depth of the triangle's plane along the pixel's
 * ray, ties to the lower triangle id, so intersecting triangles composite correctly.
 * Under TRI_SORT_PIXEL tri_preprocess also writes each item's inverse-depth plane (16 B
 * per item); tri_render_fwd counts every pixel's candidates, reads their total back
 * (a stream synchronisation; under stream capture the buffer sized by an earlier
 * uncaptured forward must suffice, else tri_ctx_check reports an index error), and
 * keeps each pixel's sorted candidates (8 B each) for tri_render_bwd. Not with
 * tri_render_fwd_stats (TRI_ERR_INVALID_ARG) or tri_render_solid (which always uses
 * the tile order). Resets the context's stage. TRI_ERR_INVALID_ARG for another value. */
/* Whether tri_render_fwd counts its evaluated and composited fragments into
 * tri_ctx_info (off by default: the counting costs ~2 % of the forward). Takes effect
 * from the next tri_render_fwd. */
tri_status tri_set_fragment_counting(tri_ctx *ctx, int on);

#define TRI_SORT_TILE 0
#define TRI_SORT_PIXEL 1
tri_status tri_set_sort(tri_ctx *ctx, int sort);

/* Densification moves (Sec. 3.3 "Densification"), in place on scene arrays with room
 * for `capacity` triangles (device, same layouts as tri_scene; verts / sh 16-byte
 * aligned not required). For each of the k distinct indices in sel (device int32):
 *   - area >= tau_small: midpoint subdivision into four triangles that tile it: the
 *     triangle becomes (v0, m01, m02) and (m01, v1, m12), (m02, m12, v2),
 *     (m01, m12, m02) are appended (colour, opacity, sigma copied);
 *   - area < tau_small: a clone translated by noise_scale (a e1 + b e2) is appended,
 *     e1 the unit direction of v1 - v0, e2 = n x e1 (n the unit normal), (a, b) =
 *     noise[2j], noise[2j + 1] (device, caller-drawn standard normals); the triangle
 *     and its clone take opacity 1 - sqrt(1 - o) (the two composite to o).
 * Appended triangles follow the order of sel, starting at index n. *n_out (device
 * int64) receives the new count. The selection policy (the paper samples by opacity
 * and 1 / sigma) is the caller's. Errors: TRI_ERR_CAPACITY when n + 3 k > capacity;
 * out-of-range indices are skipped and reported by tri_ctx_check. Asynchronous. */
tri_status tri_densify(tri_ctx *ctx, float *verts, float *sh, float *opacity, float *sigma, int sh_degree,
                       int64_t n, int64_t capacity, const int32_t *sel, int64_t k, const float *noise,
                       float noise_scale, float tau_small, int64_t *n_out, void *stream);

/* Size regulariser of Sec. 3.4: loss = weight * sum_i 2 / |(v1 - v0) x (v2 - v0)|
 * (weight = beta / n for the mean), written to the device scalar `loss` (nullable),
 * and its gradient added to dverts [n][3][3] (nullable). Triangles with |cross| below
 * 1e-12 contribute nothing. Uses the current device; asynchronous. */
tri_status tri_size_reg(const float *verts, int64_t n, float weight, float *loss, float *dverts,
                        void *stream);

/* Pruning rule of Sec. 3.3 ("Pruning") on the device, over the statistics that
 * tri_render_fwd_stats writes. tri_prune_fold folds one call's [nviews][n] (view-major)
 * max_weight and n_pixels into running per-triangle state: best[n] = max(best,
 * max_weight of every view), views[n] += the number of views with n_pixels >=
 * min_pixels ("rendered ... with more than one pixel": min_pixels = 2). Zero best and
 * views (or keep them from earlier folds) before the first call. tri_prune_mask writes
 * keep[n] = 1 where best >= tau_prune and views >= min_views ("at least twice":
 * min_views = 2), else 0. All arrays are caller-owned device memory (float32, int32,
 * uint8); both calls are asynchronous on `stream`, use the current device, allocate
 * nothing, and return TRI_ERR_INVALID_ARG for a negative size or a null array (when
 * there is work: n > 0 and, for the fold, nviews > 0). */
tri_status tri_prune_fold(const float *max_weight, const int32_t *n_pixels, int nviews, int64_t n, int min_pixels,
                          float *best, int32_t *views, void *stream);
tri_status tri_prune_mask(const float *best, const int32_t *views, int64_t n, float tau_prune, int min_views,
                          uint8_t *keep, void *stream);

/* L1 photometric loss helper (Sec. 3.3 lists L1 among the loss terms): loss = mean
 * |image - target| over n values, written to the device scalar `loss` (may be null),
 * and dL/dimage = sign(image - target) / n into `dL_dimage`. */
tri_status tri_loss_l1(const float *image, const float *target, int64_t n, float *dL_dimage,
                       float *loss, void *stream);

/* ---------------------------------------------------------------------------------
 * Allocation-free forward render. The paper has no counterpart: this is a deployment
 * aid for callers that cannot allocate device memory (a plugin inside an application
 * that owns the device allocator, a real-time loop that reserved every byte up front).
 * It runs the steps of tri_preprocess + tri_bin_sort + tri_render_fwd for one view with
 * all workspace carved from one fixed array in device global memory declared by the
 * library (37,730,816 bytes = 36.0 MiB, held by every GPU that loads the library until
 * the process exits); it calls no cudaMalloc, cudaFree or other allocating routine.
 * Having no context, it always uses the paper's window (Eq. indicator1) and the
 * per-tile centre-depth order: tri_set_window and tri_set_sort do not apply to it.
 * Limits: scene->n <= TRI_NOALLOC_MAX_TRIANGLES and width * height <=
 * TRI_NOALLOC_MAX_PIXELS (else TRI_ERR_CAPACITY, nothing runs); pairs beyond
 * TRI_NOALLOC_MAX_PAIRS are dropped and reported in *device_status.
 * Outputs: image [3][H][W]; T_final / n_contrib [H][W] (nullable); device_status (a
 * device int32, nullable) receives bit 0 = a bounded wait gave up, bit 1 = an index
 * check failed, bit 2 = pair overflow. Asynchronous on `stream`.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture. All
 * calls share the array and it keeps the last call's contents: each call clears what
 * must start at zero, and calls that overlap on the GPU (other streams or threads)
 * race on it. */
#define TRI_NOALLOC_MAX_TRIANGLES 65536
#define TRI_NOALLOC_MAX_PAIRS 524288
#define TRI_NOALLOC_MAX_PIXELS (2048 * 1088)
tri_status tri_render_fwd_noalloc(const tri_scene *scene, const tri_camera *cam, float *image,
                                  float *T_final, int32_t *n_contrib, int32_t *device_status,
                                  void *stream);

/* ---------------------------------------------------------------------------------
 * Serving: resident scenes, admission by device memory, continuous batching of camera
 * requests of mixed resolutions into batched launches (one batched preprocess + sort
 * and one persistent render over all (request, tile) work items per batch), completion
 * by CUDA event, p50/p99 latency.
 * --------------------------------------------------------------------------------- */
typedef struct tri_serve tri_serve;

typedef struct {
    size_t mem_budget_bytes;   /* scenes + batch workspaces; 0 = 80 % of free memory */
    int32_t max_batch;         /* views per batch (>= 1) */
    int32_t max_width, max_height;
    int32_t slots;             /* batches in flight (>= 1); each has its own stream */
    int32_t timeout_ms;        /* per-request deadline (0 = none) */
    int32_t use_graphs;        /* capture each slot's launch sequence in a CUDA graph */
    int32_t batch_window_us;   /* wait this long for more requests before launching */
    int32_t graph_after;       /* capture a composition's graph once it has run eagerly this
                                  many times (<= 1: on its first run) */
} tri_serve_opts;

typedef struct {
    uint64_t submitted, completed, rejected, timed_out, batches;
    double p50_ms, p99_ms, max_ms, mean_ms;
    double fps;                /* completed frames per second of wall time */
    double mean_batch;         /* views per batch */
    size_t bytes_resident;     /* scene bytes held */
    size_t bytes_workspace;    /* batch workspaces held */
    uint64_t graph_replays;    /* batches launched by replaying a captured graph */
    uint64_t graph_captures;   /* graphs captured and instantiated */
    uint64_t eager_batches;    /* batches launched call by call */
    uint64_t reruns;           /* batches run again after a pair-list overflow */
    uint64_t reallocs;         /* workspace buffers (re)allocated by the slots */
    double eager_ms;           /* dispatcher time spent launching eager batches */
    double capture_ms;         /* dispatcher time spent capturing and instantiating */
    double queue_p99_ms;       /* p99 of submit -> launch of the completed requests */
} tri_serve_stats_t;

/* Create a server on `device`. Starts one dispatcher thread; the slots' streams take
 * the device's highest stream priority. */
tri_status tri_serve_create(tri_serve **out, const tri_serve_opts *opts, int device);

/* Copy a scene into server-owned device memory (the scene's pointers may be host or
 * device memory). Returns TRI_ERR_CAPACITY when it does not fit the budget. */
tri_status tri_serve_add_scene(tri_serve *srv, const tri_scene *scene, int32_t *scene_id);

/* Drop a scene once no queued or running request uses it. */
tri_status tri_serve_remove_scene(tri_serve *srv, int32_t scene_id);

/* Queue a request: render `cam` of `scene_id` into device buffer `out_image`
 * [3][H][W] (caller-owned, must stay valid until the ticket completes). Never blocks
 * on the GPU. Returns TRI_ERR_CAPACITY when the resolution exceeds max_width/height. */
tri_status tri_serve_submit(tri_serve *srv, int32_t scene_id, const tri_camera *cam,
                            float *out_image, uint64_t *ticket);

/* Finished tickets since the last poll (up to max); the status of each is in
 * `status` (may be null): TRI_OK or TRI_ERR_TIMEOUT. */
tri_status tri_serve_poll(tri_serve *srv, uint64_t *done, int32_t *status, int32_t max,
                          int32_t *ndone);

/* Block the host until `ticket` completes or `timeout_ms` passes (TRI_ERR_TIMEOUT). */
tri_status tri_serve_wait(tri_serve *srv, uint64_t ticket, int32_t timeout_ms);

/* Latency percentiles and counters over completed requests. */
tri_status tri_serve_stats(tri_serve *srv, tri_serve_stats_t *stats);

/* Start a new statistics window: clears latencies and counters (requests in flight
 * still complete normally and count in the new window). */
tri_status tri_serve_reset_stats(tri_serve *srv);

/* Stop the dispatcher after the queued work drains, free everything. */
void tri_serve_destroy(tri_serve *srv);

#ifdef __cplusplus
}
#endif

#endif /* TRISPLAT_H */
