// Allocation-free forward render: tri_render_fwd_noalloc (declared in trisplat.h).
//
// Some callers cannot allocate device memory at all: a renderer plugin living inside a
// host application whose device memory is owned by another allocator, a real-time
// loop that has reserved every byte up front, or code running while allocation is
// forbidden. For them this entry point runs the same kernels as tri_preprocess +
// tri_bin_sort + tri_render_fwd on one view, with every piece of workspace carved from
// one fixed array in device global memory that this file declares; it calls no
// cudaMalloc, cudaFree or other allocating routine. The caller passes the scene, the
// camera and the output image (and, optionally, per-pixel outputs). It takes no
// context, so it always renders with the paper's window (Eq. indicator1) and the
// per-tile centre-depth order, whatever tri_set_window / tri_set_sort set elsewhere.
//
// The array has a fixed size (37,730,816 bytes, 36.0 MiB), so the scene, pair list and image have
// fixed maxima (TRI_NOALLOC_MAX_* in trisplat.h); larger inputs are rejected with
// TRI_ERR_CAPACITY before anything runs. Every GPU that loads this library holds the
// array until the process exits. All calls share it and it keeps the contents of the
// last call, so each call clears what must start at zero, and calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it.
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "trisplat.h"

using namespace ts;

namespace {

constexpr int64_t NA_TRIS = TRI_NOALLOC_MAX_TRIANGLES;
constexpr int64_t NA_PAIRS = TRI_NOALLOC_MAX_PAIRS;
constexpr int64_t NA_PIXELS = TRI_NOALLOC_MAX_PIXELS;
constexpr int64_t NA_TILES = (NA_PIXELS / 256) + 4096;   // covers any shape within the pixel limit
constexpr int64_t NA_DEPTH_TILE = 1024;                   // smallest onesweep tile
constexpr int64_t NA_TILE_PASSES = 3;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets inside the scratch array
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_VIEW = OFF_CTL + align256(sizeof(Ctl));
constexpr size_t OFF_OUT = OFF_VIEW + align256(sizeof(ViewDev));
constexpr size_t OFF_RECS = OFF_OUT + align256(sizeof(ViewOut));
constexpr size_t OFF_NTILES = OFF_RECS + align256(sizeof(Rec) * NA_TRIS);
constexpr size_t OFF_RECTS = OFF_NTILES + align256(4 * NA_TRIS);
constexpr size_t OFF_DKEYS = OFF_RECTS + align256(8 * NA_TRIS);
constexpr size_t OFF_CK0 = OFF_DKEYS + align256(4 * NA_TRIS);
constexpr size_t OFF_CK1 = OFF_CK0 + align256(4 * NA_TRIS);
constexpr size_t OFF_CV0 = OFF_CK1 + align256(4 * NA_TRIS);
constexpr size_t OFF_CV1 = OFF_CV0 + align256(4 * NA_TRIS);
constexpr size_t OFF_PK0 = OFF_CV1 + align256(4 * NA_TRIS);
constexpr size_t OFF_PK1 = OFF_PK0 + align256(4 * NA_PAIRS);
constexpr size_t OFF_PV0 = OFF_PK1 + align256(4 * NA_PAIRS);
constexpr size_t OFF_PV1 = OFF_PV0 + align256(4 * NA_PAIRS);
constexpr size_t OFF_RANGES = OFF_PV1 + align256(4 * NA_PAIRS);
constexpr size_t OFF_TMAX = OFF_RANGES + align256(8 * NA_TILES);
constexpr size_t OFF_TFIN = OFF_TMAX + align256(4 * GROUPS_PER_TILE * NA_TILES);
constexpr size_t OFF_NCON = OFF_TFIN + align256(4 * NA_PIXELS);
constexpr size_t DEPTH_WORDS = (NA_TRIS + NA_DEPTH_TILE - 1) / NA_DEPTH_TILE * 256;
constexpr size_t PAIR_WORDS = (NA_PAIRS + NA_DEPTH_TILE - 1) / NA_DEPTH_TILE * 256;
constexpr size_t OFF_STDEPTH = OFF_NCON + align256(4 * NA_PIXELS);
constexpr size_t OFF_STEMIT = OFF_STDEPTH + align256(4 * 4 * DEPTH_WORDS);
constexpr size_t OFF_STPAIRS = OFF_STEMIT + align256(4 * (NA_TRIS / 256 + 2));
constexpr size_t SCRATCH_BYTES = OFF_STPAIRS + align256(4 * NA_TILE_PASSES * PAIR_WORDS);
// the size quoted in trisplat.h and above; a change of the limits or of the layout must
// update both
static_assert(SCRATCH_BYTES == 37730816, "allocation-free workspace size differs from the documented size");

// The fixed workspace. Host code must not use this name as an address: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_ptr[64] = {};   // per device ordinal

// Copies the control block's error bits and the pair-overflow flag to the caller's
// status word: bit 0 a bounded wait gave up, bit 1 an index check failed, bit 2 the
// pair list exceeded TRI_NOALLOC_MAX_PAIRS (pairs were dropped).
__global__ void status_kernel(const Ctl *ctl, int32_t *out) {
    if (threadIdx.x == 0) *out = (int32_t)((ctl->error & 3u) | (ctl->overflow ? 4u : 0u));
}

// Writes the one-view tables into the scratch array from kernel parameters, so that
// no host -> device copy (and no driver staging of pageable memory) is needed.
__global__ void write_tables_kernel(ViewDev v, ViewOut o, ViewDev *dv, ViewOut *dout) {
    if (threadIdx.x == 0) {
        *dv = v;
        *dout = o;
    }
}

tri_status scratch_of(int device, unsigned char **out) {
    if (device < 0 || device >= 64) return TRI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TRI_ERR_CUDA;
        }
        g_scratch_ptr[device] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[device];
    return TRI_OK;
}

int digits_for(int tiles) {
    int bits = 0;
    while (bits < 31 && (1ll << bits) < (int64_t)tiles) ++bits;
    const int d = (bits + 7) / 8;
    return d < 1 ? 1 : d;
}

}  // namespace

extern "C" tri_status tri_render_fwd_noalloc(const tri_scene *scene, const tri_camera *cam, float *image,
                                             float *T_final, int32_t *n_contrib, int32_t *device_status,
                                             void *stream) {
    if (!scene || !cam || !image) return TRI_ERR_INVALID_ARG;
    if (scene->n < 0 || scene->sh_degree < 0 || scene->sh_degree > 3) return TRI_ERR_INVALID_ARG;
    if (scene->n > 0 && (!scene->verts || !scene->sh || !scene->opacity || !scene->sigma)) return TRI_ERR_INVALID_ARG;
    if (((uintptr_t)scene->verts & 15) || ((uintptr_t)scene->sh & 15)) return TRI_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 || cam->height > 65535) return TRI_ERR_INVALID_ARG;
    if (scene->n > NA_TRIS || (int64_t)cam->width * cam->height > NA_PIXELS) return TRI_ERR_CAPACITY;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return TRI_ERR_CUDA;
    unsigned char *base = nullptr;
    tri_status s = scratch_of(device, &base);
    if (s != TRI_OK) return s;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return TRI_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    ViewDev V;
    memcpy(V.R, cam->R, sizeof V.R);
    memcpy(V.t, cam->t, sizeof V.t);
    V.fx = cam->fx; V.fy = cam->fy; V.cx = cam->cx; V.cy = cam->cy;
    memcpy(V.bg, cam->bg, sizeof V.bg);
    for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int i = 0; i < 3; ++i) acc -= (double)cam->R[i * 3 + j] * (double)cam->t[i];
        V.campos[j] = (float)acc;
    }
    V.W = cam->width; V.H = cam->height;
    V.tiles_x = (V.W + TILE - 1) / TILE;
    V.tiles_y = (V.H + TILE - 1) / TILE;
    V.tile_base = 0;
    V.pix_base = 0;
    const int tiles = V.tiles_x * V.tiles_y;
    if (tiles > NA_TILES) return TRI_ERR_CAPACITY;
    const int tile_passes = digits_for(tiles);
    const int64_t M = scene->n;

    Ctl *ctl = (Ctl *)(base + OFF_CTL);
    ViewDev *dview = (ViewDev *)(base + OFF_VIEW);
    ViewOut *dout = (ViewOut *)(base + OFF_OUT);
    Rec *recs = (Rec *)(base + OFF_RECS);
    uint32_t *ntiles = (uint32_t *)(base + OFF_NTILES);
    ushort4 *rects = (ushort4 *)(base + OFF_RECTS);
    uint32_t *dkeys = (uint32_t *)(base + OFF_DKEYS);
    uint32_t *ck[2] = {(uint32_t *)(base + OFF_CK0), (uint32_t *)(base + OFF_CK1)};
    uint32_t *cv[2] = {(uint32_t *)(base + OFF_CV0), (uint32_t *)(base + OFF_CV1)};
    uint32_t *pk[2] = {(uint32_t *)(base + OFF_PK0), (uint32_t *)(base + OFF_PK1)};
    uint32_t *pv[2] = {(uint32_t *)(base + OFF_PV0), (uint32_t *)(base + OFF_PV1)};
    uint2 *ranges = (uint2 *)(base + OFF_RANGES);
    uint32_t *tmax = (uint32_t *)(base + OFF_TMAX);
    float *tfin = (float *)(base + OFF_TFIN);
    int32_t *ncon = (int32_t *)(base + OFF_NCON);
    uint32_t *st_depth = (uint32_t *)(base + OFF_STDEPTH);
    uint32_t *st_emit = (uint32_t *)(base + OFF_STEMIT);
    uint32_t *st_pairs = (uint32_t *)(base + OFF_STPAIRS);

#define NA_CK(call)                                   \
    do {                                              \
        if ((call) != cudaSuccess) {                  \
            cudaGetLastError();                       \
            return TRI_ERR_CUDA;                      \
        }                                             \
    } while (0)

    // what must start at zero: the control block and every look-back status word
    NA_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
    NA_CK(cudaMemsetAsync(st_depth, 0, 4 * 4 * DEPTH_WORDS, st));
    NA_CK(cudaMemsetAsync(st_emit, 0, 4 * (NA_TRIS / 256 + 2), st));
    NA_CK(cudaMemsetAsync(st_pairs, 0, 4 * (size_t)tile_passes * PAIR_WORDS, st));
    NA_CK(cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)tiles, st));
    write_tables_kernel<<<1, 32, 0, st>>>(V, ViewOut{image, nullptr}, dview, dout);
    NA_CK(cudaGetLastError());

    if (M > 0) {
        PreArgs a;
        a.verts = scene->verts; a.sh = scene->sh; a.opacity = scene->opacity; a.sigma = scene->sigma;
        a.n = M; a.sh_degree = scene->sh_degree;
        a.views = dview; a.nviews = 1;
        a.recs = recs; a.ntiles = ntiles; a.rects = rects; a.dkeys = dkeys; a.ctl = ctl;
        a.depth_hist = 1;
        launch_preprocess_fwd(a, st);
        NA_CK(cudaGetLastError());
        // depth sort of all items (tile size fixed to the smallest, as the status area assumes)
        int cur = 1;
        for (int p = 0; p < 4; ++p) {
            const uint32_t *kin = p == 0 ? dkeys : ck[cur ^ 1];
            const uint32_t *vin = p == 0 ? nullptr : cv[cur ^ 1];
            launch_onesweep_pass(kin, vin, ck[cur], cv[cur], nullptr, (uint32_t)M, ctl->depth_hist[p],
                                 st_depth + p * DEPTH_WORDS, &ctl->pass_counter[p], 8 * p, &ctl->error,
                                 (int)NA_DEPTH_TILE, sms, st);
            cur ^= 1;
        }
        EmitArgs e;
        e.sorted_items = cv[0]; e.ntiles = ntiles; e.rects = rects; e.views = dview; e.nviews = 1; e.n = M;
        e.pkeys = pk[0]; e.pvals = pv[0]; e.cap = (uint32_t)NA_PAIRS; e.tile_passes = tile_passes;
        e.lb_status = st_emit; e.ctl = ctl;
        launch_emit(e, M, st);
        cur = 0;
        for (int p = 0; p < tile_passes; ++p) {
            launch_onesweep_pass(pk[cur], pv[cur], pk[cur ^ 1], pv[cur ^ 1], &ctl->n_pairs_used, (uint32_t)NA_PAIRS,
                                 ctl->tile_hist[p], st_pairs + p * PAIR_WORDS, &ctl->pass_counter[4 + p], 8 * p,
                                 &ctl->error, (int)NA_DEPTH_TILE, sms, st);
            cur ^= 1;
        }
        launch_ranges(pk[cur], &ctl->n_pairs_used, ranges, (uint32_t)tiles, &ctl->error, sms * 8, st);
        NA_CK(cudaGetLastError());
        RenderArgs r;
        r.views = dview; r.outs = dout; r.nviews = 1; r.total_tiles = tiles; r.ranges = ranges;
        r.items = pv[cur]; r.recs = recs; r.rects = rects; r.T_final = tfin; r.n_contrib = ncon; r.tile_max = tmax;
        r.grad2d = nullptr; r.n_items = (uint32_t)M; r.ctl = ctl; r.kmask = nullptr; r.stat_w = r.stat_n = nullptr;
        launch_render_fwd(r, sms, st);
    } else {
        // no triangles: one tile pass over zero pairs still renders the background
        RenderArgs r;
        r.views = dview; r.outs = dout; r.nviews = 1; r.total_tiles = tiles; r.ranges = ranges;
        r.items = pv[0]; r.recs = recs; r.rects = rects; r.T_final = tfin; r.n_contrib = ncon; r.tile_max = tmax;
        r.grad2d = nullptr; r.n_items = 1; r.ctl = ctl; r.kmask = nullptr; r.stat_w = r.stat_n = nullptr;
        launch_render_fwd(r, sms, st);
    }
    NA_CK(cudaGetLastError());
    const size_t np = (size_t)V.W * V.H;
    if (T_final) NA_CK(cudaMemcpyAsync(T_final, tfin, 4 * np, cudaMemcpyDeviceToDevice, st));
    if (n_contrib) NA_CK(cudaMemcpyAsync(n_contrib, ncon, 4 * np, cudaMemcpyDeviceToDevice, st));
    if (device_status) {
        status_kernel<<<1, 32, 0, st>>>(ctl, device_status);
        NA_CK(cudaGetLastError());
    }
#undef NA_CK
    return TRI_OK;
}
