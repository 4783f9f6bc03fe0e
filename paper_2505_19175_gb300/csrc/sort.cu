// Binning and sorting of the triangle-splat renderer (Supp. "Tile assignment",
// "Depth sorting": triangles are duplicated into the tiles their tight rectangle
// touches and composited in order of their centre depth).
//
// The result equals a stable sort of the 64-bit keys (tile << 32 | depth bits)
// emitted in item order. It is reached as an LSD radix sort whose low (depth) digits
// are sorted on the item list before duplication, since every pair of an item shares
// its depth:
//   1. onesweep passes over the visible items' 32-bit depth keys (4 x 8 bits);
//   2. emission of (tile, item) pairs in depth order (single-pass scan of the tile
//      counts with decoupled look-back; coalesced, load-balanced writes), with the
//      digit histograms of the tile keys;
//   3. onesweep passes over the pairs' tile keys (ceil(log2 tiles / 8) digits);
//   4. per-tile [start, end) ranges.
// A onesweep pass ranks keys stably inside a CTA tile with warp-level match (warp
// multisplit) and obtains the tile's global digit offsets by decoupled look-back, so
// each pass reads and writes the keys once.
#include "kernels.h"

namespace ts {

template <int SORT_IPT>
__global__ void __launch_bounds__(SORT_THREADS)
onesweep_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                uint32_t *__restrict__ vout, const uint32_t *count_ptr, uint32_t cap, const uint32_t *hist,
                uint32_t *status, uint32_t *tile_counter, int shift, uint32_t *err) {
    constexpr int SORT_TILE = SORT_THREADS * SORT_IPT;
    __shared__ uint32_t s_keys[SORT_TILE];
    __shared__ uint32_t s_vals[SORT_TILE];
    __shared__ uint32_t s_whist[SORT_THREADS / 32][256];
    __shared__ uint32_t s_bucket[256];
    __shared__ uint32_t s_dstart[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t n = count_ptr ? min(*count_ptr, cap) : cap;
    const uint32_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
    {
        uint32_t tot;
        s_bucket[tid] = block_excl_scan(hist[tid], s_tmp, tot);
    }
    const unsigned lt = lanemask_lt();
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
        for (int k = tid; k < (SORT_THREADS / 32) * 256; k += SORT_THREADS) (&s_whist[0][0])[k] = 0u;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t base = tile * SORT_TILE;
        const uint32_t wbase = base + w * (SORT_IPT * 32);
        uint32_t keys[SORT_IPT], vals[SORT_IPT], rank[SORT_IPT];
#pragma unroll
        for (int j = 0; j < SORT_IPT; ++j) {
            const uint32_t idx = wbase + j * 32 + lane;
            const bool valid = idx < n;
            const uint32_t key = valid ? kin[idx] : 0u;
            const uint32_t val = valid ? (vin ? vin[idx] : idx) : 0u;
            const uint32_t d = valid ? (key >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader && valid) {
                old = s_whist[w][d];
                s_whist[w][d] = old + __popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[j] = old + __popc(peers & lt);
            keys[j] = key;
            vals[j] = val;
            __syncwarp();
        }
        __syncthreads();
        // digit `tid`: exclusive offsets across warps, tile total, look-back
        uint32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < SORT_THREADS / 32; ++ww) {
            const uint32_t c = s_whist[ww][tid];
            s_whist[ww][tid] = tot;
            tot += c;
        }
        uint32_t *st = status + (size_t)tile * 256 + tid;
        uint32_t excl = 0;
        if (tile == 0) {
            st_relaxed(st, LB_PREFIX | tot);
        } else {
            st_relaxed(st, LB_AGG | tot);
            // walk back through the predecessors of this digit, four at a time
            int k = (int)tile - 1;
            bool found = false;
            while (!found) {
                uint32_t w4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w4[q] = (k - q >= 0) ? wait_status(status + (size_t)(k - q) * 256 + tid, err) : LB_PREFIX;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!found) {
                        excl += w4[q] & LB_MASK;
                        found = (w4[q] >> 30) == 2u;
                    }
                }
                k -= 4;
            }
            st_relaxed(st, LB_PREFIX | ((excl + tot) & LB_MASK));
        }
        s_gbase[tid] = s_bucket[tid] + excl;
        uint32_t all;
        s_dstart[tid] = block_excl_scan(tot, s_tmp, all);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SORT_IPT; ++j) {
            const uint32_t idx = wbase + j * 32 + lane;
            if (idx < n) {
                const uint32_t d = (keys[j] >> shift) & 255u;
                const uint32_t lp = s_dstart[d] + s_whist[w][d] + rank[j];
                s_keys[lp] = keys[j];
                s_vals[lp] = vals[j];
            }
        }
        __syncthreads();
        const uint32_t tcount = min((uint32_t)SORT_TILE, n - base);
        for (uint32_t i = tid; i < tcount; i += SORT_THREADS) {
            const uint32_t key = s_keys[i];
            const uint32_t d = (key >> shift) & 255u;
            const uint32_t pos = s_gbase[d] + (i - s_dstart[d]);
            if (pos < n) {
                kout[pos] = key;
                vout[pos] = s_vals[i];
            } else {
                atomicOr(err, ERR_INDEX);
            }
        }
        __syncthreads();
    }
}

int onesweep_tile(uint32_t cap, int sm_count) {
    const uint64_t target = (uint64_t)sm_count * 4;   // tiles wanted for a full machine
    if ((uint64_t)cap >= target * SORT_THREADS * SORT_IPT_MAX) return SORT_THREADS * SORT_IPT_MAX;
    if ((uint64_t)cap >= target * SORT_THREADS * 8) return SORT_THREADS * 8;
    return SORT_THREADS * 4;
}

template <int IPT>
static void launch_ipt(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                       const uint32_t *count, uint32_t cap, const uint32_t *hist, uint32_t *status,
                       uint32_t *tile_counter, int shift, uint32_t *err, int sm_count, cudaStream_t st) {
    static int occ = -1;
    if (occ < 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, onesweep_kernel<IPT>, SORT_THREADS, 0) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    const int64_t tiles = ((int64_t)cap + SORT_THREADS * IPT - 1) / (SORT_THREADS * IPT);
    int64_t g = (int64_t)sm_count * occ;
    if (tiles < g) g = tiles;
    if (g < 1) g = 1;
    onesweep_kernel<IPT><<<(unsigned)g, SORT_THREADS, 0, st>>>(kin, vin, kout, vout, count, cap, hist, status,
                                                               tile_counter, shift, err);
}

void launch_onesweep_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                          const uint32_t *count, uint32_t cap, const uint32_t *hist, uint32_t *status,
                          uint32_t *tile_counter, int shift, uint32_t *err, int tile, int sm_count,
                          cudaStream_t st) {
    if (tile == SORT_THREADS * SORT_IPT_MAX)
        launch_ipt<SORT_IPT_MAX>(kin, vin, kout, vout, count, cap, hist, status, tile_counter, shift, err, sm_count, st);
    else if (tile == SORT_THREADS * 8)
        launch_ipt<8>(kin, vin, kout, vout, count, cap, hist, status, tile_counter, shift, err, sm_count, st);
    else
        launch_ipt<4>(kin, vin, kout, vout, count, cap, hist, status, tile_counter, shift, err, sm_count, st);
}

// ---------------------------------------------------------------------------------
// pair emission
// ---------------------------------------------------------------------------------
constexpr int EMIT_THREADS = 256;

__global__ void __launch_bounds__(EMIT_THREADS) emit_kernel(EmitArgs a) {
    __shared__ uint32_t s_off[EMIT_THREADS];
    __shared__ uint32_t s_item[EMIT_THREADS];
    __shared__ uint32_t s_base_tile[EMIT_THREADS];   // global id of the rectangle's first tile
    __shared__ uint32_t s_wx[EMIT_THREADS];          // (rect width in tiles, view tiles_x)
    __shared__ float s_iw[EMIT_THREADS];             // 1 / rect width
    __shared__ uint32_t s_hist[3][256];
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_cta, s_base;
    __shared__ int2 s_vt[MAX_VIEWS];   // (tiles_x, tile_base)

    const int tid = threadIdx.x;
    if (tid == 0) s_cta = atomicAdd(&a.ctl->cta_counter[1], 1u);
    for (int k = tid; k < 3 * 256; k += EMIT_THREADS) (&s_hist[0][0])[k] = 0u;
    for (int k = tid; k < a.nviews; k += EMIT_THREADS) s_vt[k] = make_int2(a.views[k].tiles_x, a.views[k].tile_base);
    __syncthreads();
    const uint32_t K = a.ctl->n_visible;
    const uint32_t cta = s_cta;
    if ((uint64_t)cta * EMIT_THREADS >= K) return;
    const uint32_t j = cta * EMIT_THREADS + tid;
    const bool valid = j < K;
    uint32_t item = valid ? a.sorted_items[j] : 0u;
    if ((int64_t)item >= a.n * a.nviews) {
        atomicOr(&a.ctl->error, ERR_INDEX);
        item = 0;
    }
    const uint32_t nt = valid ? a.ntiles[item] : 0u;
    uint32_t total;
    const uint32_t local = block_excl_scan(nt, s_tmp, total);
    s_off[tid] = local;
    s_item[tid] = item;
    {
        const ushort4 pr = valid ? a.rects[item] : make_ushort4(0, 0, 0, 0);
        const uint32_t tx0 = pr.x / TILE, ty0 = pr.y / TILE, wdt = pr.z / TILE - tx0 + 1;
        const int2 vt = s_vt[a.nviews > 1 ? (int)(item / (uint32_t)a.n) : 0];
        s_base_tile[tid] = (uint32_t)vt.y + ty0 * (uint32_t)vt.x + tx0;
        s_wx[tid] = (wdt << 16) | (uint32_t)vt.x;
        s_iw[tid] = 1.0f / (float)wdt;
    }
    if (tid < 32) {
        const uint32_t b = warp_lookback_excl(a.lb_status, cta, total, &a.ctl->error);
        if (tid == 0) s_base = b;
    }
    __syncthreads();
    const uint32_t base = s_base;
    if (tid == 0 && cta == (K - 1) / EMIT_THREADS) {
        const uint64_t np = (uint64_t)base + total;
        a.ctl->n_pairs = (uint32_t)(np < 0xffffffffull ? np : 0xffffffffull);
        a.ctl->n_pairs_used = (uint32_t)(np < a.cap ? np : a.cap);
        a.ctl->overflow = np > a.cap ? 1u : 0u;
    }
    for (uint32_t o = tid; o < total; o += EMIT_THREADS) {
        // owner: the last thread whose offset is <= o
        int lo = 0, hi = EMIT_THREADS - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= o) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t k = o - s_off[lo];
        const uint32_t wx = s_wx[lo], wdt = wx >> 16, tiles_x = wx & 0xffffu;
        // row = k / wdt: an FP32 estimate (relative error ~2^-23 of the row, so off by at
        // most one for large rectangles), then corrected to the exact quotient
        uint32_t row = (uint32_t)(((float)k + 0.5f) * s_iw[lo]);
        if (row * wdt > k) --row;
        else if ((row + 1) * wdt <= k) ++row;
        const uint32_t col = k - row * wdt;
        const uint32_t it = s_item[lo];
        const uint32_t tile = s_base_tile[lo] + row * tiles_x + col;
        const uint32_t pos = base + o;
        if (pos < a.cap) {
            a.pkeys[pos] = tile;
            a.pvals[pos] = it;
            for (int p = 0; p < a.tile_passes; ++p) atomicAdd(&s_hist[p][(tile >> (8 * p)) & 255u], 1u);
        }
    }
    __syncthreads();
    for (int k = tid; k < a.tile_passes * 256; k += EMIT_THREADS) {
        const uint32_t c = (&s_hist[0][0])[k];
        if (c) atomicAdd(&(&a.ctl->tile_hist[0][0])[k], c);
    }
}

void launch_emit(const EmitArgs &a, int64_t max_items, cudaStream_t st) {
    const int64_t grid = (max_items + EMIT_THREADS - 1) / EMIT_THREADS;
    if (grid > 0) emit_kernel<<<(unsigned)grid, EMIT_THREADS, 0, st>>>(a);
}

// ---------------------------------------------------------------------------------
// tile ranges
// ---------------------------------------------------------------------------------
__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const uint32_t *count_ptr, uint2 *ranges,
                              uint32_t total_tiles, uint32_t *err) {
    const uint32_t n = *count_ptr;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (k >= total_tiles) {
            atomicOr(err, ERR_INDEX);
            continue;
        }
        if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = i + 1;
    }
}

void launch_ranges(const uint32_t *keys, const uint32_t *count, uint2 *ranges, uint32_t total_tiles, uint32_t *err,
                   int grid, cudaStream_t st) {
    ranges_kernel<<<grid, 256, 0, st>>>(keys, count, ranges, total_tiles, err);
}

}  // namespace ts
