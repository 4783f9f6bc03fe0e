// Tile binning of (tile, item) pairs and per-tile depth order (Supp. "Tile assignment"
// and "Depth sorting": every triangle is listed in each tile its tight rectangle
// touches, and each tile's list is ordered by the triangles' centre depth).
//
// The result equals a stable sort of the pairs by the 64-bit key (tile << 32 | depth
// bits) when the pairs are emitted in item order: within a tile, entries are ordered
// by (depth key, item id). It is reached without a global sort:
//   1. bin_count:   per-tile pair counts (warp-aggregated atomics);
//   2. bin_scan:    exclusive scan of the counts -> tile ranges and write cursors;
//   3. bin_scatter: each pair takes a slot in its tile's range (order within the
//                   range is arbitrary at this point);
//   4. tile_sort:   each tile's range is sorted by (depth key << 32 | item) in shared
//                   memory (bitonic network; ranges longer than TSORT_CAP are sorted
//                   in shared-memory chunks and merged in global memory).
// Keys are unique (item ids are), so the order is deterministic although the scatter
// is not.
#include "kernels.h"

namespace ts {

constexpr int BIN_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int TSORT_THREADS = 256;
constexpr int TSORT_CAP = 2048;           // entries a tile sorts in one shared-memory pass
constexpr int MERGE_PER_THREAD = 8;

// Per-item expansion of a CTA's 256 items into their (item, tile) pairs. Calls
// f(valid, item, tile) for every pair, in rounds of BIN_THREADS pairs in which all
// threads of the block take part (so that f may use warp collectives).
template <class F>
__device__ __forceinline__ void for_each_pair(const BinArgs &a, F &&f) {
    __shared__ uint32_t s_off[BIN_THREADS];
    __shared__ uint32_t s_item[BIN_THREADS];
    __shared__ uint32_t s_base_tile[BIN_THREADS];   // global id of the rectangle's first tile
    __shared__ uint32_t s_wx[BIN_THREADS];          // (rect width in tiles << 16) | view tiles_x
    __shared__ float s_iw[BIN_THREADS];             // 1 / rect width
    __shared__ uint32_t s_tmp[33];
    __shared__ int2 s_vt[MAX_VIEWS];                // (tiles_x, tile_base)
    const int tid = threadIdx.x;
    for (int k = tid; k < a.nviews; k += BIN_THREADS) s_vt[k] = make_int2(a.views[k].tiles_x, a.views[k].tile_base);
    __syncthreads();
    for (int64_t m0 = (int64_t)blockIdx.x * BIN_THREADS; m0 < a.n_items; m0 += (int64_t)gridDim.x * BIN_THREADS) {
        const int64_t m = m0 + tid;
        const bool valid = m < a.n_items;
        const uint32_t nt = valid ? a.ntiles[m] : 0u;
        uint32_t total;
        const uint32_t local = block_excl_scan(nt, s_tmp, total);
        s_off[tid] = local;
        s_item[tid] = (uint32_t)m;
        if (nt) {
            const ushort4 pr = a.rects[m];
            const uint32_t tx0 = pr.x / TILE, ty0 = pr.y / TILE, wdt = pr.z / TILE - tx0 + 1;
            const int2 vt = s_vt[a.nviews > 1 ? (int)(m / a.n) : 0];
            s_base_tile[tid] = (uint32_t)vt.y + ty0 * (uint32_t)vt.x + tx0;
            s_wx[tid] = (wdt << 16) | (uint32_t)vt.x;
            s_iw[tid] = 1.0f / (float)wdt;
        }
        __syncthreads();
        for (uint32_t r0 = 0; r0 < total; r0 += BIN_THREADS) {
            const uint32_t o = r0 + tid;
            const bool ok = o < total;
            uint32_t item = 0, tile = 0xffffffffu;
            if (ok) {
                // owner: the last thread whose offset is <= o (threads with no tile
                // share their successor's offset and lose the search)
                int lo = 0, hi = BIN_THREADS - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= o) lo = mid;
                    else hi = mid - 1;
                }
                const uint32_t k = o - s_off[lo];
                const uint32_t wx = s_wx[lo], wdt = wx >> 16, tiles_x = wx & 0xffffu;
                uint32_t row = (uint32_t)(((float)k + 0.5f) * s_iw[lo]);
                if (row * wdt > k) --row;                 // guard the FP32 quotient
                else if ((row + 1) * wdt <= k) ++row;
                const uint32_t col = k - row * wdt;
                item = s_item[lo];
                tile = s_base_tile[lo] + row * tiles_x + col;
                if (tile >= (uint32_t)a.total_tiles) {
                    atomicOr(&a.ctl->error, ERR_INDEX);
                    tile = 0xffffffffu;
                }
            }
            f(ok && tile != 0xffffffffu, item, tile);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BIN_THREADS) bin_count_kernel(BinArgs a) {
    for_each_pair(a, [&](bool ok, uint32_t, uint32_t tile) {
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? tile : 0xffffffffu);
        if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&a.tile_count[tile], (uint32_t)__popc(peers));
    });
}

__global__ void __launch_bounds__(BIN_THREADS) bin_scatter_kernel(BinArgs a) {
    const unsigned lt = lanemask_lt();
    for_each_pair(a, [&](bool ok, uint32_t item, uint32_t tile) {
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? tile : 0xffffffffu);
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (ok && (int)(threadIdx.x & 31) == leader) slot = atomicAdd(&a.tile_cursor[tile], (uint32_t)__popc(peers));
        slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(peers & lt);
        if (ok && slot < a.cap) a.kv[slot] = ((unsigned long long)a.dkeys[item] << 32) | item;
    });
}

// One CTA: exclusive scan of the per-tile counts into ranges (clamped to the pair
// capacity) and write cursors; totals into the control block.
__global__ void __launch_bounds__(SCAN_THREADS) bin_scan_kernel(BinArgs a) {
    __shared__ unsigned long long s_w[SCAN_THREADS / 32 + 1];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int T = a.total_tiles;
    const int per = (T + SCAN_THREADS - 1) / SCAN_THREADS;
    const int b = min(T, tid * per), e = min(T, b + per);
    unsigned long long s = 0;
#pragma unroll 8
    for (int i = b; i < e; ++i) s += a.tile_count[i];
    // block exclusive scan of s
    unsigned long long x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = s_w[lane];
        unsigned long long t = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_w[lane] = t - v;
        if (lane == 31) s_w[32] = t;
    }
    __syncthreads();
    unsigned long long off = s_w[w] + x - s;
    const unsigned long long cap = a.cap;
    for (int i = b; i < e; ++i) {
        const uint32_t c = a.tile_count[i];
        const uint32_t lo = (uint32_t)(off < cap ? off : cap);
        const uint32_t hi = (uint32_t)(off + c < cap ? off + c : cap);
        a.ranges[i] = make_uint2(lo, hi);
        a.tile_cursor[i] = lo;
        off += c;
    }
    if (tid == 0) {
        const unsigned long long tot = s_w[32];
        a.ctl->n_pairs = (uint32_t)(tot < 0xffffffffull ? tot : 0xffffffffull);
        a.ctl->n_pairs_used = (uint32_t)(tot < cap ? tot : cap);
        a.ctl->overflow = tot > cap ? 1u : 0u;
    }
}

// Bitonic sort of s[0, P) ascending, P a power of two <= TSORT_CAP; all threads of the
// block call it.
__device__ __forceinline__ void bitonic_smem(unsigned long long *s, uint32_t P) {
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P / 2; i += TSORT_THREADS) {
                const uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const uint32_t hi = lo + j;
                const unsigned long long x = s[lo], y = s[hi];
                const bool up = (lo & k) == 0;
                if ((x > y) == up) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint32_t pow2_ceil(uint32_t n) {
    return n <= 2 ? 2u : 1u << (32 - __clz(n - 1));
}

// Sort kv[0, n) (n <= TSORT_CAP) into s, padding with the largest key.
__device__ __forceinline__ void sort_chunk(const unsigned long long *kv, uint32_t n, unsigned long long *s) {
    const uint32_t P = pow2_ceil(n);
    for (uint32_t i = threadIdx.x; i < P; i += TSORT_THREADS) s[i] = i < n ? kv[i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, P);
}

__global__ void __launch_bounds__(TSORT_THREADS) tile_sort_kernel(BinArgs a) {
    __shared__ unsigned long long s_kv[TSORT_CAP];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&a.ctl->work_counter[2], 1u);
        __syncthreads();
        const int t = (int)s_tile;
        if (t >= a.total_tiles) break;
        const uint2 r = a.ranges[t];
        const uint32_t n = r.y - r.x;
        if (n == 1) {
            if (tid == 0) a.items[r.x] = (uint32_t)a.kv[r.x];
        } else if (n > 1 && n <= (uint32_t)TSORT_CAP) {
            sort_chunk(a.kv + r.x, n, s_kv);
            for (uint32_t i = tid; i < n; i += TSORT_THREADS) a.items[r.x + i] = (uint32_t)s_kv[i];
        } else if (n > (uint32_t)TSORT_CAP) {
            // chunks of TSORT_CAP sorted in place, then pairwise merges (merge path)
            // between kv and kv_tmp; the last merge writes the item ids
            unsigned long long *src = a.kv + r.x, *dst = a.kv_tmp + r.x;
            for (uint32_t c0 = 0; c0 < n; c0 += TSORT_CAP) {
                const uint32_t m = min((uint32_t)TSORT_CAP, n - c0);
                sort_chunk(src + c0, m, s_kv);
                for (uint32_t i = tid; i < m; i += TSORT_THREADS) src[c0 + i] = s_kv[i];
                __syncthreads();
            }
            for (uint32_t wdt = TSORT_CAP; wdt < n; wdt <<= 1) {
                const bool last = (uint64_t)wdt * 2 >= n;
                for (uint32_t p0 = 0; p0 < n; p0 += 2 * wdt) {
                    const uint32_t la = min(wdt, n - p0), lb = min(wdt, n - p0 - la);
                    const unsigned long long *A = src + p0, *B = src + p0 + la;
                    const uint32_t tot = la + lb;
                    for (uint32_t d0 = 0; d0 < tot; d0 += TSORT_THREADS * MERGE_PER_THREAD) {
                        const uint32_t diag = min(tot, d0 + tid * MERGE_PER_THREAD);
                        uint32_t lo = diag > lb ? diag - lb : 0u, hi = min(diag, la);
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (A[mid] < B[diag - 1 - mid]) lo = mid + 1;
                            else hi = mid;
                        }
                        uint32_t i = lo, j = diag - lo;
                        for (int q = 0; q < MERGE_PER_THREAD && diag + q < tot; ++q) {
                            unsigned long long v;
                            if (j >= lb || (i < la && A[i] < B[j])) v = A[i++];
                            else v = B[j++];
                            if (last) a.items[r.x + p0 + diag + q] = (uint32_t)v;
                            else dst[p0 + diag + q] = v;
                        }
                    }
                }
                __syncthreads();
                unsigned long long *tmp = src;
                src = dst;
                dst = tmp;
            }
        }
        __syncthreads();
    }
}

void launch_bin_count(const BinArgs &a, int sms, cudaStream_t st) {
    int64_t g = (a.n_items + BIN_THREADS - 1) / BIN_THREADS;
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    if (g > 0) bin_count_kernel<<<(unsigned)g, BIN_THREADS, 0, st>>>(a);
}

void launch_bin_scan(const BinArgs &a, cudaStream_t st) {
    if (a.total_tiles > 0) bin_scan_kernel<<<1, SCAN_THREADS, 0, st>>>(a);
}

void launch_bin_scatter(const BinArgs &a, int sms, cudaStream_t st) {
    int64_t g = (a.n_items + BIN_THREADS - 1) / BIN_THREADS;
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    if (g > 0) bin_scatter_kernel<<<(unsigned)g, BIN_THREADS, 0, st>>>(a);
}

void launch_tile_sort(const BinArgs &a, int sms, cudaStream_t st) {
    static int occ = -1;
    if (occ < 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tile_sort_kernel, TSORT_THREADS, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
    }
    int64_t g = (int64_t)sms * occ;
    if (g > a.total_tiles) g = a.total_tiles;
    if (g > 0) tile_sort_kernel<<<(unsigned)g, TSORT_THREADS, 0, st>>>(a);
}

}  // namespace ts
