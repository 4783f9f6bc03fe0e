// Tile binning of (tile, item) pairs and per-tile depth order (Supp. "Tile assignment"
// and "Depth sorting": every triangle is listed in each tile its tight rectangle
// touches, and each tile's list is ordered by the triangles' centre depth).
//
// The result equals a stable sort of the pairs by the 64-bit key (tile << 32 | depth
// bits) when the pairs are emitted in item order: within a tile, entries are ordered
// by (depth key, item id). It is reached without a global sort:
//   1. per-tile pair counts, accumulated by the preprocess kernel;
//   2. bin_scan:    exclusive scan of the counts -> tile ranges and write cursors
//                   (single pass, decoupled look-back);
//   3. bin_scatter: each pair takes a slot in its tile's range (order within the
//                   range is arbitrary at this point);
//   4. tile_sort:   each tile's range is sorted by (depth key, item id) in shared
//                   memory (radix sort by one warp or, for long ranges, one CTA;
//                   ranges longer than one CTA's shared memory are sorted in chunks and
//                   merged in global memory).
// Keys are unique (item ids are), so the order is deterministic although the scatter
// is not.
#include "kernels.h"

namespace ts {

constexpr int BIN_THREADS = 256;
constexpr int TSORT_THREADS = 256;
constexpr int WS_MAX = 512;               // words one warp sorts; longer ranges take a CTA
constexpr int MERGE_PER_THREAD = 8;

// Expansion of the visible items into (item, tile) pairs. A CTA takes chunks of 256
// entries of the visible-item list (coalesced 16-byte loads: item, depth key, pixel
// rectangle; holes skipped) and expands them in rounds of 2 x BIN_THREADS pairs in which all threads
// of the block take part (so that f may use warp collectives): each thread decodes two
// pairs, o and o + BIN_THREADS, and f(ok, item, tile, depth key) is called with both
// (so that their memory operations overlap).
template <class F>
__device__ __forceinline__ void for_each_pair(const BinArgs &a, F &&f) {
    __shared__ uint32_t s_off[BIN_THREADS];
    __shared__ uint32_t s_item[BIN_THREADS];
    __shared__ uint32_t s_base_tile[BIN_THREADS];   // global id of the rectangle's first tile
    __shared__ uint32_t s_wx[BIN_THREADS];          // (rect width in tiles << 16) | view tiles_x
    __shared__ float s_iw[BIN_THREADS];             // 1 / rect width
    __shared__ uint32_t s_key[BIN_THREADS];         // depth key
    __shared__ uint32_t s_tmp[33];
    __shared__ int2 s_vt[MAX_VIEWS];                // (tiles_x, tile_base)
    const int tid = threadIdx.x;
    for (int k = tid; k < a.nviews; k += BIN_THREADS) s_vt[k] = make_int2(a.views[k].tiles_x, a.views[k].tile_base);
    __syncthreads();
    const uint32_t K = min(a.ctl->vis_count, a.vis_cap);
    const uint32_t nchunk = (K + BIN_THREADS - 1) / BIN_THREADS;
    // chunks in a strided order (a stride near 0.618 of the chunk count, coprime with
    // it): neighbouring entries (often neighbours on screen) go to CTAs far apart in
    // time, which spreads the atomics over many tiles
    uint32_t stride = nchunk > 2 ? ((uint32_t)((float)nchunk * 0.618034f) | 1u) : 1u;
    auto gcd = [](uint32_t x, uint32_t y) {
        while (y) {
            const uint32_t t = x % y;
            x = y;
            y = t;
        }
        return x;
    };
    while (nchunk > 1 && gcd(stride, nchunk) != 1u) stride += 2u;
    // pair o of the current chunk: (item, tile, key), tile 0xffffffff when invalid
    auto decode = [&](uint32_t o, uint32_t total, uint32_t &item, uint32_t &tile, uint32_t &key) {
        item = 0u;
        tile = 0xffffffffu;
        key = 0u;
        if (o >= total) return;
        // owner: the last thread whose offset is <= o (threads with no tile share their
        // successor's offset and lose the search)
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
        key = s_key[lo];
        tile = s_base_tile[lo] + row * tiles_x + col;
        if (tile >= (uint32_t)a.total_tiles) {
            atomicOr(&a.ctl->error, ERR_INDEX);
            tile = 0xffffffffu;
        }
    };
    for (uint32_t ci = blockIdx.x; ci < nchunk; ci += gridDim.x) {
        const uint32_t j = (uint32_t)(((uint64_t)ci * stride) % nchunk) * BIN_THREADS + tid;
        uint4 e = make_uint4(0u, 0u, 0u, 0u);
        bool valid = j < K;
        if (valid) {
            e = a.vislist[j];
            if (e.x == VIS_HOLE) {
                valid = false;
            } else if ((int64_t)e.x >= a.n_items) {
                atomicOr(&a.ctl->error, ERR_INDEX);
                valid = false;
            }
        }
        const uint32_t tx0 = (e.z & 0xffffu) / TILE, ty0 = (e.z >> 16) / TILE;
        const uint32_t wdt = (e.w & 0xffffu) / TILE - tx0 + 1, hgt = (e.w >> 16) / TILE - ty0 + 1;
        const uint32_t nt = valid ? wdt * hgt : 0u;
        uint32_t total;
        const uint32_t local = block_excl_scan(nt, s_tmp, total);
        s_off[tid] = local;
        s_item[tid] = e.x;
        if (nt) {
            const int2 vt = s_vt[a.nviews > 1 ? (int)((int64_t)e.x / a.n) : 0];
            s_base_tile[tid] = (uint32_t)vt.y + ty0 * (uint32_t)vt.x + tx0;
            s_wx[tid] = (wdt << 16) | (uint32_t)vt.x;
            s_iw[tid] = 1.0f / (float)wdt;
            s_key[tid] = e.y;
        }
        __syncthreads();
        for (uint32_t r0 = 0; r0 < total; r0 += 2 * BIN_THREADS) {
            uint32_t i0, t0, k0, i1, t1, k1;
            decode(r0 + tid, total, i0, t0, k0);
            decode(r0 + BIN_THREADS + tid, total, i1, t1, k1);
            f(t0 != 0xffffffffu, i0, t0, k0, t1 != 0xffffffffu, i1, t1, k1);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BIN_THREADS) bin_scatter_kernel(BinArgs a) {
    const unsigned lt = lanemask_lt();
    const int lane = (int)(threadIdx.x & 31);
    for_each_pair(a, [&](bool ok0, uint32_t item0, uint32_t tile0, uint32_t key0, bool ok1, uint32_t item1,
                         uint32_t tile1, uint32_t key1) {
        // one slot reservation per tile among the warp's pairs (both atomics in flight)
        const unsigned p0 = __match_any_sync(0xffffffffu, ok0 ? tile0 : 0xffffffffu);
        const unsigned p1 = __match_any_sync(0xffffffffu, ok1 ? tile1 : 0xffffffffu);
        const int l0 = __ffs(p0) - 1, l1 = __ffs(p1) - 1;
        uint32_t s0 = 0, s1 = 0;
        if (ok0 && lane == l0) s0 = atomicAdd(&a.tile_cursor[tile0], (uint32_t)__popc(p0));
        if (ok1 && lane == l1) s1 = atomicAdd(&a.tile_cursor[tile1], (uint32_t)__popc(p1));
        s0 = __shfl_sync(0xffffffffu, s0, l0) + __popc(p0 & lt);
        s1 = __shfl_sync(0xffffffffu, s1, l1) + __popc(p1 & lt);
        if (ok0 && s0 < a.cap) a.kv[s0] = ((unsigned long long)key0 << 32) | item0;
        if (ok1 && s1 < a.cap) a.kv[s1] = ((unsigned long long)key1 << 32) | item1;
    });
}

// Exclusive scan of the per-tile counts into ranges (clamped to the pair capacity) and
// write cursors; totals into the control block. CTA b (ticket order) scans tiles
// [1024 b, 1024 b + 1024) and takes its offset from a single-pass decoupled look-back
// over 64-bit words.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

__global__ void __launch_bounds__(SCAN_THREADS) bin_scan_kernel(BinArgs a) {
    __shared__ unsigned long long s_w[SCAN_THREADS / 32 + 1];
    __shared__ uint32_t s_cta;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_oh[ORD_BUCKETS];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid < ORD_BUCKETS) s_oh[tid] = 0u;
    if (tid == 0) s_cta = atomicAdd(a.scan_ticket, 1u);
    __syncthreads();
    const uint32_t cta = s_cta;
    const int T = a.total_tiles;
    const int64_t t0 = (int64_t)cta * SCAN_TILE + tid * SCAN_PER;
    uint32_t c[SCAN_PER];
#pragma unroll
    for (int q = 0; q < SCAN_PER; ++q) c[q] = t0 + q < T ? a.tile_count[t0 + q] : 0u;
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < SCAN_PER; ++q) sum += c[q];
    // block exclusive scan of the per-thread sums
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = lane < SCAN_THREADS / 32 ? s_w[lane] : 0ull;
        unsigned long long t = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, t, SCAN_THREADS / 32 - 1);
        if (lane < SCAN_THREADS / 32) s_w[lane] = t - v;
        const unsigned long long b =
            warp_lookback_excl64(a.scan_status, cta, total, &a.ctl->error, a.wait_ns, a.withhold != cta + 1);
        if (lane == 0) {
            s_base = b;
            if ((int64_t)(cta + 1) * SCAN_TILE >= T) {
                const unsigned long long tot = b + total, cap = a.cap;
                a.ctl->n_pairs = (uint32_t)(tot < 0xffffffffull ? tot : 0xffffffffull);
                a.ctl->n_pairs_used = (uint32_t)(tot < cap ? tot : cap);
                a.ctl->overflow = tot > cap ? 1u : 0u;
            }
        }
    }
    __syncthreads();
    unsigned long long off = s_base + s_w[w] + x - sum;
    const unsigned long long cap = a.cap;
#pragma unroll
    for (int q = 0; q < SCAN_PER; ++q) {
        if (t0 + q < T) {
            const uint32_t lo = (uint32_t)(off < cap ? off : cap);
            const uint32_t hi = (uint32_t)(off + c[q] < cap ? off + c[q] : cap);
            a.ranges[t0 + q] = make_uint2(lo, hi);
            a.tile_cursor[t0 + q] = lo;
            if (hi - lo > (uint32_t)WS_MAX) {
                // queued for a CTA-wide sort
                const uint32_t k = atomicAdd(&a.ctl->big_count, 1u);
                if (k < (uint32_t)T) a.big_tiles[k] = (uint32_t)(t0 + q);
                else atomicOr(&a.ctl->error, ERR_INDEX);
            }
            if (a.tile_order) atomicAdd(&s_oh[tile_order_key(hi - lo)], 1u);
        }
        off += c[q];
    }
    if (a.tile_order) {
        // tiles per order key, for tile_sort's placement
        __syncthreads();
        if (tid < ORD_BUCKETS && s_oh[tid]) atomicAdd(&a.ctl->ord_hist[tid], s_oh[tid]);
    }
    if (last_cta_done(&a.ctl->done[3])) {
        // every CTA's look-back is over: clear the status words and the ticket
        const int words = (T + SCAN_TILE - 1) / SCAN_TILE + 1;
        for (int k = tid; k < words; k += SCAN_THREADS) a.scan_status[k] = 0ull;
        if (tid == 0) *a.scan_ticket = 0u;
    }
}

// ---- per-tile order ----
// Each tile's range of (depth key << 32 | item) words is sorted ascending, which is
// the (depth key, item id) order, by one kernel (tile_sort_kernel). Ranges of at most
// WS_MAX words are sorted by one warp in registers (bitonic network: lane l holds
// words [l E, l E + E), strides below E are exchanges between registers and larger
// ones warp shuffles); longer ranges, queued by the scan, take a whole CTA, whose warps
// sort 256-word chunks the same way and merge them in shared memory (merge path).
// Ranges beyond BS_MAX words are sorted in BS_MAX chunks that are then merged pairwise
// in global memory.
constexpr int BS_MAX = 2048;              // words one CTA sorts in shared memory

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

// Register stages J, J/2, ..., 1 (those below the block size k) of a bitonic merge.
template <int E, int J>
__device__ __forceinline__ void reg_stages(unsigned long long (&x)[E], uint32_t base, uint32_t k) {
    if constexpr (J >= 1) {
        if ((uint32_t)J <= (k >> 1)) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if ((e & J) == 0) {
                    const bool asc = ((base + e) & k) == 0;
                    const unsigned long long p = x[e], q = x[e | J];
                    const bool sw = (p > q) == asc;
                    x[e] = sw ? q : p;
                    x[e | J] = sw ? p : q;
                }
            }
        }
        reg_stages<E, J / 2>(x, base, k);
    }
}

// Ascending bitonic sort of the 32 E words a warp holds, E per lane (blocked: lane l
// holds indices [l E, l E + E)). Strides of E and more are warp shuffles with lane
// ^ (j / E); smaller strides are exchanges between a lane's registers. Loops over the
// block sizes k keep the code small.
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[E]) {
    const uint32_t base = (uint32_t)(threadIdx.x & 31) * E;   // index of x[0]
    for (uint32_t k = 2; k <= 32u * E; k <<= 1) {
        for (uint32_t j = k >> 1; j >= (uint32_t)E; j >>= 1) {
            // the pair's lower index keeps the smaller word in an ascending block
            const bool keep_min = ((base & j) == 0) == ((base & k) == 0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const unsigned long long y = shfl_xor_u64(x[e], (int)(j / E));
                x[e] = keep_min ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
            }
        }
        reg_stages<E, E / 2>(x, base, k);
    }
}

// One warp sorts kv[start, start + n) (n <= 32 E, padded with the largest word) and
// writes the item ids.
template <int E>
__device__ __forceinline__ void warp_sort_range(const BinArgs &a, uint32_t start, int n) {
    const int base = (threadIdx.x & 31) * E;
    unsigned long long x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = base + e < n ? a.kv[start + base + e] : ~0ull;
    warp_bitonic<E>(x);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (base + e < n) a.items[start + base + e] = (uint32_t)x[e];
}

// The CTA sorts src[0, n) (1 <= n <= BS_MAX) into shared memory: warps sort 256-word
// chunks in registers, then merge levels 256 -> 512 -> ... between A and B. Returns
// the buffer with the result (padded with the largest word to a power of two).
__device__ unsigned long long *block_sort(const unsigned long long *src, int n, unsigned long long *A,
                                          unsigned long long *B) {
    const int tid = threadIdx.x, w = tid >> 5;
    int P = 256;
    while (P < n) P <<= 1;
    if (w < P / 256) {
        const int base = w * 256 + (tid & 31) * 8;
        unsigned long long x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = base + e < n ? src[base + e] : ~0ull;
        warp_bitonic<8>(x);
#pragma unroll
        for (int e = 0; e < 8; ++e) A[base + e] = x[e];
    }
    __syncthreads();
    const int per = P / TSORT_THREADS;   // outputs per thread, 1..8
    for (int wdt = 256; wdt < P; wdt <<= 1) {
        const int d0 = tid * per;
        const int p0 = d0 / (2 * wdt) * (2 * wdt);
        const int diag = d0 - p0;
        const unsigned long long *Ar = A + p0, *Br = A + p0 + wdt;
        int lo = diag > wdt ? diag - wdt : 0, hi = diag < wdt ? diag : wdt;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Ar[mid] < Br[diag - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = diag - lo;
        for (int q = 0; q < per; ++q) {
            unsigned long long v;
            if (j >= wdt || (i < wdt && Ar[i] < Br[j])) v = Ar[i++];
            else v = Br[j++];
            B[d0 + q] = v;
        }
        __syncthreads();
        unsigned long long *t = A;
        A = B;
        B = t;
    }
    return A;
}

// One launch sorts every range: each CTA first takes the ranges longer than WS_MAX that
// the scan queued (one CTA each), then its warps take the others from the tile queue
// (one warp each, ranges longer than WS_MAX skipped), so the long ranges overlap with
// the many short ones.
__global__ void __launch_bounds__(TSORT_THREADS, 3) tile_sort_kernel(BinArgs a) {
    __shared__ unsigned long long s_a[BS_MAX], s_b[BS_MAX];
    __shared__ uint32_t s_q;
    __shared__ uint32_t s_ob[ORD_BUCKETS];
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t nbig = min(a.ctl->big_count, (uint32_t)a.total_tiles);
    if (a.tile_order && (tid >> 5) == 1) {
        // first slot of each order key (the tiles of larger keys come first), by warp 1
        // while thread 0 takes the first queued tile: lane l holds keys 3l .. 3l + 2
        uint32_t h[3], tot = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = 3 * lane + j;
            h[j] = k < ORD_BUCKETS ? a.ctl->ord_hist[k] : 0u;
            tot += h[j];
        }
        uint32_t suf = tot;      // inclusive sum over lanes >= this one
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_down_sync(0xffffffffu, suf, o);
            if (lane + o < 32) suf += y;
        }
        uint32_t acc = suf - tot;
#pragma unroll
        for (int j = 2; j >= 0; --j) {
            const int k = 3 * lane + j;
            if (k < ORD_BUCKETS) s_ob[k] = acc;
            acc += h[j];
        }
    }
    // (s_ob is read after the barriers of the first loop)
    for (;;) {
        if (tid == 0) s_q = atomicAdd(&a.ctl->big_next, 1u);
        __syncthreads();
        const uint32_t q = s_q;
        __syncthreads();
        if (q >= nbig) break;
        const uint32_t t = a.big_tiles[q];
        if (t >= (uint32_t)a.total_tiles) {
            if (tid == 0) atomicOr(&a.ctl->error, ERR_INDEX);
            continue;
        }
        const uint2 r = a.ranges[t];
        const uint32_t n = r.y - r.x;
        if (n <= (uint32_t)BS_MAX) {
            const unsigned long long *res = block_sort(a.kv + r.x, (int)n, s_a, s_b);
            for (uint32_t i = tid; i < n; i += TSORT_THREADS) a.items[r.x + i] = (uint32_t)res[i];
        } else {
            // chunks of BS_MAX sorted in place, then pairwise merges (merge path)
            // between kv and kv_tmp; the last merge writes the item ids
            unsigned long long *src = a.kv + r.x, *dst = a.kv_tmp + r.x;
            for (uint32_t c0 = 0; c0 < n; c0 += BS_MAX) {
                const int m = (int)min((uint32_t)BS_MAX, n - c0);
                const unsigned long long *res = block_sort(src + c0, m, s_a, s_b);
                for (int i = tid; i < m; i += TSORT_THREADS) src[c0 + i] = res[i];
                __syncthreads();
            }
            for (uint32_t wdt = BS_MAX; wdt < n; wdt <<= 1) {
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
                        for (int q2 = 0; q2 < MERGE_PER_THREAD && diag + q2 < tot; ++q2) {
                            unsigned long long v;
                            if (j >= lb || (i < la && A[i] < B[j])) v = A[i++];
                            else v = B[j++];
                            if (last) a.items[r.x + p0 + diag + q2] = (uint32_t)v;
                            else dst[p0 + diag + q2] = v;
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
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&a.ctl->work_counter[2], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (uint32_t)a.total_tiles) break;
        const uint2 r = a.ranges[t];
        const int n = (int)(r.y - r.x);
        // this tile's place in the render order: the rank is taken now and stored after
        // the sort, which hides the atomic's round trip
        uint32_t obase = 0, orank = 0;
        if (a.tile_order && lane == 0) {
            const int key = tile_order_key((uint32_t)n);
            obase = s_ob[key];
            orank = atomicAdd(&a.ctl->ord_next[key], 1u);
        }
        if (n <= 1) {
            if (n == 1 && lane == 0) a.items[r.x] = (uint32_t)a.kv[r.x];
        } else if (n > WS_MAX) {
            // sorted above
        } else if (n <= 32) {
            warp_sort_range<1>(a, r.x, n);
        } else if (n <= 64) {
            warp_sort_range<2>(a, r.x, n);
        } else if (n <= 128) {
            warp_sort_range<4>(a, r.x, n);
        } else if (n <= 256) {
            warp_sort_range<8>(a, r.x, n);
        } else {
            warp_sort_range<16>(a, r.x, n);
        }
        if (a.tile_order && lane == 0) {
            const uint32_t slot = obase + orank;
            if (slot < (uint32_t)a.total_tiles) a.tile_order[slot] = t;
            else atomicOr(&a.ctl->error, ERR_INDEX);
        }
    }
    if (last_cta_done(&a.ctl->done[2]) && tid == 0) {
        a.ctl->work_counter[2] = 0u;
        a.ctl->big_count = 0u;
        a.ctl->big_next = 0u;
        for (int k = 0; k < ORD_BUCKETS; ++k) {
            a.ctl->ord_hist[k] = 0u;
            a.ctl->ord_next[k] = 0u;
        }
    }
}

void launch_bin_scan(const BinArgs &a, cudaStream_t st) {
    const int g = (a.total_tiles + SCAN_TILE - 1) / SCAN_TILE;
    if (g > 0) bin_scan_kernel<<<g, SCAN_THREADS, 0, st>>>(a);
}

size_t bin_scan_status_words(int total_tiles) { return (size_t)((total_tiles + SCAN_TILE - 1) / SCAN_TILE) + 1; }

void launch_bin_scatter(const BinArgs &a, int sms, cudaStream_t st) {
    // (the list's length is known on the device only: enough CTAs for every item, at most 16 per SM)
    int64_t g = (a.n_items + BIN_THREADS - 1) / BIN_THREADS;
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    if (g > 0) bin_scatter_kernel<<<(unsigned)g, BIN_THREADS, 0, st>>>(a);
}

static int occupancy_of(const void *fn, int threads) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) occ = 1;
    return occ;
}

void launch_tile_sort(const BinArgs &a, int sms, cudaStream_t st) {
    static const int occ = occupancy_of((const void *)tile_sort_kernel, TSORT_THREADS);
    if (a.total_tiles <= 0) return;
    // one warp per short range: enough CTAs for every tile's warp, at most a full machine
    int64_t g = ((int64_t)a.total_tiles + TSORT_THREADS / 32 - 1) / (TSORT_THREADS / 32);
    if (g > (int64_t)sms * occ) g = (int64_t)sms * occ;
    tile_sort_kernel<<<(unsigned)g, TSORT_THREADS, 0, st>>>(a);
}

}  // namespace ts
