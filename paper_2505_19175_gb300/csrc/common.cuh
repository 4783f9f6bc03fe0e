// Internal device definitions of the triangle-splat renderer (sm_103a).
//
// Constants are this library's readings of values the paper leaves to prior
// splatting work (Sec. 3.1: "the rendering equation is the same as ...") or leaves
// unset (Supp. "Tile assignment": tau_cutoff).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ts {

constexpr int TILE = 16;                 // 16 x 16 pixel tiles
constexpr int TILE_PIX = TILE * TILE;    // one CTA of 256 threads per tile
constexpr float ALPHA_MAX = 0.99f;       // alpha clamp
constexpr float ALPHA_MIN = 1.0f / 255.0f;  // skip threshold; also tau_cutoff of the rectangle
constexpr float T_EPS = 1e-4f;           // stop before transmittance drops below this
constexpr float Z_NEAR = 0.2f;           // cull a triangle with a vertex nearer than this
constexpr float R_MIN = 1e-4f;           // cull a triangle whose inradius (px) is below this
constexpr float RECT_PAD = 1.0f / 512.0f;  // px added around the tight rectangle (FP32 slack)
constexpr float FRUSTUM_PAD = 2.0f;        // px beyond the image edges of the preprocess's view test
constexpr int MAX_VIEWS = 64;            // views per preprocess call

// Status words of the decoupled look-back scans: 2 flag bits over a 30-bit count.
constexpr uint32_t LB_AGG = 1u << 30;
constexpr uint32_t LB_PREFIX = 2u << 30;
constexpr uint32_t LB_MASK = (1u << 30) - 1;

// bits of Ctl::error
constexpr uint32_t ERR_SPIN = 1u;        // a bounded look-back wait gave up
constexpr uint32_t ERR_INDEX = 2u;       // an index check failed

// One view as the kernels see it.
struct ViewDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float bg[3];
    float campos[3];       // camera centre -R^T t in world space
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;         // first global tile id of this view
    int pix_base;          // first pixel of this view in the per-pixel buffers
};

// Per-view output pointers of one render call.
struct ViewOut {
    float *image;          // [3][H][W]
    const float *dL;       // [3][H][W] (backward)
    const float *target = nullptr;   // [3][H][W] forward with the L1 loss: target image
    float *grad = nullptr;           // [3][H][W] and its dL/dimage output
};

// Device control block: counters, histograms and work queues of one pipeline run.
// Tiles are rendered in descending order of their pair count (longest first, so that
// no long tile starts last and leaves the machine idle at the end): counts fall into
// half-octave buckets, key 0 for an empty tile and 1 + 2 floor(log2 n) + (the bit
// below the leading one) otherwise, 1..64.
constexpr int ORD_BUCKETS = 65;
__host__ __device__ __forceinline__ int tile_order_key(uint32_t n) {
    if (n == 0) return 0;
#ifdef __CUDA_ARCH__
    const int lg = 31 - __clz(n);
#else
    int lg = 0;
    while ((n >> lg) > 1u) ++lg;
#endif
    return 1 + 2 * lg + (lg > 0 ? (int)((n >> (lg - 1)) & 1u) : 0);
}

struct Ctl {
    uint32_t n_visible;        // visible items after preprocess
    uint32_t n_pairs;          // pairs emitted (may exceed capacity)
    uint32_t n_pairs_used;     // min(n_pairs, capacity)
    uint32_t overflow;
    uint32_t error;
    uint32_t cta_counter[8];   // dynamic CTA ids of the single-pass scans
    uint32_t pass_counter[8];  // dynamic tile ids of the radix passes
    uint32_t work_counter[4];  // render work queues
    uint32_t big_count;        // tiles queued for the CTA-wide sort
    uint32_t big_next;         // next queued tile to sort
    uint32_t done[8];          // CTAs finished, per self-cleaning kernel (see last_cta_done)
    uint32_t vis_count;        // entries appended to the visible-item list (may exceed its capacity)
    unsigned long long frag_eval;   // forward: (pixel, entry) evaluations
    unsigned long long frag_kept;   // forward: composited fragments
    unsigned long long pps_total;   // per-pixel sort: candidates of all pixels
    uint32_t ord_hist[ORD_BUCKETS];  // tiles per order key (bin_scan)
    uint32_t ord_next[ORD_BUCKETS];  // tiles placed per order key (tile_sort)
    uint32_t depth_hist[4][256];
    uint32_t tile_hist[4][256];
};

// Render record of one item: 16 floats = 4 x float4 (64 B).
//   a = (s_hi.x, s_hi.y, A0, B0)   b = (s_lo.x, A1, B1, s_lo.y)
//   c = (A2, B2, 0, o)              d = (sigma, r, g, b)
// The incenter is s = s_hi + s_lo (double-float); edge line i is
// m_i(p) = 1 + A_i (p.x - s.x) + B_i (p.y - s.y), evaluated with p - s =
// ((p - s_hi) - s_lo), the first difference exact; m_i = 1 at the incenter, 0 on edge
// i, and the window ratio phi(p)/phi(s) = min_i m_i(p). The line's offset about s_hi,
// C_i = 1 - A_i s_lo.x - B_i s_lo.y, serves the block tests.
struct __align__(16) Rec {
    float4 a, b, c, d;
};

// Per-item gradient record, same 16-float footprint:
//   (g_sx, g_sy, gA0, gB0, gA1, gB1, gA2, gB2, g_o, g_sigma, g_r, g_g, g_b, 0, 0, 0)
// with the slopes' gradients taken about the exact incenter, gA_i = sum dL/dm_i (p.x - s.x).
constexpr int GRAD_FIELDS = 16;

// ---------------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void red_add_v2(float *p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Longest wait of a look-back on its predecessor's status word (device time), and a
// cap on the polls of one wait in case the timer stalls.
constexpr uint64_t WAIT_NS = 1000000000ull;
constexpr uint32_t WAIT_POLLS_MAX = 1u << 24;

// Wait for a look-back predecessor's status word to leave 0, for at most `limit_ns` of
// device time (and WAIT_POLLS_MAX polls); on timeout set ERR_SPIN and return 0 (the
// result is then invalid but the kernel finishes). Waiting stops at once when an error
// is already set.
__device__ __forceinline__ uint32_t wait_status(const uint32_t *p, uint32_t *err, uint64_t limit_ns = WAIT_NS) {
    uint32_t s = ld_relaxed(p);
    if (s != 0) return s;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        s = ld_relaxed(p);
        if (s != 0) return s;
        if ((it & 63) == 63) {
            if (ld_relaxed(err) != 0 || global_ns() - t0 > limit_ns || it >= WAIT_POLLS_MAX) {
                atomicOr(err, ERR_SPIN);
                return LB_PREFIX;  // pretend a zero prefix so the chain ends
            }
            __nanosleep(100);
        }
    }
}

// Fragment evaluation shared by the forward and backward kernels, so that both take
// bitwise identical decisions: edge values, window ratio and unclamped alpha.
// dx, dy = p - s about the exact incenter.
struct Frag {
    float dx, dy, m0, m1, m2, ratio;
};

__device__ __forceinline__ Frag eval_lines(const float4 a, const float4 b, const float4 c, float px,
                                           float py) {
    Frag f;
    f.dx = __fsub_rn(__fsub_rn(px, a.x), b.x);
    f.dy = __fsub_rn(__fsub_rn(py, a.y), b.w);
    f.m0 = fmaf(a.z, f.dx, fmaf(a.w, f.dy, 1.0f));
    f.m1 = fmaf(b.y, f.dx, fmaf(b.z, f.dy, 1.0f));
    f.m2 = fmaf(c.x, f.dx, fmaf(c.y, f.dy, 1.0f));
    f.ratio = fminf(f.m0, fminf(f.m1, f.m2));
    return f;
}

// Offset of a record's edge line about s_hi: m_i(p) = C_i + A_i (p.x - s_hi.x) + B_i (p.y - s_hi.y).
__device__ __forceinline__ float line_offset(float A, float B, float4 b) {
    return fmaf(-A, b.x, fmaf(-B, b.w, 1.0f));
}

// I = ratio^sigma for ratio > 0
__device__ __forceinline__ float window_pow(float ratio, float sigma) {
    return ex2_approx(__fmul_rn(sigma, lg2_approx(ratio)));
}

// Window kinds: WIN_POWER is the paper's Eq. indicator1, I = ratio^sigma (ratio > 0);
// WIN_SIGMOID is Eq. indicator2, I = sigmoid(-phi / sigma) = sigmoid(kappa ratio) with
// kappa = r / sigma (phi = -r ratio, r the inradius in pixels); the record stores
// sigma or kappa in the same slot.
enum { WIN_POWER = 0, WIN_SIGMOID = 1 };

__device__ __forceinline__ float window_sigmoid(float ratio, float kappa) {
    return rcp_approx(1.0f + ex2_approx(-1.4426950408889634f * __fmul_rn(kappa, ratio)));
}

// Exclusive scan across the CTA of one value per thread (blockDim.x <= 1024).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
        uint32_t t = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_sums[lane] = t - s;
        if (lane == nw - 1) warp_sums[32] = t;
    }
    __syncthreads();
    total = warp_sums[32];
    uint32_t r = warp_sums[w] + x - v;
    __syncthreads();
    return r;
}

// Decoupled look-back over one status word per CTA, run by all 32 lanes of one warp:
// each round fetches the 32 nearest predecessors at once and stops at the nearest one
// that already holds an inclusive prefix. Returns the exclusive prefix of `agg` over
// CTAs 0..idx-1 in every lane.
__device__ __forceinline__ uint32_t warp_lookback_excl(uint32_t *status, uint32_t idx, uint32_t agg, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    if (idx == 0) {
        if (lane == 0) st_relaxed(&status[0], LB_PREFIX | agg);
        return 0;
    }
    if (lane == 0) st_relaxed(&status[idx], LB_AGG | agg);
    uint32_t excl = 0;
    int base = (int)idx - 1;
    while (true) {
        const int k = base - lane;  // lane 0 holds the nearest predecessor
        const uint32_t s = k >= 0 ? wait_status(&status[k], err) : LB_PREFIX;
        const unsigned pre = __ballot_sync(0xffffffffu, (s >> 30) == 2u);
        const int stop = pre ? __ffs(pre) - 1 : 31;
        uint32_t v = lane <= stop ? (s & LB_MASK) : 0u;
        v = __reduce_add_sync(0xffffffffu, v);
        excl += v;
        if (pre) break;
        base -= 32;
    }
    if (lane == 0) st_relaxed(&status[idx], LB_PREFIX | ((excl + agg) & LB_MASK));
    return excl;
}

// 64-bit look-back words: flag (LB64_AGG / LB64_PREFIX) in the top two bits, a 62-bit
// count below; 0 = not yet published.
constexpr uint64_t LB64_AGG = 1ull << 62;
constexpr uint64_t LB64_PREFIX = 2ull << 62;
constexpr uint64_t LB64_MASK = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// As wait_status, for 64-bit words (bounded: limit_ns, then ERR_SPIN and a zero prefix).
__device__ __forceinline__ uint64_t wait_status64(const uint64_t *p, uint32_t *err, uint64_t limit_ns = WAIT_NS) {
    uint64_t s = ld_relaxed64(p);
    if (s != 0) return s;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        s = ld_relaxed64(p);
        if (s != 0) return s;
        if ((it & 63) == 63) {
            if (ld_relaxed(err) != 0 || global_ns() - t0 > limit_ns || it >= WAIT_POLLS_MAX) {
                atomicOr(err, ERR_SPIN);
                return LB64_PREFIX;
            }
            __nanosleep(100);
        }
    }
}

// Warp-parallel decoupled look-back over 64-bit words (called by one full warp):
// publishes `agg` for tile `idx` and returns the exclusive prefix. `publish` = false
// leaves this tile's word unset (a failure-detection test: the successors' bounded
// waits then give up after limit_ns).
__device__ __forceinline__ uint64_t warp_lookback_excl64(uint64_t *status, uint32_t idx, uint64_t agg,
                                                         uint32_t *err, uint64_t limit_ns = WAIT_NS,
                                                         bool publish = true) {
    const int lane = threadIdx.x & 31;
    if (idx == 0) {
        if (lane == 0 && publish) st_relaxed64(&status[0], LB64_PREFIX | agg);
        return 0;
    }
    if (lane == 0 && publish) st_relaxed64(&status[idx], LB64_AGG | agg);
    uint64_t excl = 0;
    int base = (int)idx - 1;
    while (true) {
        const int k = base - lane;
        const uint64_t s = k >= 0 ? wait_status64(&status[k], err, limit_ns) : LB64_PREFIX;
        const unsigned pre = __ballot_sync(0xffffffffu, (s >> 62) == 2u);
        const int stop = pre ? __ffs(pre) - 1 : 31;
        uint64_t v = lane <= stop ? (s & LB64_MASK) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pre) break;
        base -= 32;
    }
    if (lane == 0 && publish) st_relaxed64(&status[idx], LB64_PREFIX | ((excl + agg) & LB64_MASK));
    return excl;
}

// Called by every thread of every CTA as a kernel's last step: true in the CTA that
// finishes last (every other CTA has passed this point), which then resets the
// kernel's queue counters for the next launch; the done counter resets itself. The
// kernels that use it leave their counters at zero, so no memset precedes them.
__device__ __forceinline__ bool last_cta_done(uint32_t *done) {
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(done, 1u);
        s_last = d == gridDim.x - 1;
        if (s_last) *done = 0u;
    }
    __syncthreads();
    return s_last;
}

}  // namespace ts
