// Tile rendering of the triangle-splat renderer, forward and backward.
//
// A tile is 16x16 pixels, cut into eight 8x4 blocks and each block into eight 2x2
// groups. Tiles are taken from device work queues by persistent grids, so a launch
// serves any mix of views and resolutions.
//
// Forward (Sec. 3.1, the rendering equation of prior splatting work): one warp per half
// tile (16x8 pixels) and one lane per 2x2 group of it, with no CTA-wide barrier. The warp
// takes the tile's depth-sorted pairs front to back in windows of 64: the lane of pair j
// gathers the pair's record (64 B) and tests it against the half tile's 32 groups, and a
// warp bit transpose gives each lane the list of the window's pairs that may reach its
// group. Per pixel, ratio = min_i m_i(p) (phi(p)/phi(s) of Eq. indicator1),
// I = ratio^sigma, alpha = o I, skip below 1/255, clamp at 0.99, stop before T drops
// below 1e-4, C += rgb alpha T. A warp leaves its half tile as soon as every pixel has
// stopped. It also records, per pair, which groups composited it (one bit per group,
// KM_WORDS 32-bit words per pair, word h for half tile h), and per group the largest
// composited index.
//
// Backward: one warp per half tile (16x8 pixels) and one lane per 2x2 group of it,
// with no CTA-wide barrier. The warp takes the tile's pairs back to front in windows
// of 128: the lane of pair j stages the pair's record in shared memory when any group
// of the half tile composited it, and the window's group masks are transposed across
// the warp so that each lane holds the bit list of the pairs its group composited.
// Each lane walks its list back to front and evaluates its four pixels in
// straight-line code: T_k = T_{k+1} / (1 - alpha_k),
// dL/dalpha_k = sum_c g_c (rgb_c T_k - B_c / (1 - alpha_k)) with B the colour behind
// fragment k plus T_final bg; the group's 13 record-field gradients go to the item's
// gradient record with the lane's own vector reductions.
#include "kernels.h"

namespace ts {

constexpr int REN_THREADS = TILE_PIX;
constexpr int GROUPS = GROUPS_PER_TILE;           // groups per tile

// View of a tile from the views' first tile ids, by one warp (all lanes get it): the
// last view whose first tile is <= tile.
__device__ __forceinline__ int find_view_warp(const ViewDev *vs, int nviews, int tile, int lane) {
    int v = 0;
    for (int base = 0; base < nviews; base += 32) {
        const int k = base + lane;
        const unsigned b = __ballot_sync(0xffffffffu, k < nviews && vs[k].tile_base <= tile);
        if (b) v = base + 31 - __clz((int)b);
    }
    return v;
}

__device__ __forceinline__ int find_view(const ViewDev *vs, int nviews, int tile) {
    int v = 0;
    for (int k = 1; k < nviews; ++k)
        if (vs[k].tile_base <= tile) v = k;
    return v;
}

// Pixel of lane `lane` of the warp that covers 8x4 block w of the tile: block w sits at
// ((w & 1) 8, (w >> 1) 4). A group of 8 lanes (g = lane / 8) covers the 2x4 column pair
// at x 2g, lane bit 0 as x and bits [2:1] as y; a group of 4 (g = lane / 4) the 2x2
// square at (2 (g & 3), 2 (g >> 2)), lane bit 0 as x and bit 1 as y.
__device__ __forceinline__ void block_pixel(int w, int lane, int &lx, int &ly) {
    if (GROUP == 8) {
        lx = ((w & 1) << 3) | ((lane >> 3) << 1) | (lane & 1);
        ly = ((w >> 1) << 2) | ((lane >> 1) & 3);
    } else if (GROUP == 2) {
        const int g = lane >> 1;
        lx = ((w & 1) << 3) | ((g & 3) << 1) | (lane & 1);
        ly = ((w >> 1) << 2) | (g >> 2);
    } else {
        const int g = lane >> 2;
        lx = ((w & 1) << 3) | ((g & 3) << 1) | (lane & 1);
        ly = ((w >> 1) << 2) | ((g >> 2) << 1) | ((lane >> 1) & 1);
    }
}
__device__ __forceinline__ void pixel_of(int tid, int &lx, int &ly) { block_pixel(tid >> 5, tid & 31, lx, ly); }

// Can edge line (A, B, C) be positive at some pixel centre of the block
// [x0, x1] x [y0, y1]? Its maximum over the block is at the corner its slope selects;
// the margin covers the FP32 rounding of the per-pixel evaluation at other pixels.
__device__ __forceinline__ bool line_reaches(float A, float B, float C, float sx, float sy, int x0, int x1, int y0,
                                             int y1, float thr) {
    const float dx = __fsub_rn((float)(A >= 0.f ? x1 : x0) + 0.5f, sx);
    const float dy = __fsub_rn((float)(B >= 0.f ? y1 : y0) + 0.5f, sy);
    const float t1 = A * dx, t2 = B * dy;
    const float m = C + t1 + t2;
    return m >= thr - (1e-3f + 4e-7f * (fabsf(t1) + fabsf(t2) + fabsf(C)));
}

// May the record composite at a pixel centre of [x0, x1] x [y0, y1]? Its pixel
// rectangle meets the block and every edge line can reach the cutoff ratio there (a
// separating-axis test of the block against the record's support).
__device__ __forceinline__ bool block_hit(const Rec &r, const ushort4 bx, int x0, int x1, int y0, int y1, float thr) {
    if ((int)bx.x > x1 || (int)bx.z < x0 || (int)bx.y > y1 || (int)bx.w < y0) return false;
    return line_reaches(r.a.z, r.a.w, line_offset(r.a.z, r.a.w, r.b), r.a.x, r.a.y, x0, x1, y0, y1, thr) &&
           line_reaches(r.b.y, r.b.z, line_offset(r.b.y, r.b.z, r.b), r.a.x, r.a.y, x0, x1, y0, y1, thr) &&
           line_reaches(r.c.x, r.c.y, line_offset(r.c.x, r.c.y, r.b), r.a.x, r.a.y, x0, x1, y0, y1, thr);
}

// The cutoff ratio below which alpha < 1/255:
// (1/255 / o)^(1/sigma) for the power window (taken 0.1 % low, far beyond the error of
// the approximate lg2 / ex2), ln(tau / (o - tau)) / kappa for the sigmoid window
// (negative when o > 2 tau), and 0 for solid records (the triangle itself).
template <int WIN>
__device__ __forceinline__ float cutoff_ratio(const Rec &r, bool solid) {
    if (solid) return 0.0f;
    if (WIN == WIN_SIGMOID)
        return 0.6931471805599453f * lg2_approx(ALPHA_MIN * rcp_approx(r.c.w - ALPHA_MIN)) * rcp_approx(r.d.x);
    return 0.999f * ex2_approx(lg2_approx(ALPHA_MIN / r.c.w) * rcp_approx(r.d.x));
}

// dL/dd of inv |d| (0 at d = 0): the L1 loss gradient of one value.
__device__ __forceinline__ float l1_sign(float d, float inv) { return d > 0.f ? inv : (d < 0.f ? -inv : 0.f); }

// Bit w set when the record (cutoff ratio thr) may composite at a pixel of warp w's
// 8x4 block of the tile with origin (ox, oy).
__device__ __forceinline__ uint32_t warp_mask(const Rec &r, const ushort4 bx, int ox, int oy, float thr) {
    uint32_t msk = 0;
#pragma unroll
    for (int wb = 0; wb < REN_THREADS / 32; ++wb) {
        const int x0 = ox + ((wb & 1) << 3), y0 = oy + ((wb >> 1) << 2);
        if (block_hit(r, bx, x0, x0 + 7, y0, y0 + 3, thr)) msk |= 1u << wb;
    }
    return msk;
}

// This warp's records of the staged batch, in batch order; returns the count.
__device__ __forceinline__ int warp_list(const uint16_t *s_mask, uint8_t *list, int w, int lane) {
    const unsigned lt = lanemask_lt();
    int cnt = 0;
#pragma unroll
    for (int c = 0; c < REN_THREADS / 32; ++c) {
        const int j = c * 32 + lane;
        const bool hit = (s_mask[j] >> w) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) list[cnt + __popc(bal & lt)] = (uint8_t)j;
        cnt += __popc(bal);
    }
    __syncwarp();
    return cnt;
}

// Backward, one lane per 2x2 group: a warp takes one half tile (16x8 pixels, the 32
// groups whose bits form word h of each pair's group mask, so lane l owns bit l), and
// each lane walks the pairs its group composited, back to front, evaluating its four
// pixels against one record and adding the group's gradient of that record with its
// own vector reductions (no cross-lane reduction). Lanes take their pairs from
// windows of BW_WIN * 32 pairs: the lane of pair j stages the pair's record in shared
// memory when any group composited it, and the window's mask words are transposed
// across the warp (word j -> lane l's bit j), so every lane holds its own bit list of
// the window.
static_assert(GROUP == 4 && KM_WORDS == 2, "the backward takes one 2x2 group per lane");
constexpr int BW_THREADS = 128;          // warps per CTA work independently
constexpr int BW_WARPS = BW_THREADS / 32;
constexpr int BW_WIN = 4;                // mask words per lane per window (128 pairs)
constexpr int BW_RSTRIDE = 5;            // float4 per staged record (4 used)
#ifndef BW_CTAS
#define BW_CTAS 5
#endif
#ifndef BW_DENSE
#define BW_DENSE 10              // groups per distinct record of a window from which adds are coalesced
#endif

// 32x32 bit transpose across the warp: lane j holds row word r_j; returns the word
// whose bit j is bit `lane` of r_j.
__device__ __forceinline__ uint32_t warp_transpose_bits(uint32_t x, int lane) {
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t m = sh == 16 ? 0x0000FFFFu : (sh == 8 ? 0x00FF00FFu : (sh == 4 ? 0x0F0F0F0Fu : (sh == 2 ? 0x33333333u : 0x55555555u)));
        const uint32_t p = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? (((p >> sh) & m) | (x & (m << sh))) : ((x & m) | ((p & m) << sh));
    }
    return x;
}

// Highest set bit of the 128-bit list (hi:lo), cleared; -1 when empty.
__device__ __forceinline__ int pop_last(unsigned long long &hi, unsigned long long &lo) {
    if (hi) {
        const int b = 63 - __clzll((long long)hi);
        hi &= ~(1ull << b);
        return 64 + b;
    }
    if (lo) {
        const int b = 63 - __clzll((long long)lo);
        lo &= ~(1ull << b);
        return b;
    }
    return -1;
}

// The group's gradient of one record (ca..cd) at tile-list position jt, over the
// lane's four pixels, in straight-line code (independent pixels, so their arithmetic
// interleaves): a pixel that does not composite the fragment (or all four, when `mine`
// is false) computes with safe inputs and adds zeros. Updates T and B back to front;
// returns whether any pixel composited. dL/dratio of each pixel goes to its active
// line i: W[i] sums it, and with the pixel offsets dx_p = dx_0 + (p & 1),
// dy_p = dy_0 + (p >> 1), dL/dA_i = dx_0 W[i] + (sum over odd p) and dL/dB_i likewise,
// dL/ds = -(sum_i W[i] (A_i, B_i)).
template <int WIN>
__device__ __forceinline__ bool group_grad(const float4 ca, const float4 cb, const float4 cc, const float4 cd,
                                           uint32_t jt, bool mine, int x0, int y0, const uint32_t (&last)[4],
                                           float (&T)[4], const float (&G0)[4], const float (&G1)[4],
                                           const float (&G2)[4], float (&B0)[4], float (&B1)[4], float (&B2)[4],
                                           float (&gv)[13]) {
    float W[3] = {0.f, 0.f, 0.f}, Wx[3] = {0.f, 0.f, 0.f}, Wy[3] = {0.f, 0.f, 0.f};
    float go = 0.f, gs = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f, dx0 = 0.f, dy0 = 0.f;
    bool any = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float px = (float)(x0 + (p & 1)) + 0.5f, py = (float)(y0 + (p >> 1)) + 0.5f;
        const Frag f = eval_lines(ca, cb, cc, px, py);
        if (p == 0) {
            dx0 = f.dx;
            dy0 = f.dy;
        }
        const bool pos = WIN == WIN_SIGMOID || f.ratio > 0.0f;
        const float rs = pos ? f.ratio : 1.0f;   // the power window's ratio, kept positive
        const float lg = WIN == WIN_SIGMOID ? 0.0f : lg2_approx(rs);
        const float I = WIN == WIN_SIGMOID ? window_sigmoid(f.ratio, cd.x) : ex2_approx(__fmul_rn(cd.x, lg));
        const float araw = __fmul_rn(cc.w, I);
        const bool kept = mine && jt < last[p] && pos && araw >= ALPHA_MIN;
        any = any || kept;
        const float al = fminf(araw, ALPHA_MAX);
        const float om = __fsub_rn(1.0f, al);
        const float iom = rcp_approx(om);
        const float Tn = T[p] * iom;
        T[p] = kept ? Tn : T[p];
        const float wgt = kept ? al * Tn : 0.0f;
        gc0 = fmaf(G0[p], wgt, gc0);
        gc1 = fmaf(G1[p], wgt, gc1);
        gc2 = fmaf(G2[p], wgt, gc2);
        const float gc = fmaf(G0[p], cd.y, fmaf(G1[p], cd.z, G2[p] * cd.w));
        const float gb = fmaf(G0[p], B0[p], fmaf(G1[p], B1[p], G2[p] * B2[p]));
        // dalpha/d(o I) is 0 where alpha is clamped
        const float galpha = (kept && araw <= ALPHA_MAX) ? Tn * gc - iom * gb : 0.0f;
        B0[p] = fmaf(cd.y, wgt, B0[p]);
        B1[p] = fmaf(cd.z, wgt, B1[p]);
        B2[p] = fmaf(cd.w, wgt, B2[p]);
        const float gI = galpha * cc.w;
        go = fmaf(galpha, I, go);                             // d/do
        float gr;                                              // d/dratio
        if (WIN == WIN_SIGMOID) {
            // I = sigmoid(kappa ratio): field 9 is d/dkappa
            const float s1 = I * (1.0f - I);
            gs = fmaf(gI * s1, f.ratio, gs);
            gr = gI * cd.x * s1;
        } else {
            // (a pixel that adds zeros may have a ratio whose lg2 or reciprocal
            // is infinite: those take the values of ratio 1)
            const float lgk = kept ? lg : 0.0f, rk = kept ? rs : 1.0f;
            gs = fmaf(gI * I, lgk, gs);                        // d/dsigma / ln 2: I lg2(ratio)
            gr = gI * cd.x * I * rcp_approx(rk);
        }
        // the active line: lowest index among the minima
        const bool a0 = f.m0 <= f.m1 && f.m0 <= f.m2, a1 = !a0 && f.m1 <= f.m2;
        const float w0 = a0 ? gr : 0.f, w1 = a1 ? gr : 0.f, w2 = gr - w0 - w1;
        W[0] += w0;
        W[1] += w1;
        W[2] += w2;
        if (p & 1) {
            Wx[0] += w0;
            Wx[1] += w1;
            Wx[2] += w2;
        }
        if (p >> 1) {
            Wy[0] += w0;
            Wy[1] += w1;
            Wy[2] += w2;
        }
    }
    gv[0] = -fmaf(ca.z, W[0], fmaf(cb.y, W[1], cc.x * W[2]));
    gv[1] = -fmaf(ca.w, W[0], fmaf(cb.z, W[1], cc.y * W[2]));
    gv[2] = fmaf(dx0, W[0], Wx[0]);
    gv[3] = fmaf(dy0, W[0], Wy[0]);
    gv[4] = fmaf(dx0, W[1], Wx[1]);
    gv[5] = fmaf(dy0, W[1], Wy[1]);
    gv[6] = fmaf(dx0, W[2], Wx[2]);
    gv[7] = fmaf(dy0, W[2], Wy[2]);
    gv[8] = go;
    gv[9] = WIN == WIN_SIGMOID ? gs : gs * 0.69314718055994531f;
    gv[10] = gc0;
    gv[11] = gc1;
    gv[12] = gc2;
    return any;
}

// A record no pixel composites, for the forward's lanes with no pair of their own in a
// walk step (so that they take the step's straight-line code with the others instead of
// a path of their own): its first edge line is at 1e30 (ratio < 0 everywhere), its opacity,
// sigma and colour 0, so every term it adds is a finite zero.
__device__ __forceinline__ void put_null_record(float4 *r) {
    r[0] = make_float4(1e30f, 1e30f, 1.0f, 0.0f);
    r[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    r[2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    r[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ float4 shfl_xor4(float4 v, int m) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                       __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}

template <int WIN>
__global__ void __launch_bounds__(BW_THREADS, BW_CTAS)
render_bwd_kernel(RenderArgs a) {
    // per warp: the window's records (stride of 5 float4 so that the lanes' reads of
    // different records spread over the banks) and item ids
    __shared__ float4 s_rec[BW_WARPS][32 * BW_WIN][BW_RSTRIDE];
    __shared__ uint32_t s_it[BW_WARPS][32 * BW_WIN];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *S = s_it[w];
    float4 (*SR)[BW_RSTRIDE] = s_rec[w];
    const uint32_t n_units = (uint32_t)a.total_tiles * 2u;
    const Rec *__restrict__ recs = a.recs;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(&a.ctl->work_counter[1], 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        // tiles in the forward's order (longest first), each as its two halves
        uint32_t tq = u >> 1;
        if (a.tile_order) {
            const uint32_t t = a.tile_order[tq];
            if (t < (uint32_t)a.total_tiles) tq = t;
            else if (lane == 0) atomicOr(&a.ctl->error, ERR_INDEX);
        }
        const int tile = (int)tq, h = (int)(u & 1u);
        const int vw = find_view_warp(a.views, a.nviews, tile, lane);
        const ViewDev *V = a.views + vw;
        const int lt = tile - V->tile_base;
        // this lane's group: group g of 8x4 block b of the tile
        const int b = 4 * h + (lane >> 3), g = lane & 7;
        const int x0 = (lt % V->tiles_x) * TILE + ((b & 1) << 3) + ((g & 3) << 1);
        const int y0 = (lt / V->tiles_x) * TILE + ((b >> 1) << 2) + ((g >> 2) << 1);
        const int64_t HW = (int64_t)V->W * V->H;
        const float *dL = view_out(a, vw).dL;
        // the four pixels: (x0 + (p & 1), y0 + (p >> 1))
        float T[4], G0[4], G1[4], G2[4], B0[4], B1[4], B2[4];
        uint32_t last[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int x = x0 + (p & 1), y = y0 + (p >> 1);
            T[p] = 1.f; G0[p] = G1[p] = G2[p] = 0.f; last[p] = 0u;
            if (x < V->W && y < V->H) {
                const int64_t pix = (int64_t)y * V->W + x;
                T[p] = a.T_final[V->pix_base + pix];
                last[p] = (uint32_t)a.n_contrib[V->pix_base + pix];
                G0[p] = dL[pix];
                G1[p] = dL[HW + pix];
                G2[p] = dL[2 * HW + pix];
            }
            B0[p] = T[p] * V->bg[0];
            B1[p] = T[p] * V->bg[1];
            B2[p] = T[p] * V->bg[2];
        }
        const uint32_t start = a.ranges[tile].x;
        const uint32_t gmax = a.tile_max[(size_t)tile * GROUPS + 8 * b + g];
        const int wmax = (int)__reduce_max_sync(0xffffffffu, gmax);
        for (int wend = wmax; wend > 0; wend -= 32 * BW_WIN) {
            const int wst = max(0, wend - 32 * BW_WIN);
            // this lane's bits of the window: bit j of word q = pair wst + 32 q + j
            uint32_t m[BW_WIN];
#pragma unroll
            for (int q = 0; q < BW_WIN; ++q) {
                const int jj = wst + 32 * q + lane;
                uint32_t word = 0u, it = 0u;
                if (jj < wend) {
                    word = a.kmask[(size_t)(start + jj) * KM_WORDS + h];
                    it = a.items[start + jj];
                    if (word && it >= a.n_items) {
                        atomicOr(&a.ctl->error, ERR_INDEX);
                        word = 0u;
                    }
                }
                S[32 * q + lane] = it;
                if (word) {
                    const float4 *rp = reinterpret_cast<const float4 *>(recs + it);
#pragma unroll
                    for (int e = 0; e < 4; ++e) SR[32 * q + lane][e] = __ldg(rp + e);
                }
                m[q] = warp_transpose_bits(word, lane);
            }
            __syncwarp();
            unsigned long long lo = ((unsigned long long)m[1] << 32) | m[0];
            unsigned long long hi = ((unsigned long long)m[3] << 32) | m[2];
            float gv[13];
            const int k4 = lane & 3;
            // Many groups per record (triangles wider than the groups) make the records'
            // reductions contend in L2: then the quads' transposed, coalesced adds below;
            // otherwise each lane adds its own record directly (fewer instructions).
            const uint32_t nb = __reduce_add_sync(0xffffffffu, (uint32_t)(__popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3])));
            const uint32_t nu = (uint32_t)(__popc(__reduce_or_sync(0xffffffffu, m[0])) + __popc(__reduce_or_sync(0xffffffffu, m[1])) +
                                           __popc(__reduce_or_sync(0xffffffffu, m[2])) + __popc(__reduce_or_sync(0xffffffffu, m[3])));
            const bool dense = nb >= BW_DENSE * nu;
            if (!dense) {
                for (;;) {
                    const int cpos = pop_last(hi, lo);
                    if (!__any_sync(0xffffffffu, cpos >= 0)) break;
                    if (cpos < 0) continue;      // (the warp's next pop meets this lane at the vote)
                    const uint32_t citem = S[cpos];
                    const float4 ca = SR[cpos][0], cb = SR[cpos][1], cc = SR[cpos][2], cd = SR[cpos][3];
                    if (group_grad<WIN>(ca, cb, cc, cd, (uint32_t)(wst + cpos), true, x0, y0, last, T, G0, G1, G2, B0, B1,
                                        B2, gv)) {
                        float *dst = a.grad2d + (size_t)citem * GRAD_FIELDS;
                        red_add_v4(dst, gv[0], gv[1], gv[2], gv[3]);
                        red_add_v4(dst + 4, gv[4], gv[5], gv[6], gv[7]);
                        red_add_v4(dst + 8, gv[8], gv[9], gv[10], gv[11]);
                        red_add_v2(dst + 12, gv[12], 0.f);
                    }
                }
            } else {
                for (;;) {
                    const int cpos = pop_last(hi, lo);
                    if (!__any_sync(0xffffffffu, cpos >= 0)) break;
                    bool any = false;
                    uint32_t citem = 0u;
                    if (cpos >= 0) {
                        citem = S[cpos];
                        const float4 ca = SR[cpos][0], cb = SR[cpos][1], cc = SR[cpos][2], cd = SR[cpos][3];
                        any = group_grad<WIN>(ca, cb, cc, cd, (uint32_t)(wst + cpos), true, x0, y0, last, T, G0, G1, G2,
                                              B0, B1, B2, gv);
                    }
                    // The four lanes of a quad exchange their records' 16-byte chunks (a 4x4
                    // transpose in two rounds) so that each vector reduction below writes one
                    // whole 64-byte record from four lanes: one coalesced request instead of four.
                    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 c0 = any ? make_float4(gv[0], gv[1], gv[2], gv[3]) : z;
                    float4 c1 = any ? make_float4(gv[4], gv[5], gv[6], gv[7]) : z;
                    float4 c2 = any ? make_float4(gv[8], gv[9], gv[10], gv[11]) : z;
                    float4 c3 = any ? make_float4(gv[12], 0.f, 0.f, 0.f) : z;
                    {
                        // lanes 0, 1 keep chunks 0, 1 and take their partner's; lanes 2, 3 chunks 2, 3
                        const bool low = !(k4 & 2);
                        const float4 ra = shfl_xor4(low ? c2 : c0, 2), rb = shfl_xor4(low ? c3 : c1, 2);
                        if (low) { c2 = ra; c3 = rb; } else { c0 = ra; c1 = rb; }
                    }
                    {
                        // even lanes keep slots 0, 2, odd lanes slots 1, 3, and take the partner's
                        const bool ev = !(k4 & 1);
                        const float4 ra = shfl_xor4(ev ? c1 : c0, 1), rb = shfl_xor4(ev ? c3 : c2, 1);
                        const float4 n0 = ev ? c0 : c1, n1 = ev ? c2 : c3;
                        c0 = n0; c1 = n1; c2 = ra; c3 = rb;
                    }
                    // lane k now holds chunk k of the quad's records (0, 2, 1, 3) in its slots
                    // (odd lanes (1, 3, 0, 2), put in the same order)
                    if (k4 & 1) {
                        const float4 t0 = c0, t1 = c1;
                        c0 = c2; c1 = c3; c2 = t0; c3 = t1;
                    }
                    const int qb = lane & ~3;
                    const uint32_t vi = any ? citem : 0xffffffffu;
                    const uint32_t i0 = __shfl_sync(0xffffffffu, vi, qb), i1 = __shfl_sync(0xffffffffu, vi, qb + 1);
                    const uint32_t i2 = __shfl_sync(0xffffffffu, vi, qb + 2), i3 = __shfl_sync(0xffffffffu, vi, qb + 3);
                    if (i0 != 0xffffffffu) red_add_v4(a.grad2d + (size_t)i0 * GRAD_FIELDS + 4 * k4, c0.x, c0.y, c0.z, c0.w);
                    if (i2 != 0xffffffffu) red_add_v4(a.grad2d + (size_t)i2 * GRAD_FIELDS + 4 * k4, c1.x, c1.y, c1.z, c1.w);
                    if (i1 != 0xffffffffu) red_add_v4(a.grad2d + (size_t)i1 * GRAD_FIELDS + 4 * k4, c2.x, c2.y, c2.z, c2.w);
                    if (i3 != 0xffffffffu) red_add_v4(a.grad2d + (size_t)i3 * GRAD_FIELDS + 4 * k4, c3.x, c3.y, c3.z, c3.w);
                }
            }
            __syncwarp();
        }
    }
    if (last_cta_done(&a.ctl->done[1]) && threadIdx.x == 0) a.ctl->work_counter[1] = 0u;
}

// ---------------------------------------------------------------------------------
// Forward, one lane per 2x2 group (the backward's layout): a warp takes one half tile
// (16x8 pixels, the 32 groups of word h of the pairs' group masks; lane l owns group l)
// and composites the tile's records front to back in windows of FW_WIN * 32 pairs. The
// lane of pair j gathers the pair's record, tests it against the 32 groups (group_cover)
// and stages it in shared memory when any group may see it; the window's coverage words
// are transposed across the warp so that each lane holds the bit list of the pairs its
// group may see, and walks it in order, compositing its four pixels in straight-line code
// with the arithmetic of one pixel per thread. The kept bits go back through the same
// transpose as the pairs' group masks for the backward. No CTA-wide barrier: a warp
// leaves its half tile when its 32 groups have stopped.
constexpr int FW_THREADS = 128;
constexpr int FW_WARPS = FW_THREADS / 32;
#ifndef FW_WIN
#define FW_WIN 2                 // mask words per lane per window (64 pairs)
#endif
#ifndef FW_CTAS
#define FW_CTAS 5
#endif

// One edge line's bound on the group column of each of the half tile's 4 group rows:
// line (A, B, C) about s = (sx, sy) can reach `t` at a pixel centre of group column c of
// row r only if c >= lo[r] (A > 0) or c <= hi[r] (A < 0). Each row takes its best
// pixel row (the lower one when B >= 0) and the column bound from one division, widened
// by a slack that covers its rounding; ex bounds |p.x - sx| over the half tile.
__device__ __forceinline__ void line_cols(float A, float B, float C, float sx, float sy, int X0, int Y0, float ex,
                                          float t, int (&lo)[4], int (&hi)[4]) {
    const float dy0 = __fsub_rn((float)Y0 + (B >= 0.f ? 1.5f : 0.5f), sy);
    const float dxs = __fsub_rn(sx, (float)X0);
    if (fabsf(A) < 1e-6f) {
        // (nearly) horizontal line: the row passes where its best value can reach t
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float need = t - C - B * (dy0 + 2.0f * (float)r);
            if (need > fabsf(A) * ex) lo[r] = 8;
        }
        return;
    }
    const float rA = rcp_approx(A);
    const float num = t - C - B * dy0;
    // column bound of row r: 0.5 (sx - X0 - off) + 0.5 (t - C - B dy_r) / A
    const float al = fmaf(0.5f, dxs - (A > 0.f ? 1.5f : 0.5f), 0.5f * num * rA);
    const float be = B * rA;
    const float sl = 0.05f + 1e-6f * (fabsf(dxs) + fabsf(rA) * (fabsf(t) + fabsf(C) + fabsf(B * dy0)) + 4.0f * fabsf(be));
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float v = fminf(fmaxf(fmaf(-(float)r, be, al), -4.0f), 12.0f);
        if (A > 0.f) lo[r] = max(lo[r], (int)ceilf(v - sl));
        else hi[r] = min(hi[r], (int)floorf(v + sl));
    }
}

// Bit l set when the record (cutoff ratio thr) may composite at a pixel centre of 2x2
// group l of the half tile with pixel origin (X0, Y0): group l sits at column
// c = 4 ((l >> 3) & 1) + (l & 3) and row r = 2 (l >> 4) + ((l >> 2) & 1), pixels
// (X0 + 2c + {0, 1}, Y0 + 2r + {0, 1}). The record's pixel rectangle and each edge
// line bound the columns of each row; the margin covers the FP32 rounding of the
// per-pixel evaluation, as in line_reaches.
__device__ __forceinline__ uint32_t group_cover(const Rec &r, const ushort4 bx, int X0, int Y0, float thr) {
    const float sx = r.a.x, sy = r.a.y;
    const float ex = fmaxf(fabsf((float)X0 + 0.5f - sx), fabsf((float)X0 + 15.5f - sx));
    const float ey = fmaxf(fabsf((float)Y0 + 0.5f - sy), fabsf((float)Y0 + 7.5f - sy));
    const int clo = ((int)bx.x - X0) >> 1, chi = ((int)bx.z - X0) >> 1;
    int lo[4], hi[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool rows = (int)bx.y <= Y0 + 2 * q + 1 && (int)bx.w >= Y0 + 2 * q;
        lo[q] = rows ? max(clo, 0) : 8;
        hi[q] = min(chi, 7);
    }
    const float C0 = line_offset(r.a.z, r.a.w, r.b), C1 = line_offset(r.b.y, r.b.z, r.b),
                C2 = line_offset(r.c.x, r.c.y, r.b);
    line_cols(r.a.z, r.a.w, C0, sx, sy, X0, Y0, ex,
              thr - (1e-3f + 4e-7f * (fabsf(r.a.z) * ex + fabsf(r.a.w) * ey + fabsf(C0))), lo, hi);
    line_cols(r.b.y, r.b.z, C1, sx, sy, X0, Y0, ex,
              thr - (1e-3f + 4e-7f * (fabsf(r.b.y) * ex + fabsf(r.b.z) * ey + fabsf(C1))), lo, hi);
    line_cols(r.c.x, r.c.y, C2, sx, sy, X0, Y0, ex,
              thr - (1e-3f + 4e-7f * (fabsf(r.c.x) * ex + fabsf(r.c.y) * ey + fabsf(C2))), lo, hi);
    uint32_t word = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int l = min(max(lo[q], 0), 8), h = min(max(hi[q], -1), 7);
        const uint32_t M = (0xFFu << l) & (0xFFu >> (7 - h));
        const int base = 16 * (q >> 1) + 4 * (q & 1);
        word |= ((M & 0xFu) << base) | (((M >> 4) & 0xFu) << (base + 8));
    }
    return word;
}

// Composite one record (ca..cd, tile-list position jt1 - 1) at the lane's four pixels
// (x0 + (p & 1), y0 + (p >> 1)), front to back, in straight-line code with the per-pixel
// arithmetic of the rendering equation: bit p of `done` marks a pixel that has stopped.
// Returns whether any pixel composited; STATS: the largest T o of those and their count.
template <bool SOLID, int WIN, bool STATS, bool COUNT>
__device__ __forceinline__ bool group_fwd(const float4 ca, const float4 cb, const float4 cc, const float4 cd,
                                          uint32_t jt1, int x0, int y0, float (&T)[4], float (&C0)[4],
                                          float (&C1)[4], float (&C2)[4], uint32_t (&last)[4], uint32_t &done,
                                          float &sw, uint32_t &sn, uint32_t &n_eval, uint32_t &n_kept) {
    bool any = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float px = (float)(x0 + (p & 1)) + 0.5f, py = (float)(y0 + (p >> 1)) + 0.5f;
        const bool live = !((done >> p) & 1u);
        if (COUNT) n_eval += live ? 1u : 0u;
        const Frag f = eval_lines(ca, cb, cc, px, py);
        if (SOLID) {
            const bool hit = live && f.ratio > 0.0f;
            C0[p] = hit ? cd.y : C0[p];
            C1[p] = hit ? cd.z : C1[p];
            C2[p] = hit ? cd.w : C2[p];
            T[p] = hit ? 0.0f : T[p];
            last[p] = hit ? jt1 : last[p];
            done |= hit ? 1u << p : 0u;
            if (COUNT) n_kept += hit ? 1u : 0u;
            any = any || hit;
            continue;
        }
        // (a power-window ratio <= 0 gives alpha 0 or NaN, which the threshold test skips)
        const float I = WIN == WIN_SIGMOID ? window_sigmoid(f.ratio, cd.x) : window_pow(f.ratio, cd.x);
        const float araw = __fmul_rn(cc.w, I);
        const bool act = live && araw >= ALPHA_MIN;
        const float al = fminf(araw, ALPHA_MAX);
        const float tT = __fmul_rn(T[p], __fsub_rn(1.0f, al));
        const bool stop = act && tT < T_EPS;
        const bool comp = act && !stop;
        done |= stop ? 1u << p : 0u;
        // a pixel that does not composite adds rgb x 0 (colours are finite and >= 0)
        const float wgt = comp ? __fmul_rn(al, T[p]) : 0.0f;
        if (STATS && comp) {
            // Sec. 3.3 "Pruning": blending weight T o of this fragment
            sw = fmaxf(sw, __fmul_rn(T[p], cc.w));
            ++sn;
        }
        C0[p] = fmaf(cd.y, wgt, C0[p]);
        C1[p] = fmaf(cd.z, wgt, C1[p]);
        C2[p] = fmaf(cd.w, wgt, C2[p]);
        T[p] = comp ? tT : T[p];
        last[p] = comp ? jt1 : last[p];
        if (COUNT) n_kept += comp ? 1u : 0u;
        any = any || comp;
    }
    return any;
}

// Lowest set bit of the list (hi:lo), cleared; -1 when empty.
__device__ __forceinline__ int pop_first(unsigned long long &hi, unsigned long long &lo) {
    if (lo) {
        const int b = __ffsll((long long)lo) - 1;
        lo &= lo - 1ull;
        return b;
    }
    if (hi) {
        const int b = __ffsll((long long)hi) - 1;
        hi &= hi - 1ull;
        return 64 + b;
    }
    return -1;
}

template <bool SOLID, int WIN, bool STATS, bool COUNT>
__global__ void __launch_bounds__(FW_THREADS, FW_CTAS)
render_fwd_kernel(RenderArgs a) {
    // per warp: the window's records (stride of 5 float4: lanes reading different
    // records spread over the banks), item ids and the pruning statistics of each pair
    // (slot 32 FW_WIN: the null record)
    __shared__ float4 s_rec[FW_WARPS][32 * FW_WIN + 1][BW_RSTRIDE];
    __shared__ uint32_t s_it[FW_WARPS][32 * FW_WIN];
    __shared__ uint32_t s_sw[STATS ? FW_WARPS : 1][32 * FW_WIN];
    __shared__ uint32_t s_sn[STATS ? FW_WARPS : 1][32 * FW_WIN];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *S = s_it[w];
    float4 (*SR)[BW_RSTRIDE] = s_rec[w];
    if (lane == 0) put_null_record(SR[32 * FW_WIN]);
    __syncwarp();
    if (STATS) {
#pragma unroll
        for (int q = 0; q < FW_WIN; ++q) s_sw[w][32 * q + lane] = s_sn[w][32 * q + lane] = 0u;
    }
    const uint32_t n_units = (uint32_t)a.total_tiles * 2u;
    const Rec *__restrict__ recs = a.recs;
    float l1_acc = 0.f;                 // this lane's share of the L1 loss
    uint32_t n_eval = 0, n_kept = 0;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(&a.ctl->work_counter[0], 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= n_units) break;
        // tiles in the binning's order (longest first), each as its two halves
        uint32_t tq = u >> 1;
        if (a.tile_order) {
            const uint32_t t = a.tile_order[tq];
            if (t < (uint32_t)a.total_tiles) tq = t;
            else if (lane == 0) atomicOr(&a.ctl->error, ERR_INDEX);
        }
        const int tile = (int)tq, h = (int)(u & 1u);
        const int vw = find_view_warp(a.views, a.nviews, tile, lane);
        const ViewDev *V = a.views + vw;
        const int lt = tile - V->tile_base;
        const int X0 = (lt % V->tiles_x) * TILE, Y0 = (lt / V->tiles_x) * TILE + 8 * h;
        // this lane's group: column c = 4 ((lane >> 3) & 1) + (lane & 3), row
        // r = 2 (lane >> 4) + ((lane >> 2) & 1) of the half tile
        const int x0 = X0 + 8 * ((lane >> 3) & 1) + 2 * (lane & 3);
        const int y0 = Y0 + 4 * (lane >> 4) + 2 * ((lane >> 2) & 1);
        const int W = V->W, H = V->H;
        float T[4], C0[4], C1[4], C2[4];
        uint32_t last[4], done = 0u;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            T[p] = 1.0f;
            C0[p] = C1[p] = C2[p] = 0.0f;
            last[p] = 0u;
            if (x0 + (p & 1) >= W || y0 + (p >> 1) >= H) done |= 1u << p;
        }
        const uint2 rg = a.ranges[tile];
        const uint32_t start = rg.x;
        const int n = rg.y > rg.x ? (int)(rg.y - rg.x) : 0;
        // item ids of the window, loaded one window ahead
        uint32_t nit[FW_WIN];
#pragma unroll
        for (int q = 0; q < FW_WIN; ++q) nit[q] = 32 * q + lane < n ? a.items[start + 32 * q + lane] : 0u;
        for (int wst = 0; wst < n; wst += 32 * FW_WIN) {
            if (__all_sync(0xffffffffu, done == 0xFu)) break;
            // this lane's bits of the window: bit j of word q = pair wst + 32 q + j
            uint32_t m[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int q = 0; q < FW_WIN; ++q) {
                const int jj = wst + 32 * q + lane;
                uint32_t word = 0u, it = 0u;
                if (jj < n) {
                    it = nit[q];
                    if (it >= a.n_items) {
                        atomicOr(&a.ctl->error, ERR_INDEX);
                        it = 0u;
                    } else {
                        const Rec r = recs[it];
                        word = group_cover(r, a.rects[it], X0, Y0, cutoff_ratio<WIN>(r, SOLID));
                        if (word) {
                            SR[32 * q + lane][0] = r.a;
                            SR[32 * q + lane][1] = r.b;
                            SR[32 * q + lane][2] = r.c;
                            SR[32 * q + lane][3] = r.d;
                        }
                    }
                }
                S[32 * q + lane] = it;
                m[q] = warp_transpose_bits(word, lane);
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < FW_WIN; ++q) {
                const int jn = wst + 32 * FW_WIN + 32 * q + lane;
                nit[q] = jn < n ? a.items[start + jn] : 0u;
            }
            unsigned long long lo = ((unsigned long long)m[1] << 32) | m[0];
            unsigned long long hi = ((unsigned long long)m[3] << 32) | m[2];
            unsigned long long klo = 0ull, khi = 0ull;   // pairs this lane's group composited
            for (;;) {
                int cpos = pop_first(hi, lo);
                if (done == 0xFu) cpos = -1;     // (a lane whose pixels have all stopped drops its list)
                if (!__any_sync(0xffffffffu, cpos >= 0)) break;
                // (a lane with no pair takes the null record, or, when counting fragments,
                // meets the others at the next vote)
                if (COUNT && cpos < 0) continue;
                const int slot = cpos >= 0 ? cpos : 32 * FW_WIN;
                const float4 ca = SR[slot][0], cb = SR[slot][1], cc = SR[slot][2], cd = SR[slot][3];
                float sw = 0.0f;
                uint32_t sn = 0u;
                if (group_fwd<SOLID, WIN, STATS, COUNT>(ca, cb, cc, cd, (uint32_t)(wst + slot + 1), x0, y0, T, C0, C1,
                                                        C2, last, done, sw, sn, n_eval, n_kept)) {
                    if (cpos < 64) klo |= 1ull << cpos;
                    else khi |= 1ull << (cpos - 64);
                    if (STATS) {
                        atomicMax(&s_sw[w][cpos], __float_as_uint(sw));
                        atomicAdd(&s_sn[w][cpos], sn);
                    }
                }
            }
            if (a.kmask) {
                // back through the transpose: lane j gets the groups that composited pair j
#pragma unroll
                for (int q = 0; q < FW_WIN; ++q) {
                    const unsigned long long src = q < 2 ? klo : khi;
                    const uint32_t kw = (uint32_t)(src >> (32 * (q & 1)));
                    const uint32_t word = warp_transpose_bits(kw, lane);
                    const int jj = wst + 32 * q + lane;
                    if (jj < n) a.kmask[(size_t)(start + jj) * KM_WORDS + h] = word;
                }
            }
            if (STATS) {
                __syncwarp();
#pragma unroll
                for (int q = 0; q < FW_WIN; ++q) {
                    const int k = 32 * q + lane;
                    const uint32_t sn = s_sn[w][k];
                    if (sn) {
                        atomicAdd(&a.stat_n[S[k]], sn);
                        atomicMax(&a.stat_w[S[k]], s_sw[w][k]);
                    }
                    s_sn[w][k] = 0u;
                    s_sw[w][k] = 0u;
                }
            }
            __syncwarp();
        }
        const int64_t HW = (int64_t)W * H;
        const ViewOut vo = view_out(a, vw);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int x = x0 + (p & 1), y = y0 + (p >> 1);
            if (x >= W || y >= H) continue;
            const int64_t pix = (int64_t)y * W + x;
            const float c[3] = {fmaf(T[p], V->bg[0], C0[p]), fmaf(T[p], V->bg[1], C1[p]), fmaf(T[p], V->bg[2], C2[p])};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) vo.image[ch * HW + pix] = c[ch];
            if (vo.target) {
                // the L1 loss of the pixel and its gradient, while the colour is in registers
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float d = c[ch] - vo.target[ch * HW + pix];
                    l1_acc += fabsf(d);
                    vo.grad[ch * HW + pix] = l1_sign(d, a.loss_scale);
                }
            }
            a.T_final[V->pix_base + pix] = T[p];
            a.n_contrib[V->pix_base + pix] = (int32_t)last[p];
            if (SOLID && a.ids)
                a.ids[V->pix_base + pix] =
                    last[p] ? (int32_t)((int64_t)a.items[start + last[p] - 1] - (int64_t)vw * a.n_per_view) : -1;
        }
        a.tile_max[(size_t)tile * GROUPS + 32 * h + lane] = max(max(last[0], last[1]), max(last[2], last[3]));
    }
    if (COUNT) {
        const uint32_t we = __reduce_add_sync(0xffffffffu, n_eval), wk = __reduce_add_sync(0xffffffffu, n_kept);
        if (lane == 0) {
            atomicAdd(&a.ctl->frag_eval, (unsigned long long)we);
            atomicAdd(&a.ctl->frag_kept, (unsigned long long)wk);
        }
    }
    if (a.loss) {
        float v = l1_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(a.loss, v * a.loss_scale);
    }
    if (last_cta_done(&a.ctl->done[0]) && threadIdx.x == 0) a.ctl->work_counter[0] = 0u;
}

static int occupancy(const void *fn, int threads) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) occ = 1;
    return occ;
}

template <bool STATS, bool COUNT>
static void launch_fwd_kind(const RenderArgs &a, unsigned g, cudaStream_t st, bool solid) {
    if (solid) render_fwd_kernel<true, WIN_POWER, false, COUNT><<<g, FW_THREADS, 0, st>>>(a);
    else if (a.window == WIN_SIGMOID) render_fwd_kernel<false, WIN_SIGMOID, STATS, COUNT><<<g, FW_THREADS, 0, st>>>(a);
    else render_fwd_kernel<false, WIN_POWER, STATS, COUNT><<<g, FW_THREADS, 0, st>>>(a);
}

void launch_render_fwd(const RenderArgs &a, int grid, cudaStream_t st, bool solid) {
    static int occ = occupancy((const void *)render_fwd_kernel<false, WIN_POWER, false, false>, FW_THREADS);
    int64_t g = grid > 0 ? (int64_t)grid * occ : occ;
    const int64_t need = ((int64_t)a.total_tiles * 2 + FW_WARPS - 1) / FW_WARPS;
    if (g > need) g = need;
    if (g <= 0) return;
    const bool stats = a.stat_n != nullptr && !solid;
    if (stats) {
        if (a.count_frags) launch_fwd_kind<true, true>(a, (unsigned)g, st, solid);
        else launch_fwd_kind<true, false>(a, (unsigned)g, st, solid);
    } else {
        if (a.count_frags) launch_fwd_kind<false, true>(a, (unsigned)g, st, solid);
        else launch_fwd_kind<false, false>(a, (unsigned)g, st, solid);
    }
}

void launch_render_bwd(const RenderArgs &a, int grid, cudaStream_t st) {
    static int occ = occupancy((const void *)render_bwd_kernel<WIN_POWER>, BW_THREADS);
    int64_t g = grid > 0 ? (int64_t)grid * occ : occ;
    const int64_t need = ((int64_t)a.total_tiles * 2 + BW_WARPS - 1) / BW_WARPS;
    if (g > need) g = need;
    if (g <= 0) return;
    if (a.window == WIN_SIGMOID) render_bwd_kernel<WIN_SIGMOID><<<(unsigned)g, BW_THREADS, 0, st>>>(a);
    else render_bwd_kernel<WIN_POWER><<<(unsigned)g, BW_THREADS, 0, st>>>(a);
}

// ---------------------------------------------------------------------------------
// Per-pixel sort (the ordering the paper leaves to future work after its per-tile
// centroid sort): each pixel's fragments composite in the order of the depth of their
// triangle's plane along the pixel's ray, z(p) = 1 / (a (p.x - cx) + b (p.y - cy) + c)
// from the item's inverse-depth plane, ties to the lower item id. Three passes over
// each tile's list: count the pixel's candidates (alpha >= 1/255), scan the counts
// into offsets, then write the candidates as (z bits << 32 | item), sort each pixel's
// run on its own thread and composite: the run becomes a min-heap and fragments are
// taken nearest first until transmittance stops the pixel (O(n + k log n) for k
// composited of n candidates), each taken one moving to the run's free tail, so the
// k composited fragments end at positions [n - k, n), the farthest first.
// The backward walks those positions in order (back to front), one thread per pixel,
// adding each fragment's 13 gradient fields to its item with four vector reductions.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ float pps_depth(const float4 zp, const ViewDev &V, float px, float py) {
    return 1.0f / fmaf(zp.x, px - V.cx, fmaf(zp.y, py - V.cy, zp.z));
}

// Fragment alpha o I of record r at (px, py) before the clamp (0 below 1/255), as the
// tile-sorted forward; the window value into I.
template <int WIN>
__device__ __forceinline__ float pps_alpha(const Rec &r, float px, float py, Frag &f, float &I) {
    f = eval_lines(r.a, r.b, r.c, px, py);
    I = 0.0f;
    if (WIN == WIN_POWER && f.ratio <= 0.0f) return 0.0f;
    I = WIN == WIN_SIGMOID ? window_sigmoid(f.ratio, r.d.x) : window_pow(f.ratio, r.d.x);
    const float al = __fmul_rn(r.c.w, I);
    return al < ALPHA_MIN ? 0.0f : al;
}

// Min-heap of a pixel's run: v[i] <= v[2 i + 1], v[2 i + 2].
__device__ __forceinline__ void heap_sift_down(unsigned long long *v, int i, int end) {
    const unsigned long long x = v[i];
    while (true) {
        int c = 2 * i + 1;
        if (c >= end) break;
        if (c + 1 < end && v[c + 1] < v[c]) ++c;
        if (v[c] >= x) break;
        v[i] = v[c];
        i = c;
    }
    v[i] = x;
}

// PASS 0: candidate counts; PASS 1: candidates, per-pixel sort, compositing.
template <int PASS, int WIN>
__global__ void __launch_bounds__(REN_THREADS) pps_tile_kernel(RenderArgs a) {
    __shared__ Rec s_rec[REN_THREADS];
    __shared__ float4 s_zp[REN_THREADS];
    __shared__ uint32_t s_item[REN_THREADS];
    __shared__ uint16_t s_mask[REN_THREADS];
    __shared__ uint8_t s_list[REN_THREADS / 32][REN_THREADS];
    __shared__ ViewDev s_view[MAX_VIEWS];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int k = tid; k < a.nviews * (int)(sizeof(ViewDev) / 4); k += REN_THREADS)
        reinterpret_cast<uint32_t *>(s_view)[k] = reinterpret_cast<const uint32_t *>(a.views)[k];
    int lx, ly;
    pixel_of(tid, lx, ly);
    const uint8_t *L = s_list[w];
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&a.ctl->work_counter[PASS == 0 ? 0 : 3], 1u);
        __syncthreads();
        const int tile = (int)s_tile;
        if (tile >= a.total_tiles) break;
        const int vw = find_view(s_view, a.nviews, tile);
        const ViewDev &V = s_view[vw];
        const int lt = tile - V.tile_base;
        const int ox = (lt % V.tiles_x) * TILE, oy = (lt / V.tiles_x) * TILE;
        const int x = ox + lx, y = oy + ly;
        const bool inside = x < V.W && y < V.H;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const int64_t pg = inside ? V.pix_base + (int64_t)y * V.W + x : 0;
        const uint2 rg = a.ranges[tile];
        const uint32_t start = rg.x, end = rg.y > rg.x ? rg.y : rg.x;
        uint32_t cnt = 0, want = 0;
        unsigned long long off = 0;
        if (PASS == 1 && inside) {
            off = a.poff[pg];
            want = a.pcount[pg];
        }
        for (uint32_t b0 = start; b0 < end; b0 += REN_THREADS) {
            __syncthreads();
            const uint32_t idx = b0 + tid;
            if (idx < end) {
                uint32_t it = a.items[idx];
                if (it >= a.n_items) {
                    atomicOr(&a.ctl->error, ERR_INDEX);
                    it = 0;
                }
                const Rec r = a.recs[it];
                s_rec[tid] = r;
                s_item[tid] = it;
                if (PASS == 1) s_zp[tid] = a.zplane[it];
                s_mask[tid] = (uint16_t)warp_mask(r, a.rects[it], ox, oy, cutoff_ratio<WIN>(r, false));
            } else {
                s_mask[tid] = 0;
            }
            __syncthreads();
            const int n = warp_list(s_mask, s_list[w], w, lane);
            if (!inside) continue;
            for (int k = 0; k < n; ++k) {
                const int j = L[k];
                Frag f;
                float I;
                if (pps_alpha<WIN>(s_rec[j], px, py, f, I) <= 0.0f) continue;
                if (PASS == 1) {
                    if (cnt < want && off + cnt < a.cand_cap) {
                        const float z = pps_depth(s_zp[j], V, px, py);
                        a.cand[off + cnt] = ((unsigned long long)__float_as_uint(z) << 32) | s_item[j];
                    } else {
                        atomicOr(&a.ctl->error, ERR_INDEX);
                    }
                }
                ++cnt;
            }
        }
        if (PASS == 0) {
            if (inside) a.pcount[pg] = cnt;
        } else if (inside) {
            const int m = (int)min(cnt, want);
            const bool fits = cnt == want && off + (unsigned long long)m <= a.cand_cap;
            unsigned long long *run = a.cand + off;
            float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
            uint32_t last = 0;   // fragments composited
            if (fits) {
                for (int i = m / 2 - 1; i >= 0; --i) heap_sift_down(run, i, m);
                for (int end = m; end > 0;) {
                    const unsigned long long top = run[0];
                    --end;
                    run[0] = run[end];
                    heap_sift_down(run, 0, end);
                    run[end] = top;
                    const uint32_t it = (uint32_t)top;
                    const Rec r = a.recs[it];
                    Frag f;
                    float I;
                    float al = fminf(pps_alpha<WIN>(r, px, py, f, I), ALPHA_MAX);
                    const float tT = __fmul_rn(T, __fsub_rn(1.0f, al));
                    if (tT < T_EPS) break;
                    const float wgt = __fmul_rn(al, T);
                    C0 = fmaf(r.d.y, wgt, C0);
                    C1 = fmaf(r.d.z, wgt, C1);
                    C2 = fmaf(r.d.w, wgt, C2);
                    T = tT;
                    ++last;
                }
            }
            const int64_t HW = (int64_t)V.W * V.H;
            const int64_t pix = (int64_t)y * V.W + x;
            float *img = view_out(a, vw).image;
            img[pix] = fmaf(T, V.bg[0], C0);
            img[HW + pix] = fmaf(T, V.bg[1], C1);
            img[2 * HW + pix] = fmaf(T, V.bg[2], C2);
            a.T_final[pg] = T;
            a.n_contrib[pg] = (int32_t)last;
        }
        __syncthreads();   // every thread has read s_tile before it changes
    }
    if (last_cta_done(&a.ctl->done[PASS == 0 ? 4 : 5]) && tid == 0) a.ctl->work_counter[PASS == 0 ? 0 : 3] = 0u;
}

__host__ __device__ size_t pps_scan_status_words(int64_t total_pix) { return (size_t)((total_pix + 1023) / 1024) + 1; }

// Exclusive scan of the per-pixel counts into 64-bit offsets (single pass, decoupled
// look-back over 1024-count blocks, CTA order by ticket); the total into ctl->pps_total.
__global__ void __launch_bounds__(256) pps_scan_kernel(RenderArgs a) {
    __shared__ unsigned long long s_w[9];
    __shared__ uint32_t s_cta;
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_cta = atomicAdd(&a.ctl->cta_counter[4], 1u);
    __syncthreads();
    const uint32_t cta = s_cta;
    const int64_t p0 = (int64_t)cta * 1024 + tid * 4;
    uint32_t c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = p0 + q < a.total_pix ? a.pcount[p0 + q] : 0u;
    const unsigned long long sum = (unsigned long long)c[0] + c[1] + c[2] + c[3];
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const unsigned long long v = lane < 8 ? s_w[lane] : 0ull;
        unsigned long long t = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, t, 7);
        if (lane < 8) s_w[lane] = t - v;
        const unsigned long long b =
            warp_lookback_excl64(reinterpret_cast<uint64_t *>(a.pscan_status), cta, total, &a.ctl->error);
        if (lane == 0) {
            s_base = b;
            if ((int64_t)(cta + 1) * 1024 >= a.total_pix) a.ctl->pps_total = b + total;
        }
    }
    __syncthreads();
    unsigned long long off = s_base + s_w[w] + x - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (p0 + q < a.total_pix) a.poff[p0 + q] = off;
        off += c[q];
    }
    if (last_cta_done(&a.ctl->done[6])) {
        // every CTA's look-back is over: clear the status words and the ticket
        const int64_t words = (int64_t)pps_scan_status_words(a.total_pix);
        for (int64_t k = tid; k < words; k += 256) a.pscan_status[k] = 0ull;
        if (tid == 0) a.ctl->cta_counter[4] = 0u;
    }
}


// Backward of the per-pixel sort: one thread per pixel, its sorted run from the last
// composited fragment back to the first.
template <int WIN>
__global__ void __launch_bounds__(256) pps_bwd_kernel(RenderArgs a) {
    for (int64_t pg = (int64_t)blockIdx.x * 256 + threadIdx.x; pg < a.total_pix;
         pg += (int64_t)gridDim.x * 256) {
        int vw = 0;
        for (int k = 1; k < a.nviews; ++k)
            if (a.views[k].pix_base <= pg) vw = k;
        const ViewDev &V = a.views[vw];
        const int64_t pix = pg - V.pix_base;
        const int x = (int)(pix % V.W), y = (int)(pix / V.W);
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const int64_t HW = (int64_t)V.W * V.H;
        const float *dL = view_out(a, vw).dL;
        const float g0 = dL[pix], g1 = dL[HW + pix], g2 = dL[2 * HW + pix];
        float T = a.T_final[pg];
        float B0 = T * V.bg[0], B1 = T * V.bg[1], B2 = T * V.bg[2];
        const int last = a.n_contrib[pg];
        // the composited fragments at [n - last, n), the farthest first
        const unsigned long long *run = a.cand + a.poff[pg] + a.pcount[pg] - last;
        for (int k = 0; k < last; ++k) {
            const uint32_t it = (uint32_t)run[k];
            if (it >= a.n_items) {
                atomicOr(&a.ctl->error, ERR_INDEX);
                continue;
            }
            const Rec r = a.recs[it];
            Frag f;
            float I;
            const float araw = pps_alpha<WIN>(r, px, py, f, I);
            if (araw <= 0.0f) continue;
            float gv[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) gv[q] = 0.f;
            const float al = fminf(araw, ALPHA_MAX);
            const float iom = rcp_approx(__fsub_rn(1.0f, al));
            T = T * iom;
            const float wgt = al * T;
            gv[10] = g0 * wgt;
            gv[11] = g1 * wgt;
            gv[12] = g2 * wgt;
            const float gc = fmaf(g0, r.d.y, fmaf(g1, r.d.z, g2 * r.d.w));
            const float gb = fmaf(g0, B0, fmaf(g1, B1, g2 * B2));
            const float galpha = T * gc - iom * gb;
            B0 = fmaf(r.d.y, wgt, B0);
            B1 = fmaf(r.d.z, wgt, B1);
            B2 = fmaf(r.d.w, wgt, B2);
            if (araw <= ALPHA_MAX) {
                const float gI = galpha * r.c.w;
                gv[8] = galpha * I;
                float gr;
                if (WIN == WIN_SIGMOID) {
                    const float s1 = I * (1.0f - I);
                    gv[9] = gI * s1 * f.ratio;
                    gr = gI * r.d.x * s1;
                } else {
                    gv[9] = gI * I * lg2_approx(f.ratio) * 0.69314718055994531f;
                    gr = gI * r.d.x * I * rcp_approx(f.ratio);
                }
                const int ia = (f.m0 <= f.m1 && f.m0 <= f.m2) ? 0 : (f.m1 <= f.m2 ? 1 : 2);
                const float Aa = ia == 0 ? r.a.z : (ia == 1 ? r.b.y : r.c.x);
                const float Ba = ia == 0 ? r.a.w : (ia == 1 ? r.b.z : r.c.y);
                gv[0] = -gr * Aa;
                gv[1] = -gr * Ba;
                const float gA = gr * f.dx, gB = gr * f.dy;
                gv[2] = ia == 0 ? gA : 0.f;
                gv[3] = ia == 0 ? gB : 0.f;
                gv[4] = ia == 1 ? gA : 0.f;
                gv[5] = ia == 1 ? gB : 0.f;
                gv[6] = ia == 2 ? gA : 0.f;
                gv[7] = ia == 2 ? gB : 0.f;
            }
            float *dst = a.grad2d + (size_t)it * GRAD_FIELDS;
            red_add_v4(dst, gv[0], gv[1], gv[2], gv[3]);
            red_add_v4(dst + 4, gv[4], gv[5], gv[6], gv[7]);
            red_add_v4(dst + 8, gv[8], gv[9], gv[10], gv[11]);
            red_add_v4(dst + 12, gv[12], 0.f, 0.f, 0.f);
        }
    }
}

void launch_pps_count(const RenderArgs &a, int grid, cudaStream_t st) {
    static int occ = occupancy((const void *)pps_tile_kernel<0, WIN_POWER>, REN_THREADS);
    int g = grid > 0 ? grid * occ : occ;
    if (g > a.total_tiles) g = a.total_tiles;
    if (g <= 0) return;
    if (a.window == WIN_SIGMOID) pps_tile_kernel<0, WIN_SIGMOID><<<g, REN_THREADS, 0, st>>>(a);
    else pps_tile_kernel<0, WIN_POWER><<<g, REN_THREADS, 0, st>>>(a);
}

void launch_pps_scan(const RenderArgs &a, cudaStream_t st) {
    const int64_t g = (a.total_pix + 1023) / 1024;
    if (g > 0) pps_scan_kernel<<<(unsigned)g, 256, 0, st>>>(a);
}

void launch_pps_fwd(const RenderArgs &a, int grid, cudaStream_t st) {
    static int occ = occupancy((const void *)pps_tile_kernel<1, WIN_POWER>, REN_THREADS);
    int g = grid > 0 ? grid * occ : occ;
    if (g > a.total_tiles) g = a.total_tiles;
    if (g <= 0) return;
    if (a.window == WIN_SIGMOID) pps_tile_kernel<1, WIN_SIGMOID><<<g, REN_THREADS, 0, st>>>(a);
    else pps_tile_kernel<1, WIN_POWER><<<g, REN_THREADS, 0, st>>>(a);
}

void launch_pps_bwd(const RenderArgs &a, cudaStream_t st) {
    int64_t g = (a.total_pix + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g <= 0) return;
    if (a.window == WIN_SIGMOID) pps_bwd_kernel<WIN_SIGMOID><<<(unsigned)g, 256, 0, st>>>(a);
    else pps_bwd_kernel<WIN_POWER><<<(unsigned)g, 256, 0, st>>>(a);
}

// ---------------------------------------------------------------------------------
// L1 loss: mean |image - target| and its gradient sign(image - target) / n
// ---------------------------------------------------------------------------------

// VEC: img, tgt and grad are 16-byte aligned; float4 accesses, 4 in flight per thread.
template <bool VEC>
__global__ void __launch_bounds__(256) loss_l1_kernel(const float *__restrict__ img, const float *__restrict__ tgt,
                                                      int64_t n, float *__restrict__ grad, float *loss) {
    const float inv = 1.0f / (float)n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    int64_t done = 0;
    if (VEC) {
        constexpr int U = 4;
        const int64_t n4 = n >> 2;
        const float4 *i4 = reinterpret_cast<const float4 *>(img), *g4 = reinterpret_cast<const float4 *>(tgt);
        float4 *o4 = reinterpret_cast<float4 *>(grad);
        for (int64_t i = t0; i < n4; i += U * stride) {
            float4 a[U], b[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = i + u * stride;
                if (k < n4) {
                    a[u] = __ldg(i4 + k);
                    b[u] = __ldg(g4 + k);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = i + u * stride;
                if (k < n4) {
                    const float dx = a[u].x - b[u].x, dy = a[u].y - b[u].y, dz = a[u].z - b[u].z, dw = a[u].w - b[u].w;
                    acc += (fabsf(dx) + fabsf(dy)) + (fabsf(dz) + fabsf(dw));
                    o4[k] = make_float4(l1_sign(dx, inv), l1_sign(dy, inv), l1_sign(dz, inv), l1_sign(dw, inv));
                }
            }
        }
        done = n4 << 2;
    }
    for (int64_t i = done + t0; i < n; i += stride) {
        const float d = img[i] - tgt[i];
        acc += fabsf(d);
        grad[i] = l1_sign(d, inv);
    }
    if (loss) {
        __shared__ float s_part[32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_part[k];
            atomicAdd(loss, t * inv);
        }
    }
}

void launch_loss_l1(const float *img, const float *tgt, int64_t n, float *grad, float *loss, cudaStream_t st) {
    int64_t g = (n + 255) / 256;
    if (g > 1216) g = 1216;  // 8 CTAs per SM on 152 SMs: one atomic per CTA
    if (g <= 0) return;
    const bool vec = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(tgt) |
                       reinterpret_cast<uintptr_t>(grad)) & 15u) == 0;
    if (vec) loss_l1_kernel<true><<<(unsigned)g, 256, 0, st>>>(img, tgt, n, grad, loss);
    else loss_l1_kernel<false><<<(unsigned)g, 256, 0, st>>>(img, tgt, n, grad, loss);
}

}  // namespace ts
