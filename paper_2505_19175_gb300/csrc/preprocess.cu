// Preprocess (forward and backward) of the triangle-splat renderer.
//
// Forward, one thread per triangle looping over views so that the triangle's
// parameters (36 B of vertices, up to 192 B of SH, o, sigma) are read from HBM once
// per call, staged through shared memory with coalesced float4 loads:
//   - projection, culling, normalised edge lines and incenter (Sec. 3.1);
//   - SH colour for the direction camera centre -> centroid (Sec. 4: degree 3);
//   - tight rectangle of the triangle shrunk about its incenter by
//     f = 1 - (tau/o)^(1/sigma), tau = ALPHA_MIN (Supp. "Tile assignment");
//   - the count of visible items, the per-tile pair counts of the binning and, on
//     request (the global radix-sort path of the allocation-free render), the digit
//     histograms of the 32-bit depth keys.
// Backward: the chain rule of all of the above from the per-item gradient record.
#include "geometry.cuh"
#include "kernels.h"

namespace ts {

constexpr int PRE_THREADS = 128;
constexpr int PRE_BWD_THREADS = 64;

// Asynchronous global -> shared copies (cp.async): every copy of a CTA's staging is in
// flight at once, with no register round trip.
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage `count` floats starting at `src` (16-byte aligned) into shared memory.
template <int T>
__device__ __forceinline__ void stage_floats(float *dst, const float *src, int count) {
    const int n4 = count >> 2;
    for (int k = threadIdx.x; k < n4; k += T) cp_async16(dst + 4 * k, src + 4 * k);
    for (int k = (n4 << 2) + threadIdx.x; k < count; k += T) cp_async4(dst + k, src + k);
}

// Shared-memory layout of per-thread records of `len` floats. With len a multiple of 4
// the records are read as float4 at a stride of an odd number of float4 (conflict-free
// per quarter-warp) and staged with 16-byte copies; otherwise they are read as floats
// at an odd stride (conflict-free per warp) and staged with 4-byte copies.
template <int len>
struct RecLayout {
    static constexpr bool V4 = len % 4 == 0;
    static constexpr int stride = V4 ? ((len / 4) % 2 ? len : len + 4) : (len | 1);
};

// Stage records of `len` floats (count of them, contiguous in global memory, 16-byte
// aligned when len is a multiple of 4) into shared memory in RecLayout<len>. `len` is
// a compile-time constant, so the divisions below are multiplications.
template <int len, int T>
__device__ __forceinline__ void stage_records(float *dst, const float *src, int count) {
    constexpr int stride = RecLayout<len>::stride;
    if constexpr (RecLayout<len>::V4) {
        constexpr int q4 = len / 4;
        const int n4 = count * q4;
        for (int q = threadIdx.x; q < n4; q += T) {
            const int r = q / q4;
            cp_async16(dst + r * stride + 4 * (q - r * q4), src + 4 * q);
        }
    } else {
        const int total = count * len;
        for (int f = threadIdx.x; f < total; f += T) {
            const int r = f / len;
            cp_async4(dst + r * stride + (f - r * len), src + f);
        }
    }
}

// col[c] += sum_k Y[k] sh[3 k + c] over the nk coefficients of a record staged in
// RecLayout<3 nk>.
template <int nk>
__device__ __forceinline__ void sh_accumulate(const float *shp, const float *Y, float *col) {
    constexpr int len = 3 * nk;
    if constexpr (RecLayout<len>::V4) {
#pragma unroll
        for (int q = 0; q < len / 4; ++q) {
            const float4 x = *reinterpret_cast<const float4 *>(shp + 4 * q);
            const float e[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) col[(4 * q + t) % 3] = fmaf(Y[(4 * q + t) / 3], e[t], col[(4 * q + t) % 3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < nk; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) col[c] = fmaf(Y[k], shp[k * 3 + c], col[c]);
    }
}

__device__ __forceinline__ int clamp_pix(float v, int n) {
    v = fminf(fmaxf(v, -2.0f), (float)n + 2.0f);
    return (int)v;
}

// One item (view vw, triangle i) of the forward: geometry and culling, rectangle,
// record, depth key, its entry `lslot` of the visible-item list, and the binning's tile
// counts. Returns the item's tile count.
template <int DEG, int WIN, bool ZP>
__device__ __forceinline__ uint32_t preprocess_item(const PreArgs &a, const ViewDev &V, int vw, int64_t i,
                                                    uint32_t lslot, const float (&v)[9], const float *shp,
                                                    const float (&cen)[3], float o, float sig, float fshrink_pow,
                                                    float lgt, uint32_t (*s_hist)[256]) {
    constexpr int nk = (DEG + 1) * (DEG + 1);
    const int64_t m = (int64_t)vw * a.n + i;
    Geom g;
    int cull = item_geometry(v, V, g);
    uint32_t nt = 0;
    ushort4 rect = make_ushort4(0, 0, 0, 0);
    Rec rec;
    float fshrink = fshrink_pow;
    if (WIN == WIN_SIGMOID && !a.solid && cull == CULL_NONE)
        fshrink = o > ALPHA_MIN ? 1.0f - sig * lgt / g.r : 0.0f;   // > 1: support beyond the triangle
    if (cull == CULL_NONE && fshrink > 0.0f) {
        // shrunk triangle: S + f (Q_k - S), Q_0 = 0
        const float wx0 = g.S.x - fshrink * g.S.x, wy0 = g.S.y - fshrink * g.S.y;
        const float wx1 = fmaf(fshrink, g.Q1.x - g.S.x, g.S.x), wy1 = fmaf(fshrink, g.Q1.y - g.S.y, g.S.y);
        const float wx2 = fmaf(fshrink, g.Q2.x - g.S.x, g.S.x), wy2 = fmaf(fshrink, g.Q2.y - g.S.y, g.S.y);
        const float xmin = g.u0.hi + fminf(wx0, fminf(wx1, wx2)) - RECT_PAD;
        const float xmax = g.u0.hi + fmaxf(wx0, fmaxf(wx1, wx2)) + RECT_PAD;
        const float ymin = g.v0.hi + fminf(wy0, fminf(wy1, wy2)) - RECT_PAD;
        const float ymax = g.v0.hi + fmaxf(wy0, fmaxf(wy1, wy2)) + RECT_PAD;
        // pixels whose centres x + 0.5 lie in [min, max]
        int px0 = max(clamp_pix(ceilf(fminf(fmaxf(xmin, -2.f), V.W + 2.f) - 0.5f), V.W), 0);
        int px1 = min(clamp_pix(floorf(fminf(fmaxf(xmax, -2.f), V.W + 2.f) - 0.5f), V.W), V.W - 1);
        int py0 = max(clamp_pix(ceilf(fminf(fmaxf(ymin, -2.f), V.H + 2.f) - 0.5f), V.H), 0);
        int py1 = min(clamp_pix(floorf(fminf(fmaxf(ymax, -2.f), V.H + 2.f) - 0.5f), V.H), V.H - 1);
        if (px0 <= px1 && py0 <= py1) {
            rect = make_ushort4(px0, py0, px1, py1);
            nt = (uint32_t)(px1 / TILE - px0 / TILE + 1) * (uint32_t)(py1 / TILE - py0 / TILE + 1);
        }
    }
    uint32_t key = 0xffffffffu;   // invisible items sort after every depth
    if (nt > 0) {
        // incenter s = q0 + S in double-float (s_hi + s_lo)
        ff sx = two_sum(g.u0.hi, g.S.x);
        ff sy = two_sum(g.v0.hi, g.S.y);
        const float slx = sx.lo + g.u0.lo, sly = sy.lo + g.v0.lo;
        // colour
        float w0 = cen[0] - V.campos[0], w1 = cen[1] - V.campos[1], w2 = cen[2] - V.campos[2];
        float inv = rsqrtf(fmaf(w0, w0, fmaf(w1, w1, w2 * w2)));
        float Y[16];
        sh_basis(DEG, w0 * inv, w1 * inv, w2 * inv, Y);
        float col[3] = {0.5f, 0.5f, 0.5f};
        sh_accumulate<nk>(shp, Y, col);
#pragma unroll
        for (int c = 0; c < 3; ++c) col[c] = fmaxf(col[c], 0.0f);
        rec.a = make_float4(sx.hi, sy.hi, g.A[0], g.B[0]);
        rec.b = make_float4(slx, g.A[1], g.B[1], sly);
        rec.c = make_float4(g.A[2], g.B[2], 0.0f, a.solid ? 1.0f : o);
        rec.d = make_float4(WIN == WIN_SIGMOID ? g.r / sig : sig, col[0], col[1], col[2]);
        key = __float_as_uint(g.depth);
        if (ZP) {
            // inverse depth along the ray through p: (n . d) / (n . x0), n the plane
            // normal (x1 - x0) x (x2 - x0), d = ((p.x - cx) / fx, (p.y - cy) / fy, 1)
            float e[2][3];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float dx = v[3 * q + 3] - v[0], dy = v[3 * q + 4] - v[1], dz = v[3 * q + 5] - v[2];
#pragma unroll
                for (int r = 0; r < 3; ++r) e[q][r] = fmaf(V.R[3 * r], dx, fmaf(V.R[3 * r + 1], dy, V.R[3 * r + 2] * dz));
            }
            const float nx = e[0][1] * e[1][2] - e[0][2] * e[1][1];
            const float ny = e[0][2] * e[1][0] - e[0][0] * e[1][2];
            const float nz = e[0][0] * e[1][1] - e[0][1] * e[1][0];
            const float D = fmaf(nx, g.xc[0].x, fmaf(ny, g.xc[0].y, nz * g.xc[0].z));
            a.zplane[m] = D != 0.0f ? make_float4(nx / (V.fx * D), ny / (V.fy * D), nz / D, 0.0f)
                                    : make_float4(0.0f, 0.0f, 1.0f / g.depth, 0.0f);
        }
    }
    // records and rectangles are read only through the tile lists: an item that
    // touches no tile skips them (most items of a many-view batch are off screen)
    if (nt > 0) {
        a.recs[m] = rec;
        a.rects[m] = rect;
    }
    if (!a.vmask) {
        a.ntiles[m] = nt;
        a.dkeys[m] = key;
    }
    if (a.vislist && lslot < a.vis_cap) {
        // this candidate's list entry (a hole when the item touches no tile)
        a.vislist[lslot] = nt ? make_uint4((uint32_t)m, key, (uint32_t)rect.x | ((uint32_t)rect.y << 16),
                                           (uint32_t)rect.z | ((uint32_t)rect.w << 16))
                              : make_uint4(VIS_HOLE, 0u, 0u, 0u);
    }
    if (a.tile_count && nt) {
        // per-tile pair counts of the binning (fire-and-forget reductions)
        const uint32_t tx0 = rect.x / TILE, tx1 = rect.z / TILE, ty0 = rect.y / TILE, ty1 = rect.w / TILE;
        for (uint32_t ty = ty0; ty <= ty1; ++ty) {
            uint32_t *row = a.tile_count + V.tile_base + ty * (uint32_t)V.tiles_x;
            for (uint32_t tx = tx0; tx <= tx1; ++tx) atomicAdd(row + tx, 1u);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
        if (a.depth_hist) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
    return nt;
}

// Position of the j-th (from 0) set bit of m (which has more than j).
__device__ __forceinline__ int nth_set_bit(uint64_t m, int j) {
    int pos = 0;
#pragma unroll
    for (int w = 32; w > 0; w >>= 1) {
        const int c = __popcll(m & ((1ull << w) - 1ull));
        if (j >= c) {
            j -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// ZP: also write the items' inverse-depth planes (per-pixel sort). MULTI: several views,
// whose candidate items each warp deals out to its lanes.
template <int DEG, int WIN, bool ZP, bool MULTI>
__global__ void __launch_bounds__(PRE_THREADS, 6)
preprocess_fwd_kernel(PreArgs a) {
    __shared__ __align__(16) float s_v[PRE_THREADS * 9];
    __shared__ __align__(16) float s_sh[PRE_THREADS * 52];
    __shared__ uint32_t s_nvis;
    // several views: per warp, each lane's candidate views and its first item; per
    // triangle, its view mask and (o, sigma, shrink factor, sigmoid log term)
    __shared__ uint64_t s_wvis[MULTI ? PRE_THREADS / 32 : 1][32];
    __shared__ uint32_t s_wofs[MULTI ? PRE_THREADS / 32 : 1][33];
    __shared__ uint64_t s_vm[MULTI ? PRE_THREADS : 1];
    __shared__ float4 s_tri[MULTI ? PRE_THREADS : 1];
    // dynamic: per view, the frustum test's side-plane offsets (left, right, top,
    // bottom) and the reciprocal lengths of the planes' normals, the view table, and
    // (depth_hist only) the 4 digit histograms of the depth keys
    extern __shared__ float4 s_dyn[];
    float4 *s_pofs = s_dyn, *s_pinv = s_dyn + a.nviews;
    ViewDev *s_view = reinterpret_cast<ViewDev *>(s_dyn + 2 * a.nviews);
    uint32_t (*s_hist)[256] = reinterpret_cast<uint32_t (*)[256]>(s_view + a.nviews);

    const int tid = threadIdx.x;
    if (a.depth_hist)
        for (int k = tid; k < 4 * 256; k += PRE_THREADS) (&s_hist[0][0])[k] = 0u;
    if (tid == 0) s_nvis = 0;
    for (int k = tid; k < a.nviews * (int)(sizeof(ViewDev) / 4); k += PRE_THREADS)
        reinterpret_cast<uint32_t *>(s_view)[k] = reinterpret_cast<const uint32_t *>(a.views)[k];
    for (int k = tid; k < a.nviews; k += PRE_THREADS) {
        const ViewDev &V = a.views[k];
        const float ul = V.cx + FRUSTUM_PAD, ur = (float)V.W + FRUSTUM_PAD - V.cx;
        const float vt = V.cy + FRUSTUM_PAD, vb = (float)V.H + FRUSTUM_PAD - V.cy;
        s_pofs[k] = make_float4(ul, ur, vt, vb);
        s_pinv[k] = make_float4(rsqrtf(fmaf(V.fx, V.fx, ul * ul)), rsqrtf(fmaf(V.fx, V.fx, ur * ur)),
                                rsqrtf(fmaf(V.fy, V.fy, vt * vt)), rsqrtf(fmaf(V.fy, V.fy, vb * vb)));
    }
    const int64_t i0 = (int64_t)blockIdx.x * PRE_THREADS;
    const int cnt = (int)(a.n - i0 < PRE_THREADS ? a.n - i0 : PRE_THREADS);
    constexpr int nk = (DEG + 1) * (DEG + 1);
    stage_floats<PRE_THREADS>(s_v, a.verts + i0 * 9, cnt * 9);
    stage_records<nk * 3, PRE_THREADS>(s_sh, a.sh + i0 * nk * 3, cnt);
    const int64_t i = i0 + tid;
    const bool alive = tid < cnt;
    const float o = alive ? __ldg(a.opacity + i) : 1.0f;
    const float sig = alive ? __ldg(a.sigma + i) : 1.0f;
    cp_async_wait_all();
    __syncthreads();

    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = s_v[tid * 9 + k];
    const float *shp = s_sh + tid * RecLayout<nk * 3>::stride;
    // shrink factor of the tight rectangle (Supp. "Tile assignment")
    // (solid records: the whole triangle, whatever its opacity; for the sigmoid window
    // the factor depends on the inradius and is set per view below)
    const float fshrink_pow = a.solid ? 1.0f : (WIN == WIN_POWER ? 1.0f - powf(ALPHA_MIN / o, 1.0f / sig) : 0.0f);
    // sigmoid window: o I >= tau where kappa ratio >= ln(tau / (o - tau))
    const float lgt = (WIN == WIN_SIGMOID && o > ALPHA_MIN) ? logf(ALPHA_MIN / (o - ALPHA_MIN)) : 0.0f;
    float cen[3];
    centroid(v, cen);

    // views the triangle may touch: its bounding sphere (centroid, largest vertex
    // distance) against the near plane and the four side planes of each view's frustum
    // widened by FRUSTUM_PAD pixels. A sphere wholly outside a side plane means that
    // either a vertex is nearer than Z_NEAR (the exact test culls the item) or every
    // vertex projects beyond the image by more than FP32 error (no tile); wholly in
    // front of the near plane means all vertices are. Either way the exact path would
    // emit nothing, so only the views left are visited, which most triangles of a
    // many-view batch are not in. (Not for the sigmoid window, whose support reaches
    // beyond the triangle.)
    uint64_t vis = 0;
    if (alive) {
        float rad2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float dx = v[3 * k] - cen[0], dy = v[3 * k + 1] - cen[1], dz = v[3 * k + 2] - cen[2];
            rad2 = fmaxf(rad2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        const float rad = fmaf(sqrtf(rad2), 1.0001f, 1e-6f);
        const bool test = (WIN == WIN_POWER || a.solid) && rad < 1e30f;
        for (int vw = 0; vw < a.nviews; ++vw) {
            const ViewDev &V = s_view[vw];
            bool out = false;
            if (test && V.fx > 0.0f && V.fy > 0.0f) {
                const float xc = fmaf(V.R[0], cen[0], fmaf(V.R[1], cen[1], fmaf(V.R[2], cen[2], V.t[0])));
                const float yc = fmaf(V.R[3], cen[0], fmaf(V.R[4], cen[1], fmaf(V.R[5], cen[2], V.t[1])));
                const float zc = fmaf(V.R[6], cen[0], fmaf(V.R[7], cen[1], fmaf(V.R[8], cen[2], V.t[2])));
                const float4 po = s_pofs[vw], pi = s_pinv[vw];
                // (the near test keeps half the plane distance as slack for the FP32
                // vertex depths of the exact test)
                out = zc + rad < 0.5f * Z_NEAR || fmaf(V.fx, xc, po.x * zc) * pi.x < -rad ||
                      fmaf(-V.fx, xc, po.y * zc) * pi.y < -rad || fmaf(V.fy, yc, po.z * zc) * pi.z < -rad ||
                      fmaf(-V.fy, yc, po.w * zc) * pi.w < -rad;
            }
            if (!out) {
                vis |= 1ull << vw;
                continue;
            }
            const int64_t m = (int64_t)vw * a.n + i;
            if (!a.vmask) {
                a.ntiles[m] = 0u;
                a.dkeys[m] = 0xffffffffu;
            }
            if (a.depth_hist) {
#pragma unroll
                for (int p = 0; p < 4; ++p) atomicAdd(&s_hist[p][255], 1u);
            }
        }
    }

    // the warp's candidate items (this thread's first at woff of wtot) and their list
    // slots from wbase: one reservation per warp
    uint32_t woff, wtot, wbase = 0;
    {
        const uint32_t c = (uint32_t)__popcll(vis);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o) incl += y;
        }
        wtot = __shfl_sync(0xffffffffu, incl, 31);
        woff = incl - c;
        if (a.vislist) {
            if ((tid & 31) == 0 && wtot) wbase = atomicAdd(&a.ctl->vis_count, wtot);
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
        }
    }
    uint32_t lslot = wbase + woff;
    uint32_t nvis = 0;
    uint64_t vm = 0;    // views in which the triangle touches a tile
    if (!MULTI) {
#pragma unroll 1
        for (; vis; vis &= vis - 1) {
            const int vw = __ffsll((long long)vis) - 1;
            const uint32_t nt =
                preprocess_item<DEG, WIN, ZP>(a, s_view[vw], vw, i, lslot++, v, shp, cen, o, sig, fshrink_pow, lgt, s_hist);
            nvis += nt ? 1u : 0u;
            vm |= nt ? 1ull << vw : 0ull;
        }
    } else {
        // the warp's candidate items are dealt out to its lanes in rounds (a lane per
        // triangle looping over its views would leave about half of them idle): item c
        // of the warp belongs to the last lane whose first item is <= c
        const int lane = tid & 31, w = tid >> 5;
        s_wvis[w][lane] = vis;
        s_wofs[w][lane] = woff;
        s_vm[tid] = 0ull;
        s_tri[tid] = make_float4(o, sig, fshrink_pow, lgt);
        __syncwarp();
        for (uint32_t c = (uint32_t)lane; c < wtot; c += 32u) {
            int lo = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
                if (s_wofs[w][lo + st] <= c) lo += st;
            const int t = 32 * w + lo;       // the owner's thread
            const int vw = nth_set_bit(s_wvis[w][lo], (int)(c - s_wofs[w][lo]));
            float vt[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) vt[q] = s_v[t * 9 + q];
            float ct[3];
            centroid(vt, ct);
            const float4 tp = s_tri[t];
            const uint32_t nt = preprocess_item<DEG, WIN, ZP>(a, s_view[vw], vw, i0 + t, wbase + c, vt,
                                                              s_sh + t * RecLayout<nk * 3>::stride, ct, tp.x, tp.y, tp.z,
                                                              tp.w, s_hist);
            nvis += nt ? 1u : 0u;
            if (nt) atomicOr(reinterpret_cast<unsigned long long *>(&s_vm[t]), 1ull << vw);
        }
        __syncwarp();
        vm = s_vm[tid];
    }
    if (a.vmask && alive) a.vmask[i] = vm;
    const uint32_t wv = __reduce_add_sync(0xffffffffu, nvis);
    if ((tid & 31) == 0 && wv) atomicAdd(&s_nvis, wv);
    __syncthreads();
    if (a.depth_hist) {
        for (int k = tid; k < 4 * 256; k += PRE_THREADS) {
            const uint32_t c = (&s_hist[0][0])[k];
            if (c) atomicAdd(&(&a.ctl->depth_hist[0][0])[k], c);
        }
    }
    if (tid == 0 && s_nvis) atomicAdd(&a.ctl->n_visible, s_nvis);
}

template <int DEG, int WIN, bool MULTI>
__global__ void __launch_bounds__(PRE_BWD_THREADS, MULTI ? 6 : 8)
preprocess_bwd_kernel(PreBwdArgs a) {
    __shared__ __align__(16) float s_v[PRE_BWD_THREADS * 9];
    __shared__ __align__(16) float s_sh[PRE_BWD_THREADS * 52];
    __shared__ __align__(16) float s_gsh[PRE_BWD_THREADS * 52];
    extern __shared__ ViewDev s_view[];   // nviews entries
    const int tid = threadIdx.x;
    for (int k = tid; k < a.nviews * (int)(sizeof(ViewDev) / 4); k += PRE_BWD_THREADS)
        reinterpret_cast<uint32_t *>(s_view)[k] = reinterpret_cast<const uint32_t *>(a.views)[k];
    const int64_t i0 = (int64_t)blockIdx.x * PRE_BWD_THREADS;
    const int cnt = (int)(a.n - i0 < PRE_BWD_THREADS ? a.n - i0 : PRE_BWD_THREADS);
    constexpr int nk = (DEG + 1) * (DEG + 1);
    stage_floats<PRE_BWD_THREADS>(s_v, a.verts + i0 * 9, cnt * 9);
    stage_records<nk * 3, PRE_BWD_THREADS>(s_sh, a.sh + i0 * nk * 3, cnt);
    const int64_t i = i0 + tid;
    const bool alive = tid < cnt;
    // one view: its tile count and gradient record load while the staging completes
    uint32_t nt1 = 0;
    float4 R0 = make_float4(0.f, 0.f, 0.f, 0.f), R1 = R0, R2 = R0, R3 = R0;
    if (!MULTI && alive) {
        nt1 = a.vmask ? (uint32_t)(__ldg(a.vmask + i) & 1ull) : __ldg(a.ntiles + i);
        const float4 *gp = reinterpret_cast<const float4 *>(a.grad2d + i * GRAD_FIELDS);
        R0 = __ldg(gp);
        R1 = __ldg(gp + 1);
        R2 = __ldg(gp + 2);
        R3 = __ldg(gp + 3);
    }
    cp_async_wait_all();
    __syncthreads();
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = s_v[tid * 9 + k];
    constexpr int sstride = RecLayout<nk * 3>::stride;
    float *shp = s_sh + tid * sstride;
    float cen[3];
    centroid(v, cen);
    float gv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) gv[k] = 0.f;
    float go = 0.f, gsig = 0.f;
    float *gsh = s_gsh + tid * sstride;
    if constexpr (RecLayout<nk * 3>::V4) {
#pragma unroll
        for (int q = 0; q < nk * 3 / 4; ++q) reinterpret_cast<float4 *>(gsh)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int k = 0; k < nk * 3; ++k) gsh[k] = 0.f;
    }

    // views in which the triangle was binned: its view mask, or with several views the
    // tile counts of all views loaded back to back (one latency) into a bit mask; then
    // only those views are visited
    uint64_t vis = 0;
    if (!MULTI) {
        vis = nt1 != 0u ? 1ull : 0ull;
    } else if (alive && a.vmask) {
        vis = __ldg(a.vmask + i);
    } else if (alive) {
        for (int v0 = 0; v0 < a.nviews; v0 += 8) {
            uint32_t nt[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) nt[q] = v0 + q < a.nviews ? __ldg(a.ntiles + (int64_t)(v0 + q) * a.n + i) : 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) vis |= (uint64_t)(nt[q] != 0u) << (v0 + q);
        }
    }
#pragma unroll 1
    for (; vis; vis &= vis - 1) {
        const int vw = __ffsll((long long)vis) - 1;
        const int64_t m = (int64_t)vw * a.n + i;
        const float4 *gp = reinterpret_cast<const float4 *>(a.grad2d + m * GRAD_FIELDS);
        const float4 G0 = MULTI ? gp[0] : R0, G1 = MULTI ? gp[1] : R1, G2 = MULTI ? gp[2] : R2,
                     G3 = MULTI ? gp[3] : R3;
        const ViewDev &V = s_view[vw];
        Geom g;
        item_geometry<false>(v, V, g);
        go += G2.x;
        // sigmoid window: field 9 holds dL/dkappa, kappa = r / sigma
        const float sig_i = WIN == WIN_SIGMOID ? __ldg(a.sigma + i) : 0.0f;
        if constexpr (WIN == WIN_SIGMOID) gsig -= G2.y * g.r / (sig_i * sig_i);
        else gsig += G2.y;
        // s = q0 + S
        const float gsx = G0.x, gsy = G0.y;
        const float gA[3] = {G0.z, G1.x, G1.z}, gB[3] = {G0.w, G1.y, G1.w};
        float gq0x = gsx, gq0y = gsy;
        float gQ1x = 0.f, gQ1y = 0.f, gQ2x = 0.f, gQ2y = 0.f;
        float gell[3] = {0.f, 0.f, 0.f};
        float gP = 0.f, gA2 = 0.f;
        const float P = g.perim, iP = rcp_approx(P);
        // S = (ell1 Q1 + ell2 Q2) / P
        gQ1x += gsx * g.ell[1] * iP; gQ1y += gsy * g.ell[1] * iP;
        gQ2x += gsx * g.ell[2] * iP; gQ2y += gsy * g.ell[2] * iP;
        gell[1] += (gsx * g.Q1.x + gsy * g.Q1.y) * iP;
        gell[2] += (gsx * g.Q2.x + gsy * g.Q2.y) * iP;
        gP -= (gsx * g.S.x + gsy * g.S.y) * iP;
        // A_i = -E_i.y k_i, B_i = E_i.x k_i, k_i = P / (ell_i area2)
        const float Ex[3] = {g.Q2.x - g.Q1.x, -g.Q2.x, g.Q1.x};
        const float Ey[3] = {g.Q2.y - g.Q1.y, -g.Q2.y, g.Q1.y};
        float gEx[3], gEy[3];
        const float ia2 = rcp_approx(g.area2);
        if constexpr (WIN == WIN_SIGMOID) {
            // r = |area2| / P
            const float gr_in = G2.y / sig_i;
            gA2 += gr_in * (g.area2 >= 0.0f ? iP : -iP);
            gP -= gr_in * g.r * iP;
        }
        float iell[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) iell[k] = rcp_approx(g.ell[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float kk = P * iell[k] * ia2;
            const float gk = -gA[k] * Ey[k] + gB[k] * Ex[k];
            gEx[k] = gB[k] * kk;
            gEy[k] = -gA[k] * kk;
            gP += gk * kk * iP;
            gell[k] -= gk * kk * iell[k];
            gA2 -= gk * kk * ia2;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float gl = (gell[k] + gP) * iell[k];
            gEx[k] += gl * Ex[k];
            gEy[k] += gl * Ey[k];
        }
        // E0 = Q2 - Q1, E1 = -Q2, E2 = Q1
        gQ2x += gEx[0] - gEx[1]; gQ2y += gEy[0] - gEy[1];
        gQ1x += gEx[2] - gEx[0]; gQ1y += gEy[2] - gEy[0];
        // area2 = Q1.x Q2.y - Q1.y Q2.x
        gQ1x += gA2 * g.Q2.y; gQ1y -= gA2 * g.Q2.x;
        gQ2x -= gA2 * g.Q1.y; gQ2y += gA2 * g.Q1.x;
        // Q_k = q_k - q_0
        gq0x -= gQ1x + gQ2x; gq0y -= gQ1y + gQ2y;
        const float gqx[3] = {gq0x, gQ1x, gQ2x}, gqy[3] = {gq0y, gQ1y, gQ2y};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float iz = rcp_approx(g.xc[k].z);
            const float gx = gqx[k] * V.fx * iz;
            const float gy = gqy[k] * V.fy * iz;
            const float gz = -(gx * g.xc[k].x + gy * g.xc[k].y) * iz;
            // x_k = R v_k + t
            gv[3 * k + 0] += V.R[0] * gx + V.R[3] * gy + V.R[6] * gz;
            gv[3 * k + 1] += V.R[1] * gx + V.R[4] * gy + V.R[7] * gz;
            gv[3 * k + 2] += V.R[2] * gx + V.R[5] * gy + V.R[8] * gz;
        }
        // colour: rgb = max(0, 0.5 + sum Y_k sh_k)
        float w0 = cen[0] - V.campos[0], w1 = cen[1] - V.campos[1], w2 = cen[2] - V.campos[2];
        const float inv = rsqrtf(fmaf(w0, w0, fmaf(w1, w1, w2 * w2)));
        const float dx = w0 * inv, dy = w1 * inv, dz = w2 * inv;
        float Y[16];
        sh_basis(DEG, dx, dy, dz, Y);
        const float grgb[3] = {G2.z, G2.w, G3.x};
        float raw[3] = {0.5f, 0.5f, 0.5f};
        sh_accumulate<nk>(shp, Y, raw);
        float graw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) graw[c] = raw[c] > 0.0f ? grgb[c] : 0.0f;
        float gY[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) gY[k] = 0.f;
        if constexpr (RecLayout<nk * 3>::V4) {
#pragma unroll
            for (int q = 0; q < nk * 3 / 4; ++q) {
                const float4 x = reinterpret_cast<const float4 *>(shp)[q];
                float4 &gq = reinterpret_cast<float4 *>(gsh)[q];
                float4 gg = gq;
                const float e[4] = {x.x, x.y, x.z, x.w};
                float ge[4] = {gg.x, gg.y, gg.z, gg.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int k = (4 * q + t) / 3, c = (4 * q + t) % 3;
                    ge[t] = fmaf(graw[c], Y[k], ge[t]);
                    gY[k] = fmaf(graw[c], e[t], gY[k]);
                }
                gq = make_float4(ge[0], ge[1], ge[2], ge[3]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < nk; ++k) {
                gsh[k * 3 + 0] += graw[0] * Y[k];
                gsh[k * 3 + 1] += graw[1] * Y[k];
                gsh[k * 3 + 2] += graw[2] * Y[k];
                gY[k] = graw[0] * shp[k * 3] + graw[1] * shp[k * 3 + 1] + graw[2] * shp[k * 3 + 2];
            }
        }
        if (DEG > 0) {
            const float3 gd = sh_basis_vjp(DEG, dx, dy, dz, gY);
            const float dd = gd.x * dx + gd.y * dy + gd.z * dz;
            const float gwx = (gd.x - dx * dd) * inv, gwy = (gd.y - dy * dd) * inv, gwz = (gd.z - dz * dd) * inv;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gv[3 * k + 0] += gwx * (1.0f / 3.0f);
                gv[3 * k + 1] += gwy * (1.0f / 3.0f);
                gv[3 * k + 2] += gwz * (1.0f / 3.0f);
            }
        }
    }
    __syncthreads();
    // stage and write (coalesced): vertices, then SH
    if (alive) {
#pragma unroll
        for (int k = 0; k < 9; ++k) s_v[tid * 9 + k] = gv[k];
        if (a.dopacity) a.dopacity[i] = a.accumulate ? a.dopacity[i] + go : go;
        if (a.dsigma) a.dsigma[i] = a.accumulate ? a.dsigma[i] + gsig : gsig;
    }
    __syncthreads();
    if (a.dverts) {
        float *dst = a.dverts + i0 * 9;
        for (int k = tid; k < cnt * 9; k += PRE_BWD_THREADS) dst[k] = a.accumulate ? dst[k] + s_v[k] : s_v[k];
    }
    if (a.dsh) {
        constexpr int len = nk * 3;
        float *dst = a.dsh + i0 * len;
        for (int f = tid; f < cnt * len; f += PRE_BWD_THREADS) {
            const int r = f / len;
            const float g = s_gsh[r * sstride + (f - r * len)];
            dst[f] = a.accumulate ? dst[f] + g : g;
        }
    }
}

template <int NV>
struct InitArgs {
    ViewDev views[NV];
    const ViewDev *pinned;   // if set: the table is read from here instead
    int nviews, tiles;
    ViewDev *views_d;
    uint32_t *ctl;
    uint32_t *tile_count;
};

template <int NV>
__global__ void __launch_bounds__(256) step_init_kernel(const __grid_constant__ InitArgs<NV> a) {
    constexpr int vw = (int)(sizeof(ViewDev) / 4), cw = (int)(sizeof(Ctl) / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.pinned ? a.pinned : a.views);
    const int n = max(max(a.nviews * vw, cw), a.tiles);
    for (int k = blockIdx.x * 256 + threadIdx.x; k < n; k += gridDim.x * 256) {
        if (k < a.nviews * vw) reinterpret_cast<uint32_t *>(a.views_d)[k] = src[k];
        if (k < cw) a.ctl[k] = 0u;
        if (k < a.tiles) a.tile_count[k] = 0u;
    }
}

template <int NV>
static void step_init(const ViewDev *views, const ViewDev *pinned, int nviews, ViewDev *views_d, Ctl *ctl,
                      uint32_t *tile_count, int tiles, cudaStream_t st) {
    InitArgs<NV> a;
    if (!pinned)
        for (int v = 0; v < nviews; ++v) a.views[v] = views[v];
    a.pinned = pinned;
    a.nviews = nviews;
    a.tiles = tiles;
    a.views_d = views_d;
    a.ctl = reinterpret_cast<uint32_t *>(ctl);
    a.tile_count = tile_count;
    const int words = max(max(nviews * (int)(sizeof(ViewDev) / 4), (int)(sizeof(Ctl) / 4)), tiles);
    int g = (words + 255) / 256;
    if (g > 304) g = 304;
    step_init_kernel<NV><<<g, 256, 0, st>>>(a);
}

void launch_step_init(const ViewDev *views, const ViewDev *pinned, int nviews, ViewDev *views_d, Ctl *ctl,
                      uint32_t *tile_count, int tiles, cudaStream_t st) {
    if (pinned || nviews <= 4) step_init<4>(views, pinned, nviews, views_d, ctl, tile_count, tiles, st);
    else step_init<MAX_VIEWS>(views, pinned, nviews, views_d, ctl, tile_count, tiles, st);
}

template <bool ZP, bool MULTI>
static void launch_fwd_zp(const PreArgs &a, int grid, size_t smem, cudaStream_t st) {
    const bool sg = a.window == WIN_SIGMOID;
    switch (a.sh_degree) {
        case 0: sg ? preprocess_fwd_kernel<0, 1, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a)
                   : preprocess_fwd_kernel<0, 0, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a); break;
        case 1: sg ? preprocess_fwd_kernel<1, 1, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a)
                   : preprocess_fwd_kernel<1, 0, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a); break;
        case 2: sg ? preprocess_fwd_kernel<2, 1, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a)
                   : preprocess_fwd_kernel<2, 0, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a); break;
        default: sg ? preprocess_fwd_kernel<3, 1, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a)
                    : preprocess_fwd_kernel<3, 0, ZP, MULTI><<<grid, PRE_THREADS, smem, st>>>(a); break;
    }
}

void launch_preprocess_fwd(const PreArgs &a, cudaStream_t st) {
    const int grid = (int)((a.n + PRE_THREADS - 1) / PRE_THREADS);
    if (grid <= 0) return;
    const size_t smem = (2 * sizeof(float4) + sizeof(ViewDev)) * a.nviews + (a.depth_hist ? 4 * 256 * 4 : 0);
    if (a.nviews > 1) {
        if (a.zplane) launch_fwd_zp<true, true>(a, grid, smem, st);
        else launch_fwd_zp<false, true>(a, grid, smem, st);
    } else {
        if (a.zplane) launch_fwd_zp<true, false>(a, grid, smem, st);
        else launch_fwd_zp<false, false>(a, grid, smem, st);
    }
}

template <bool MULTI>
static void launch_bwd_views(const PreBwdArgs &a, int grid, size_t smem, cudaStream_t st) {
    const bool sg = a.window == WIN_SIGMOID;
    switch (a.sh_degree) {
        case 0: sg ? preprocess_bwd_kernel<0, 1, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a)
                   : preprocess_bwd_kernel<0, 0, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a); break;
        case 1: sg ? preprocess_bwd_kernel<1, 1, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a)
                   : preprocess_bwd_kernel<1, 0, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a); break;
        case 2: sg ? preprocess_bwd_kernel<2, 1, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a)
                   : preprocess_bwd_kernel<2, 0, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a); break;
        default: sg ? preprocess_bwd_kernel<3, 1, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a)
                    : preprocess_bwd_kernel<3, 0, MULTI><<<grid, PRE_BWD_THREADS, smem, st>>>(a); break;
    }
}

void launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t st) {
    const int grid = (int)((a.n + PRE_BWD_THREADS - 1) / PRE_BWD_THREADS);
    if (grid <= 0) return;
    const size_t smem = sizeof(ViewDev) * a.nviews;
    if (a.nviews > 1) launch_bwd_views<true>(a, grid, smem, st);
    else launch_bwd_views<false>(a, grid, smem, st);
}

}  // namespace ts
