// Densification moves, the size regulariser and the pruning rule (declared in
// trisplat.h: tri_densify, tri_size_reg, tri_prune_fold, tri_prune_mask).
//
// Sec. 3.3 ("Densification"): a selected triangle is split by midpoint subdivision
// into four that tile it (combined area and region unchanged); one whose area is
// below tau_small is cloned instead, the clone translated within the triangle's
// plane by caller-drawn noise. Sec. 3.4: L_s = 2 / |(v1 - v0) x (v2 - v0)|.
//
// tri_densify is one kernel: each CTA takes 256 selected triangles in order (ticket),
// counts the triangles each appends (3 or 1), and finds its output offset with a
// single-pass scan (decoupled look-back), so the appended triangles follow the order
// of the selection list. Geometry is written per thread, SH records per warp.
#include "kernels.h"

namespace ts {

constexpr int DENS_THREADS = 256;
constexpr float DENS_EPS = 1e-30f;

__device__ __forceinline__ float3 f3(const float *p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 mul3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float norm3(float3 a) { return sqrtf(a.x * a.x + a.y * a.y + a.z * a.z); }
__device__ __forceinline__ void put3(float *p, float3 a) {
    p[0] = a.x;
    p[1] = a.y;
    p[2] = a.z;
}

__global__ void __launch_bounds__(DENS_THREADS) densify_kernel(DensifyArgs a) {
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_cta, s_base;
    const int tid = threadIdx.x;
    if (tid == 0) s_cta = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint32_t cta = s_cta;
    const int64_t j = (int64_t)cta * DENS_THREADS + tid;
    int64_t i = -1;
    if (j < a.k) {
        i = a.sel[j];
        if (i < 0 || i >= a.n) {
            atomicOr(a.err, ERR_INDEX);
            i = -1;
        }
    }
    float3 v0 = make_float3(0.f, 0.f, 0.f), v1 = v0, v2 = v0, c = v0;
    bool small = false;
    if (i >= 0) {
        const float *vp = a.verts + i * 9;
        v0 = f3(vp);
        v1 = f3(vp + 3);
        v2 = f3(vp + 6);
        c = cross3(sub3(v1, v0), sub3(v2, v0));
        small = 0.5f * norm3(c) < a.tau_small;
    }
    const uint32_t cnt = i < 0 ? 0u : (small ? 1u : 3u);
    uint32_t total;
    const uint32_t local = block_excl_scan(cnt, s_tmp, total);
    if (tid < 32) {
        const uint32_t b = warp_lookback_excl(a.lb_status, cta, total, a.err);
        if (tid == 0) s_base = b;
    }
    __syncthreads();
    const int64_t base = a.n + s_base;
    if (tid == 0 && (int64_t)(cta + 1) * DENS_THREADS >= a.k) *a.n_out = base + total;
    const int64_t pos = base + local;
    if (i >= 0) {
        auto copy_scalars = [&](int64_t dst) {
            a.opacity[dst] = a.opacity[i];
            a.sigma[dst] = a.sigma[i];
        };
        if (!small) {
            const float3 m01 = mul3(add3(v0, v1), 0.5f), m12 = mul3(add3(v1, v2), 0.5f), m02 = mul3(add3(v0, v2), 0.5f);
            float *vp = a.verts + i * 9;
            put3(vp + 3, m01);
            put3(vp + 6, m02);
            float *d = a.verts + pos * 9;
            put3(d, m01), put3(d + 3, v1), put3(d + 6, m12);
            put3(d + 9, m02), put3(d + 12, m12), put3(d + 15, v2);
            put3(d + 18, m01), put3(d + 21, m12), put3(d + 24, m02);
            for (int q = 0; q < 3; ++q) copy_scalars(pos + q);
        } else {
            const float nc = fmaxf(norm3(c), DENS_EPS);
            const float3 nrm = mul3(c, 1.0f / nc);
            const float3 e = sub3(v1, v0);
            const float3 e1 = mul3(e, 1.0f / fmaxf(norm3(e), DENS_EPS));
            const float3 e2 = cross3(nrm, e1);
            const float na = a.noise[2 * j], nb = a.noise[2 * j + 1];
            const float3 t = mul3(add3(mul3(e1, na), mul3(e2, nb)), a.noise_scale);
            // both copies take 1 - sqrt(1 - o) = o / (1 + sqrt(1 - o)) (no cancellation):
            // together they composite to o
            const float oi = a.opacity[i];
            a.opacity[i] = oi / (1.0f + sqrtf(fmaxf(1.0f - oi, 0.0f)));
            float *d = a.verts + pos * 9;
            put3(d, add3(v0, t)), put3(d + 3, add3(v1, t)), put3(d + 6, add3(v2, t));
            copy_scalars(pos);
        }
    }
    // SH records of the appended triangles, copied by the whole warp one selected
    // triangle at a time (32 consecutive floats per access instead of one record per
    // thread at a 4-byte stride)
    const int nsh = a.nk * 3, lane = tid & 31;
    for (int l = 0; l < 32; ++l) {
        const long long si = __shfl_sync(0xffffffffu, (long long)i, l);
        if (si < 0) continue;
        const long long dp = __shfl_sync(0xffffffffu, (long long)pos, l);
        const int ncp = __shfl_sync(0xffffffffu, (int)cnt, l);
        const float *src = a.sh + si * nsh;
        for (int q = lane; q < nsh; q += 32) {
            const float x = src[q];
            for (int k = 0; k < ncp; ++k) a.sh[(dp + k) * nsh + q] = x;
        }
    }
}

// L_s = weight * sum_i 2 / |c_i|, c_i = (v1 - v0) x (v2 - v0); dverts += dL_s/dverts.
// Blocks of 256 triangles pass through shared memory, so that global accesses are
// consecutive floats rather than 9-float records at a stride.
__global__ void __launch_bounds__(DENS_THREADS) size_reg_kernel(const float *__restrict__ verts, int64_t n, float weight,
                                                              float *loss, float *dverts) {
    __shared__ float s_part[DENS_THREADS / 32];
    __shared__ float s_v[DENS_THREADS * 9];
    __shared__ float s_d[DENS_THREADS * 9];
    const int tid = threadIdx.x;
    float acc = 0.f;
    for (int64_t b0 = (int64_t)blockIdx.x * DENS_THREADS; b0 < n; b0 += (int64_t)gridDim.x * DENS_THREADS) {
        const int cnt = (int)(n - b0 < DENS_THREADS ? n - b0 : DENS_THREADS);
        for (int k = tid; k < cnt * 9; k += DENS_THREADS) {
            s_v[k] = verts[b0 * 9 + k];
            if (dverts) s_d[k] = dverts[b0 * 9 + k];
        }
        __syncthreads();
        if (tid < cnt) {
            const float *vp = s_v + tid * 9;
            const float3 v0 = f3(vp), e1 = sub3(f3(vp + 3), v0), e2 = sub3(f3(vp + 6), v0);
            const float3 c = cross3(e1, e2);
            const float nc = norm3(c);
            if (nc >= 1e-12f) {
                const float inv = 1.0f / nc;
                acc += 2.0f * inv;
                if (dverts) {
                    const float3 g = mul3(c, -2.0f * weight * inv * inv * inv);   // dL/dc
                    const float3 d1 = cross3(e2, g), d2 = cross3(g, e1);
                    float *dp = s_d + tid * 9;
                    dp[0] -= d1.x + d2.x, dp[1] -= d1.y + d2.y, dp[2] -= d1.z + d2.z;
                    dp[3] += d1.x, dp[4] += d1.y, dp[5] += d1.z;
                    dp[6] += d2.x, dp[7] += d2.y, dp[8] += d2.z;
                }
            }
        }
        __syncthreads();
        if (dverts)
            for (int k = tid; k < cnt * 9; k += DENS_THREADS) dverts[b0 * 9 + k] = s_d[k];
        __syncthreads();
    }
    if (loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) s_part[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int k = 0; k < DENS_THREADS / 32; ++k) t += s_part[k];
            atomicAdd(loss, weight * t);
        }
    }
}

// Sec. 3.3 ("Pruning"): fold the per-(view, triangle) statistics of one forward into
// running per-triangle state, best = largest blending weight T o seen, views = number
// of views in which the triangle was composited at >= min_pixels pixels. One thread
// per triangle reads its column of the [nviews][n] arrays (coalesced across threads).
__global__ void __launch_bounds__(DENS_THREADS) prune_fold_kernel(const float *__restrict__ max_weight,
                                                                const int32_t *__restrict__ n_pixels, int nviews,
                                                                int64_t n, int min_pixels, float *best,
                                                                int32_t *views) {
    for (int64_t i = (int64_t)blockIdx.x * DENS_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DENS_THREADS) {
        float b = best[i];
        int32_t c = views[i];
        for (int v = 0; v < nviews; ++v) {
            b = fmaxf(b, __ldg(max_weight + (int64_t)v * n + i));
            c += __ldg(n_pixels + (int64_t)v * n + i) >= min_pixels ? 1 : 0;
        }
        best[i] = b;
        views[i] = c;
    }
}

// keep = best >= tau_prune and views >= min_views (Sec. 3.3: the blending-weight
// threshold, and "rendered at least twice with more than one pixel").
__global__ void __launch_bounds__(DENS_THREADS) prune_mask_kernel(const float *__restrict__ best,
                                                                const int32_t *__restrict__ views, int64_t n,
                                                                float tau_prune, int min_views, uint8_t *keep) {
    for (int64_t i = (int64_t)blockIdx.x * DENS_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * DENS_THREADS)
        keep[i] = (__ldg(best + i) >= tau_prune && __ldg(views + i) >= min_views) ? 1 : 0;
}

void launch_prune_fold(const float *max_weight, const int32_t *n_pixels, int nviews, int64_t n, int min_pixels,
                       float *best, int32_t *views, int sms, cudaStream_t st) {
    int64_t g = (n + DENS_THREADS - 1) / DENS_THREADS;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    if (g > 0) prune_fold_kernel<<<(unsigned)g, DENS_THREADS, 0, st>>>(max_weight, n_pixels, nviews, n, min_pixels, best,
                                                                     views);
}

void launch_prune_mask(const float *best, const int32_t *views, int64_t n, float tau_prune, int min_views,
                       uint8_t *keep, int sms, cudaStream_t st) {
    int64_t g = (n + DENS_THREADS - 1) / DENS_THREADS;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    if (g > 0) prune_mask_kernel<<<(unsigned)g, DENS_THREADS, 0, st>>>(best, views, n, tau_prune, min_views, keep);
}

void launch_densify(const DensifyArgs &a, cudaStream_t st) {
    const int64_t g = (a.k + DENS_THREADS - 1) / DENS_THREADS;
    if (g > 0) densify_kernel<<<(unsigned)g, DENS_THREADS, 0, st>>>(a);
}

void launch_size_reg(const float *verts, int64_t n, float weight, float *loss, float *dverts, int sms,
                     cudaStream_t st) {
    int64_t g = (n + DENS_THREADS - 1) / DENS_THREADS;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    if (g > 0) size_reg_kernel<<<(unsigned)g, DENS_THREADS, 0, st>>>(verts, n, weight, loss, dverts);
}

}  // namespace ts
