// Per-item geometry of the triangle-splat renderer: projection, normalised edge
// lines, incenter, tight rectangle and SH colour (Sec. 3.1; Supp. "Tile assignment").
//
// Precision: vertex 0 is transformed and projected in double-float arithmetic
// (error-free sums and products on the FP32 pipe), vertices 1 and 2 relative to it.
// The pixel-grid position of a triangle is then exact to ~1e-9 px instead of the
// ~1e-4 px a plain FP32 transform of world coordinates would give, which matters
// because the window is steep near the edges when sigma < 1.
#pragma once

#include "common.cuh"

namespace ts {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

// r0 x + r1 y + r2 z + t in double-float
__device__ __forceinline__ ff dot3_add(float r0, float r1, float r2, float x, float y, float z,
                                       float t) {
    ff p0 = two_prod(r0, x), p1 = two_prod(r1, y), p2 = two_prod(r2, z);
    ff s = two_sum(p0.hi, p1.hi);
    float lo = s.lo + p0.lo + p1.lo;
    ff s2 = two_sum(s.hi, p2.hi);
    lo += s2.lo + p2.lo;
    ff s3 = two_sum(s2.hi, t);
    lo += s3.lo;
    return fast_two_sum(s3.hi, lo);
}

// f * (x / z) + c in double-float, x and z double-float
__device__ __forceinline__ ff project_ff(ff x, ff z, float f, float c) {
    float q = __fdiv_rn(x.hi, z.hi);
    float rem = fmaf(-q, z.hi, x.hi);  // exact remainder of the rounded quotient
    float ql = __fdiv_rn(rem + x.lo - q * z.lo, z.hi);
    ff p = two_prod(f, q);
    float plo = fmaf(f, ql, p.lo);
    ff s = two_sum(p.hi, c);
    return fast_two_sum(s.hi, s.lo + plo);
}

// Geometry of one (view, triangle) item.
struct Geom {
    float3 xc[3];      // camera-space vertices (FP32)
    ff u0, v0;         // projection of vertex 0
    float2 Q1, Q2;     // projections of vertices 1, 2 relative to vertex 0
    float ell[3];      // side opposite vertex i
    float area2;       // (q1 - q0) x (q2 - q0)
    float perim, r;    // perimeter, inradius
    float2 S;          // incenter relative to vertex 0
    float A[3], B[3];  // slopes of the normalised edge lines
    float depth;       // camera-space centroid depth
};

enum { CULL_NONE = 0, CULL_NEAR = 1, CULL_DEGENERATE = 2 };

// FWD = false (the backward pass, which needs the geometry only to 1e-6 relative):
// no projection of vertex 0 (u0, v0) and no edge-line slopes (A, B); approximate
// reciprocals instead of divisions.
template <bool FWD = true>
__device__ __forceinline__ int item_geometry(const float *v, const ViewDev &V, Geom &g) {
    ff X = dot3_add(V.R[0], V.R[1], V.R[2], v[0], v[1], v[2], V.t[0]);
    ff Y = dot3_add(V.R[3], V.R[4], V.R[5], v[0], v[1], v[2], V.t[1]);
    ff Z = dot3_add(V.R[6], V.R[7], V.R[8], v[0], v[1], v[2], V.t[2]);
    float d1x = v[3] - v[0], d1y = v[4] - v[1], d1z = v[5] - v[2];
    float d2x = v[6] - v[0], d2y = v[7] - v[1], d2z = v[8] - v[2];
    float3 e1 = make_float3(fmaf(V.R[0], d1x, fmaf(V.R[1], d1y, V.R[2] * d1z)),
                            fmaf(V.R[3], d1x, fmaf(V.R[4], d1y, V.R[5] * d1z)),
                            fmaf(V.R[6], d1x, fmaf(V.R[7], d1y, V.R[8] * d1z)));
    float3 e2 = make_float3(fmaf(V.R[0], d2x, fmaf(V.R[1], d2y, V.R[2] * d2z)),
                            fmaf(V.R[3], d2x, fmaf(V.R[4], d2y, V.R[5] * d2z)),
                            fmaf(V.R[6], d2x, fmaf(V.R[7], d2y, V.R[8] * d2z)));
    const float X0 = X.hi + X.lo, Y0 = Y.hi + Y.lo, Z0 = Z.hi + Z.lo;
    const float z1 = Z0 + e1.z, z2 = Z0 + e2.z;
    g.xc[0] = make_float3(X0, Y0, Z0);
    g.xc[1] = make_float3(X0 + e1.x, Y0 + e1.y, z1);
    g.xc[2] = make_float3(X0 + e2.x, Y0 + e2.y, z2);
    g.depth = __fadd_rn(Z.hi, __fadd_rn(Z.lo, __fmul_rn(__fadd_rn(e1.z, e2.z), 1.0f / 3.0f)));
    if (Z0 < Z_NEAR || z1 < Z_NEAR || z2 < Z_NEAR) return CULL_NEAR;
    if (FWD) {
        g.u0 = project_ff(X, Z, V.fx, V.cx);
        g.v0 = project_ff(Y, Z, V.fy, V.cy);
    }
    // q_k - q_0 = f (e.x z0 - x0 e.z) / (z0 z_k)
    const float i1 = FWD ? 1.0f / (Z0 * z1) : rcp_approx(Z0 * z1), i2 = FWD ? 1.0f / (Z0 * z2) : rcp_approx(Z0 * z2);
    g.Q1 = make_float2(V.fx * fmaf(e1.x, Z0, -X0 * e1.z) * i1, V.fy * fmaf(e1.y, Z0, -Y0 * e1.z) * i1);
    g.Q2 = make_float2(V.fx * fmaf(e2.x, Z0, -X0 * e2.z) * i2, V.fy * fmaf(e2.y, Z0, -Y0 * e2.z) * i2);
    // sides opposite each vertex: E0 = Q2 - Q1, E1 = Q0 - Q2 = -Q2, E2 = Q1 - Q0 = Q1
    const float E0x = g.Q2.x - g.Q1.x, E0y = g.Q2.y - g.Q1.y;
    g.ell[0] = sqrtf(fmaf(E0x, E0x, E0y * E0y));
    g.ell[1] = sqrtf(fmaf(g.Q2.x, g.Q2.x, g.Q2.y * g.Q2.y));
    g.ell[2] = sqrtf(fmaf(g.Q1.x, g.Q1.x, g.Q1.y * g.Q1.y));
    // area2 = Q1.x Q2.y - Q1.y Q2.x with one compensated product
    const float w = g.Q1.y * g.Q2.x;
    const float err = fmaf(-g.Q1.y, g.Q2.x, w);
    g.area2 = fmaf(g.Q1.x, g.Q2.y, -w) + err;
    g.perim = g.ell[0] + g.ell[1] + g.ell[2];
    if (!FWD) {
        const float ip = rcp_approx(g.perim);
        g.r = fabsf(g.area2) * ip;
        g.S = make_float2((g.ell[1] * g.Q1.x + g.ell[2] * g.Q2.x) * ip, (g.ell[1] * g.Q1.y + g.ell[2] * g.Q2.y) * ip);
        return g.r >= R_MIN ? CULL_NONE : CULL_DEGENERATE;
    }
    g.r = fabsf(g.area2) / g.perim;
    if (!(g.r >= R_MIN)) return CULL_DEGENERATE;
    const float ip = 1.0f / g.perim;
    g.S = make_float2((g.ell[1] * g.Q1.x + g.ell[2] * g.Q2.x) * ip, (g.ell[1] * g.Q1.y + g.ell[2] * g.Q2.y) * ip);
    // m_i(p) = lambda_i(p) * perim / ell_i; grad m_i = (-E_i.y, E_i.x) * perim / (ell_i area2)
    const float k0 = g.perim / (g.ell[0] * g.area2);
    const float k1 = g.perim / (g.ell[1] * g.area2);
    const float k2 = g.perim / (g.ell[2] * g.area2);
    g.A[0] = -E0y * k0;      g.B[0] = E0x * k0;
    g.A[1] = g.Q2.y * k1;    g.B[1] = -g.Q2.x * k1;
    g.A[2] = -g.Q1.y * k2;   g.B[2] = g.Q1.x * k2;
    return CULL_NONE;
}

// Real spherical harmonics up to degree 3 in Cartesian form at a unit direction,
// index k = l*l + l + m. Y_l^m = sqrt(2) K_l^m P_l^|m|(cos t) {cos, sin}(|m| phi)
// (no Condon-Shortley phase), K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!); the
// constants below are those closed forms evaluated by hand.
namespace shc {
constexpr float c0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float c1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float c2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float c2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float c2c = 0.5462742152960396f;   // sqrt(15/(16 pi))
constexpr float c3a = 0.5900435899266435f;   // sqrt(35/(32 pi))
constexpr float c3b = 2.890611442640554f;    // sqrt(105/(4 pi))
constexpr float c3c = 0.4570457994644658f;   // sqrt(21/(32 pi))
constexpr float c3d = 0.3731763325901154f;   // sqrt(7/(16 pi))
constexpr float c3e = 1.445305721320277f;    // sqrt(105/(16 pi))
}  // namespace shc

// Centroid of the triangle's vertices v[0..8], in explicit round-to-nearest operations
// (so that no kernel fuses it into a later subtraction: the colour's view direction has
// the same bits in every kernel).
__device__ __forceinline__ void centroid(const float (&v)[9], float (&cen)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) cen[k] = __fmul_rn(__fadd_rn(__fadd_rn(v[k], v[3 + k]), v[6 + k]), 1.0f / 3.0f);
}

// Real SH basis up to degree 3 at the unit direction (x, y, z). Every operation is an
// explicit round-to-nearest multiply, subtract or fused multiply-add, so that all the
// kernels that inline it (forward, backward, one view or many) compute the same bits.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    using namespace shc;
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = __fmul_rn(c1, y);
    Y[2] = __fmul_rn(c1, z);
    Y[3] = __fmul_rn(c1, x);
    if (deg < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float dxy = __fsub_rn(xx, yy);
    Y[4] = __fmul_rn(__fmul_rn(c2a, x), y);
    Y[5] = __fmul_rn(__fmul_rn(c2a, y), z);
    Y[6] = __fmul_rn(c2b, fmaf(3.0f, zz, -1.0f));
    Y[7] = __fmul_rn(__fmul_rn(c2a, x), z);
    Y[8] = __fmul_rn(c2c, dxy);
    if (deg < 3) return;
    const float z5 = fmaf(5.0f, zz, -1.0f);
    Y[9] = __fmul_rn(__fmul_rn(c3a, y), fmaf(3.0f, xx, -yy));
    Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(c3b, x), y), z);
    Y[11] = __fmul_rn(__fmul_rn(c3c, y), z5);
    Y[12] = __fmul_rn(__fmul_rn(c3d, z), fmaf(5.0f, zz, -3.0f));
    Y[13] = __fmul_rn(__fmul_rn(c3c, x), z5);
    Y[14] = __fmul_rn(__fmul_rn(c3e, z), dxy);
    Y[15] = __fmul_rn(__fmul_rn(c3a, x), fmaf(-3.0f, yy, xx));
}

// sum_k gY[k] dY_k/d(x, y, z), the basis taken as polynomials in free x, y, z
__device__ __forceinline__ float3 sh_basis_vjp(int deg, float x, float y, float z, const float *gY) {
    using namespace shc;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (deg >= 1) {
        gy += c1 * gY[1];
        gz += c1 * gY[2];
        gx += c1 * gY[3];
    }
    if (deg >= 2) {
        gx += c2a * y * gY[4];        gy += c2a * x * gY[4];
        gy += c2a * z * gY[5];        gz += c2a * y * gY[5];
        gz += 6.0f * c2b * z * gY[6];
        gx += c2a * z * gY[7];        gz += c2a * x * gY[7];
        gx += 2.0f * c2c * x * gY[8]; gy -= 2.0f * c2c * y * gY[8];
    }
    if (deg >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += 6.0f * c3a * x * y * gY[9];       gy += 3.0f * c3a * (xx - yy) * gY[9];
        gx += c3b * y * z * gY[10];             gy += c3b * x * z * gY[10];  gz += c3b * x * y * gY[10];
        gy += c3c * (5.0f * zz - 1.0f) * gY[11]; gz += 10.0f * c3c * y * z * gY[11];
        gz += c3d * (15.0f * zz - 3.0f) * gY[12];
        gx += c3c * (5.0f * zz - 1.0f) * gY[13]; gz += 10.0f * c3c * x * z * gY[13];
        gx += 2.0f * c3e * x * z * gY[14];      gy -= 2.0f * c3e * y * z * gY[14]; gz += c3e * (xx - yy) * gY[14];
        gx += 3.0f * c3a * (xx - yy) * gY[15];  gy -= 6.0f * c3a * x * y * gY[15];
    }
    return make_float3(gx, gy, gz);
}

}  // namespace ts
