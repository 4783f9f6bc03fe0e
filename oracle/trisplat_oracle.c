/*
 * FP64 CPU oracle for the differentiable triangle-splat rasterizer of
 * "Triangle Splatting for Real-Time Radiance Field Rendering" (arXiv 2505.19175).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference leg may load this library. It shares no code, header,
 * constant table or helper with the CUDA path, and nothing in the product calls it.
 *
 * What it computes is the plain definition of the rendered image, not the tiled
 * method that reaches it faster:
 *   - pinhole projection of each vertex (Sec. 3.1, "Differentiable rasterization";
 *     the printed q = K(Rv + t) omits the perspective divide, read here as the
 *     standard u = fx x/z + cx, v = fy y/z + cy);
 *   - the 2D signed distance field phi(p) = max_i (n_i . p + d_i) with outward unit
 *     edge normals, its minimum at the incenter s, phi(s) = -inradius (Sec. 3.1,
 *     "A new window function");
 *   - the window I(p) = ReLU(phi(p)/phi(s))^sigma (Sec. 3.1, Eq. indicator1);
 *   - alpha = min(ALPHA_MAX, o I), kept when alpha >= ALPHA_MIN, composited front to
 *     back in order of camera-space centroid depth (ties: triangle id), stopping
 *     before a fragment that would drop transmittance below T_EPS (Sec. 3.1: the
 *     rendering equation of prior splatting work; depth sort by triangle centre,
 *     Supp. "Depth sorting"); with the sort constant set to SORT_PIXEL, the order is
 *     instead each pixel's own: the depth of the triangle's plane along the pixel's
 *     ray (the per-pixel sort the paper leaves to future work);
 *   - view-dependent colour from real spherical harmonics up to degree 3
 *     (Sec. 4: 48 colour floats per triangle), rgb = max(0, sum Y_lm c_lm + 0.5);
 *   - the tight screen rectangle of Supp. "Tile assignment": edges moved inward by
 *     d = r (tau/o)^(1/sigma), i.e. the triangle scaled about its incenter by
 *     f = 1 - (tau/o)^(1/sigma), tau = ALPHA_MIN.
 * Every pixel is tested against every triangle (brute force) or, in "fast" mode,
 * every triangle visits only the pixels of its padded vertex bounding box; the two
 * evaluate the identical per-(pixel, triangle) arithmetic and are bit-identical.
 *
 * The adjoint differentiates that definition: per pixel, reverse-mode through the
 * compositing sum, and forward-mode dual numbers for alpha and rgb as functions of
 * the 9 vertex coordinates, o and sigma; SH coefficients enter linearly.
 *
 * For comparisons against an FP32 implementation it also classifies each pixel whose
 * value FP32 arithmetic cannot resolve to the image tolerance: a discontinuous
 * decision (alpha vs ALPHA_MIN, the T_EPS stop, depth order, culling) that lies within
 * an FP32 error band, or a first-order error estimate above half of 1e-4. Where a
 * decision lies in the band, either outcome is what the method computes in FP32, so
 * for those pixels it also lists every outcome reached by taking each such decision
 * both ways (and every order of depths within the band), each evaluated in FP64 by
 * the same compositing rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* constants and camera, passed as flat double arrays                  */
/* ------------------------------------------------------------------ */
/* window function: WIN_POWER is Eq. indicator1, I = ReLU(phi(p)/phi(s))^sigma;
 * WIN_SIGMOID is Eq. indicator2, I = sigmoid(-phi(p)/sigma), sigma in pixels */
enum { WIN_POWER = 0, WIN_SIGMOID = 1 };

/* compositing order: SORT_TILE is the paper's (each tile's entries by the camera depth
 * of the triangle's centroid, Supp. "Tile assignment"); SORT_PIXEL, the per-pixel
 * sort the paper leaves to future work, orders each pixel's fragments by the depth of
 * the triangle's plane along the pixel's ray. Ties go to the lower triangle id. */
enum { SORT_TILE = 0, SORT_PIXEL = 1 };

typedef struct {
    double alpha_max, alpha_min, t_eps, z_near, r_min, tile, rect_pad;
    int window, sort;
} consts_t;

typedef struct {
    double R[9], t[3], fx, fy, cx, cy;
    int W, H;
    double bg[3];
} cam_t;

static consts_t load_consts(const double *c) {
    consts_t k;
    k.alpha_max = c[0]; k.alpha_min = c[1]; k.t_eps = c[2]; k.z_near = c[3];
    k.r_min = c[4]; k.tile = c[5]; k.rect_pad = c[6];
    k.window = (int)c[7];
    k.sort = (int)c[8];
    return k;
}

static cam_t load_cam(const double *c) {
    cam_t m;
    for (int i = 0; i < 9; ++i) m.R[i] = c[i];
    for (int i = 0; i < 3; ++i) m.t[i] = c[9 + i];
    m.fx = c[12]; m.fy = c[13]; m.cx = c[14]; m.cy = c[15];
    m.W = (int)c[16]; m.H = (int)c[17];
    for (int i = 0; i < 3; ++i) m.bg[i] = c[18 + i];
    return m;
}

/* FP32 error model used only by the pixel classifier (not by the image). */
#define EPS_LINE 2.384185791015625e-07 /* 2^-22: FP32 line-evaluation error per unit term */
#define EPS_MUFU 9.5367431640625e-07   /* 2^-20: relative error of FP32 lg2/ex2 */
#define EPS_ACC  1.1920928955078125e-07 /* 2^-23: one FP32 rounding */
#define RECT_BAND 1.0e-3               /* px: FP32 error band of a rectangle bound */
#define FLAG_TOL 5.0e-5                /* flag a pixel whose error estimate exceeds this */

#define GRAD_TOL 1.0e-4               /* flag (for gradients) a fragment whose derivative is this uncertain */

/* Pixel flags. AMB_SKIP / STOP / ORDER / CULL: a decision within the FP32 band;
 * AMB_SENS: image error estimate above FLAG_TOL; AMB_UNRES: outcomes not enumerated;
 * AMB_GRAD: the image value is resolved but the pixel's gradient contribution is not
 * (a composited fragment whose window derivative or active edge FP32 cannot fix to
 * GRAD_TOL relative), so gradient comparisons leave the pixel out of the loss. */
enum { AMB_SKIP = 1, AMB_STOP = 2, AMB_ORDER = 4, AMB_SENS = 8, AMB_CULL = 16, AMB_UNRES = 32, AMB_GRAD = 64 };

/* ------------------------------------------------------------------ */
/* real spherical harmonics, degree <= 3                               */
/* ------------------------------------------------------------------ */
/* Legendre polynomial coefficients P_l(z) = sum_j leg[l][j] z^j from Bonnet's
 * recurrence (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1}. */
static double leg[4][4];
static double sh_K[4][4];   /* K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) */
static int sh_ready = 0;

static double fact(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

static void sh_init(void) {
    if (sh_ready) return;
    memset(leg, 0, sizeof leg);
    leg[0][0] = 1.0;
    leg[1][1] = 1.0;
    for (int l = 1; l < 3; ++l)
        for (int j = 0; j < 4; ++j) {
            double v = -(double)l * leg[l - 1][j];
            if (j > 0) v += (2.0 * l + 1.0) * leg[l][j - 1];
            leg[l + 1][j] = v / (l + 1.0);
        }
    for (int l = 0; l < 4; ++l)
        for (int m = 0; m <= l; ++m)
            sh_K[l][m] = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * fact(l - m) / fact(l + m));
    sh_ready = 1;
}

/* m-th derivative of P_l evaluated at z. */
static double leg_deriv(int l, int m, double z) {
    double acc = 0.0, zp = 1.0;
    for (int j = m; j <= l; ++j) {
        double c = leg[l][j];
        for (int k = 0; k < m; ++k) c *= (double)(j - k);
        acc += c * zp;
        zp *= z;
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* dual numbers: value + 11 partials (9 vertex coords, o, sigma)       */
/* ------------------------------------------------------------------ */
#define ND 11
typedef struct { double v, d[ND]; } dual;

static dual dcst(double v) { dual r; r.v = v; memset(r.d, 0, sizeof r.d); return r; }
static dual dvar(double v, int i) { dual r = dcst(v); r.d[i] = 1.0; return r; }
static dual dadd(dual a, dual b) { a.v += b.v; for (int i = 0; i < ND; ++i) a.d[i] += b.d[i]; return a; }
static dual dsub(dual a, dual b) { a.v -= b.v; for (int i = 0; i < ND; ++i) a.d[i] -= b.d[i]; return a; }
static dual dscale(dual a, double s) { a.v *= s; for (int i = 0; i < ND; ++i) a.d[i] *= s; return a; }
static dual daddc(dual a, double c) { a.v += c; return a; }
static dual dmul(dual a, dual b) {
    dual r; r.v = a.v * b.v;
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
static dual ddiv(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}
static dual dsqrt(dual a) {
    dual r; r.v = sqrt(a.v);
    for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
    return r;
}
/* 1 / (1 + exp(-a)) */
static dual dsigmoid(dual a) {
    dual r; r.v = 1.0 / (1.0 + exp(-a.v));
    const double s = r.v * (1.0 - r.v);
    for (int i = 0; i < ND; ++i) r.d[i] = s * a.d[i];
    return r;
}
/* a^b for a > 0, both dual */
static dual dpow(dual a, dual b) {
    dual r; r.v = pow(a.v, b.v);
    double la = log(a.v);
    for (int i = 0; i < ND; ++i) r.d[i] = r.v * (b.v * a.d[i] / a.v + la * b.d[i]);
    return r;
}

/* Y_k(dir) for k < (deg+1)^2, dual version (dir is a unit vector of duals). */
static void sh_eval_dual(int deg, const dual dir[3], dual *out) {
    sh_init();
    /* (x + i y)^m for m = 0..3 */
    dual re[4], im[4];
    re[0] = dcst(1.0); im[0] = dcst(0.0);
    for (int m = 1; m <= 3; ++m) {
        re[m] = dsub(dmul(re[m - 1], dir[0]), dmul(im[m - 1], dir[1]));
        im[m] = dadd(dmul(re[m - 1], dir[1]), dmul(im[m - 1], dir[0]));
    }
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            /* d^am P_l / dz^am at z, as a dual through dir[2] */
            double pv = leg_deriv(l, am, dir[2].v);
            double pd = (am < l) ? leg_deriv(l, am + 1, dir[2].v) : 0.0;
            dual P = dscale(dir[2], pd);
            P.v = pv;
            dual y;
            if (m == 0) y = dscale(P, sh_K[l][0]);
            else if (m > 0) y = dscale(dmul(P, re[am]), sqrt(2.0) * sh_K[l][am]);
            else y = dscale(dmul(P, im[am]), sqrt(2.0) * sh_K[l][am]);
            out[l * l + l + m] = y;
        }
    }
}

static void sh_eval_val(int deg, const double dir[3], double *out) {
    dual dd[3], y[16];
    for (int i = 0; i < 3; ++i) dd[i] = dcst(dir[i]);
    sh_eval_dual(deg, dd, y);
    for (int k = 0; k < (deg + 1) * (deg + 1); ++k) out[k] = y[k].v;
}

/* ------------------------------------------------------------------ */
/* 2D triangle: edges, outward normals, inradius, incenter             */
/* ------------------------------------------------------------------ */
typedef struct {
    double q[3][2];
    double ell[3];          /* side opposite vertex i */
    double area2;           /* (q1-q0) x (q2-q0) */
    double perim, r;        /* perimeter, inradius = |area2| / perim */
    double s[2];            /* incenter */
    double n[3][2], d[3];   /* L_i(p) = n_i . p + d_i, n_i outward unit normal of side i */
} tri2d_t;

static void tri2d_setup(const double q[3][2], tri2d_t *T) {
    memcpy(T->q, q, sizeof T->q);
    double ex[3], ey[3];
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        ex[i] = q[k][0] - q[j][0];
        ey[i] = q[k][1] - q[j][1];
        T->ell[i] = hypot(ex[i], ey[i]);
    }
    T->area2 = (q[1][0] - q[0][0]) * (q[2][1] - q[0][1]) - (q[1][1] - q[0][1]) * (q[2][0] - q[0][0]);
    T->perim = T->ell[0] + T->ell[1] + T->ell[2];
    T->r = T->perim > 0 ? fabs(T->area2) / T->perim : 0.0;
    if (T->perim > 0) {
        T->s[0] = (T->ell[0] * q[0][0] + T->ell[1] * q[1][0] + T->ell[2] * q[2][0]) / T->perim;
        T->s[1] = (T->ell[0] * q[0][1] + T->ell[1] * q[1][1] + T->ell[2] * q[2][1]) / T->perim;
    } else {
        T->s[0] = q[0][0]; T->s[1] = q[0][1];
    }
    double sg = T->area2 >= 0 ? 1.0 : -1.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        double l = T->ell[i] > 0 ? T->ell[i] : 1.0;
        /* edge i runs q_j -> q_k; (ey, -ex) is its right-hand normal, outward for a
         * counter-clockwise triangle, hence the sign of the signed area. */
        T->n[i][0] = sg * ey[i] / l;
        T->n[i][1] = -sg * ex[i] / l;
        T->d[i] = -(T->n[i][0] * q[j][0] + T->n[i][1] * q[j][1]);
    }
}

/* phi(p)/phi(s) with phi(s) = -r; also returns the arg-max edge (lowest index on ties) */
static double tri2d_ratio(const tri2d_t *T, double px, double py, int *amax) {
    double phi = -INFINITY;
    int am = 0;
    for (int i = 0; i < 3; ++i) {
        double L = T->n[i][0] * px + T->n[i][1] * py + T->d[i];
        if (L > phi) { phi = L; am = i; }
    }
    if (amax) *amax = am;
    return phi / (-T->r);
}

/* ------------------------------------------------------------------ */
/* per-triangle setup                                                  */
/* ------------------------------------------------------------------ */
enum { CULL_NONE = 0, CULL_NEAR = 1, CULL_DEGENERATE = 2 };
enum { RECT_OK = 0, RECT_LOW_OPACITY = 1, RECT_EMPTY = 2 };

typedef struct {
    int cull;               /* CULL_* : removes the triangle from the image */
    int amb_cull;           /* a cull decision within the FP32 band */
    double z[3], depth;
    double xc[3][3];        /* camera-space vertices */
    tri2d_t g;
    double o, sigma;
    double dir[3], rgb_raw[3], rgb[3];
    double bbox[4];         /* vertex bbox (xmin, ymin, xmax, ymax) */
    double ext[4];          /* pixel-candidate extent: bbox, or the rectangle when it is larger */
    /* tight rectangle */
    int rect_state;
    double f, rect[4];
    int pix[4], tiles[4], ntiles;
    int amb_rect;
} tri_t;

static void cam_center(const cam_t *C, double cp[3]) {
    for (int j = 0; j < 3; ++j)
        cp[j] = -(C->R[0 * 3 + j] * C->t[0] + C->R[1 * 3 + j] * C->t[1] + C->R[2 * 3 + j] * C->t[2]);
}

/* pixel range whose centres x + 0.5 lie in [lo, hi], clamped to [0, n-1] */
static void pix_range(double lo, double hi, int n, int *a, int *b) {
    if (lo < -2.0) lo = -2.0;
    if (hi > n + 2.0) hi = n + 2.0;
    if (hi < -2.0) hi = -2.0;
    if (lo > n + 2.0) lo = n + 2.0;
    int x0 = (int)ceil(lo - 0.5), x1 = (int)floor(hi - 0.5);
    if (x0 < 0) x0 = 0;
    if (x1 > n - 1) x1 = n - 1;
    *a = x0; *b = x1;
}

static void rect_tiles(const double rect[4], double pad, const cam_t *C, int tile, int pix[4], int tiles[4], int *ntiles) {
    pix_range(rect[0] - pad, rect[2] + pad, C->W, &pix[0], &pix[2]);
    pix_range(rect[1] - pad, rect[3] + pad, C->H, &pix[1], &pix[3]);
    if (pix[0] > pix[2] || pix[1] > pix[3]) {
        tiles[0] = tiles[1] = 0; tiles[2] = tiles[3] = -1; *ntiles = 0;
        return;
    }
    tiles[0] = pix[0] / tile; tiles[1] = pix[1] / tile;
    tiles[2] = pix[2] / tile; tiles[3] = pix[3] / tile;
    *ntiles = (tiles[2] - tiles[0] + 1) * (tiles[3] - tiles[1] + 1);
}

static void tri_setup(int id, const double *verts, const double *sh, int sh_deg,
                      const double *opac, const double *sigma, const cam_t *C,
                      const consts_t *K, tri_t *T) {
    memset(T, 0, sizeof *T);
    const double *v = verts + 9 * (size_t)id;
    double q[3][2];
    int near = 0, near_amb = 0;
    for (int i = 0; i < 3; ++i) {
        double X = v[3 * i], Y = v[3 * i + 1], Z = v[3 * i + 2];
        double xc = C->R[0] * X + C->R[1] * Y + C->R[2] * Z + C->t[0];
        double yc = C->R[3] * X + C->R[4] * Y + C->R[5] * Z + C->t[1];
        double zc = C->R[6] * X + C->R[7] * Y + C->R[8] * Z + C->t[2];
        T->z[i] = zc;
        T->xc[i][0] = xc; T->xc[i][1] = yc; T->xc[i][2] = zc;
        if (zc < K->z_near) near = 1;
        if (fabs(zc - K->z_near) <= 1e-5 * (1.0 + fabs(K->z_near))) near_amb = 1;
        if (zc > 0) {
            q[i][0] = C->fx * xc / zc + C->cx;
            q[i][1] = C->fy * yc / zc + C->cy;
        } else {
            q[i][0] = q[i][1] = 0.0;
        }
    }
    T->depth = (T->z[0] + T->z[1] + T->z[2]) / 3.0;
    T->o = opac[id];
    T->sigma = sigma[id];
    T->bbox[0] = fmin(q[0][0], fmin(q[1][0], q[2][0]));
    T->bbox[1] = fmin(q[0][1], fmin(q[1][1], q[2][1]));
    T->bbox[2] = fmax(q[0][0], fmax(q[1][0], q[2][0]));
    T->bbox[3] = fmax(q[0][1], fmax(q[1][1], q[2][1]));
    T->tiles[2] = T->tiles[3] = -1;
    memcpy(T->ext, T->bbox, sizeof T->ext);
    T->amb_cull = near_amb;
    tri2d_setup((const double (*)[2])q, &T->g);
    if (fabs(T->g.r - K->r_min) <= 0.01 * K->r_min) T->amb_cull = 1;
    if (near) { T->cull = CULL_NEAR; T->rect_state = RECT_EMPTY; return; }
    if (!(T->g.r >= K->r_min)) { T->cull = CULL_DEGENERATE; T->rect_state = RECT_EMPTY; return; }

    /* colour: direction from the camera centre to the world-space centroid */
    double cp[3], m[3], w2 = 0.0;
    cam_center(C, cp);
    for (int j = 0; j < 3; ++j) {
        m[j] = (v[j] + v[3 + j] + v[6 + j]) / 3.0;
        T->dir[j] = m[j] - cp[j];
        w2 += T->dir[j] * T->dir[j];
    }
    double wn = sqrt(w2);
    for (int j = 0; j < 3; ++j) T->dir[j] /= wn;
    double Y[16];
    int nk = (sh_deg + 1) * (sh_deg + 1);
    sh_eval_val(sh_deg, T->dir, Y);
    const double *c = sh + (size_t)id * nk * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < nk; ++k) acc += Y[k] * c[k * 3 + ch];
        T->rgb_raw[ch] = acc;
        T->rgb[ch] = acc > 0 ? acc : 0.0;
    }

    /* tight rectangle: triangle scaled about its incenter by f = 1 - c, c the window
     * ratio below which o I < tau (Supp. "Tile assignment"); for the sigmoid window
     * c = sigma ln(tau / (o - tau)) / r is negative when o > 2 tau: the support then
     * exceeds the triangle */
    if (K->window == WIN_SIGMOID)
        T->f = T->o > K->alpha_min ? 1.0 - T->sigma * log(K->alpha_min / (T->o - K->alpha_min)) / T->g.r : 0.0;
    else
        T->f = 1.0 - pow(K->alpha_min / T->o, 1.0 / T->sigma);
    if (fabs(T->f) <= 1e-5) T->amb_rect = 1;
    if (!(T->f > 0)) {
        T->rect_state = RECT_LOW_OPACITY;
        T->tiles[2] = T->tiles[3] = -1;
        return;
    }
    double w[3][2];
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 2; ++a) w[i][a] = T->g.s[a] + T->f * (q[i][a] - T->g.s[a]);
    T->rect[0] = fmin(w[0][0], fmin(w[1][0], w[2][0]));
    T->rect[1] = fmin(w[0][1], fmin(w[1][1], w[2][1]));
    T->rect[2] = fmax(w[0][0], fmax(w[1][0], w[2][0]));
    T->rect[3] = fmax(w[0][1], fmax(w[1][1], w[2][1]));
    if (!(T->f < 1e6)) {   /* unbounded support (sigmoid window without a cutoff) */
        T->rect[0] = T->rect[1] = -INFINITY;
        T->rect[2] = T->rect[3] = INFINITY;
    }
    int tile = (int)K->tile;
    rect_tiles(T->rect, K->rect_pad, C, tile, T->pix, T->tiles, &T->ntiles);
    T->rect_state = T->ntiles > 0 ? RECT_OK : RECT_EMPTY;
    if (T->f > 1.0) memcpy(T->ext, T->rect, sizeof T->ext);
    /* a bound within the FP32 band of a boundary that changes the tile set */
    int pp[4], tt[4], nn;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
        rect_tiles(T->rect, K->rect_pad + sgn * RECT_BAND, C, tile, pp, tt, &nn);
        if (nn != T->ntiles || (nn > 0 && memcmp(tt, T->tiles, sizeof tt) != 0)) T->amb_rect = 1;
    }
}

/* ------------------------------------------------------------------ */
/* dual setup of one triangle (only for the adjoint)                   */
/* ------------------------------------------------------------------ */
typedef struct {
    dual n[3][2], d[3], r, o, sigma, rgb_raw[3];
    double Y[16];
} tri_dual_t;

static void tri_dual_setup(int id, const double *verts, const double *sh, int sh_deg,
                           const cam_t *C, const tri_t *T, tri_dual_t *D) {
    const double *v = verts + 9 * (size_t)id;
    dual V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) V[i][a] = dvar(v[3 * i + a], 3 * i + a);
    dual q[3][2];
    for (int i = 0; i < 3; ++i) {
        dual xc = daddc(dadd(dadd(dscale(V[i][0], C->R[0]), dscale(V[i][1], C->R[1])), dscale(V[i][2], C->R[2])), C->t[0]);
        dual yc = daddc(dadd(dadd(dscale(V[i][0], C->R[3]), dscale(V[i][1], C->R[4])), dscale(V[i][2], C->R[5])), C->t[1]);
        dual zc = daddc(dadd(dadd(dscale(V[i][0], C->R[6]), dscale(V[i][1], C->R[7])), dscale(V[i][2], C->R[8])), C->t[2]);
        q[i][0] = daddc(dscale(ddiv(xc, zc), C->fx), C->cx);
        q[i][1] = daddc(dscale(ddiv(yc, zc), C->fy), C->cy);
    }
    dual ex[3], ey[3], ell[3];
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        ex[i] = dsub(q[k][0], q[j][0]);
        ey[i] = dsub(q[k][1], q[j][1]);
        ell[i] = dsqrt(dadd(dmul(ex[i], ex[i]), dmul(ey[i], ey[i])));
    }
    dual area2 = dsub(dmul(dsub(q[1][0], q[0][0]), dsub(q[2][1], q[0][1])),
                      dmul(dsub(q[1][1], q[0][1]), dsub(q[2][0], q[0][0])));
    double sg = T->g.area2 >= 0 ? 1.0 : -1.0;
    dual perim = dadd(dadd(ell[0], ell[1]), ell[2]);
    D->r = ddiv(dscale(area2, sg), perim);
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        D->n[i][0] = dscale(ddiv(ey[i], ell[i]), sg);
        D->n[i][1] = dscale(ddiv(ex[i], ell[i]), -sg);
        D->d[i] = dscale(dadd(dmul(D->n[i][0], q[j][0]), dmul(D->n[i][1], q[j][1])), -1.0);
    }
    D->o = dvar(T->o, 9);
    D->sigma = dvar(T->sigma, 10);
    /* colour */
    double cp[3];
    cam_center(C, cp);
    dual w[3], w2 = dcst(0.0);
    for (int a = 0; a < 3; ++a) {
        w[a] = daddc(dscale(dadd(dadd(V[0][a], V[1][a]), V[2][a]), 1.0 / 3.0), -cp[a]);
        w2 = dadd(w2, dmul(w[a], w[a]));
    }
    dual wn = dsqrt(w2), dir[3];
    for (int a = 0; a < 3; ++a) dir[a] = ddiv(w[a], wn);
    dual Y[16];
    int nk = (sh_deg + 1) * (sh_deg + 1);
    sh_eval_dual(sh_deg, dir, Y);
    const double *c = sh + (size_t)id * nk * 3;
    for (int ch = 0; ch < 3; ++ch) {
        dual acc = dcst(0.5);
        for (int k = 0; k < nk; ++k) acc = dadd(acc, dscale(Y[k], c[k * 3 + ch]));
        D->rgb_raw[ch] = acc;
    }
    for (int k = 0; k < nk; ++k) D->Y[k] = Y[k].v;
}

/* alpha at pixel p as a dual (same formula and arg-max rule as the value path) */
static dual frag_alpha_dual(const tri_dual_t *D, double px, double py, const consts_t *K) {
    dual phi = dcst(-INFINITY);
    for (int i = 0; i < 3; ++i) {
        dual L = dadd(dadd(dscale(D->n[i][0], px), dscale(D->n[i][1], py)), D->d[i]);
        if (L.v > phi.v) phi = L;
    }
    dual ratio = ddiv(dscale(phi, -1.0), D->r);
    dual I = K->window == WIN_SIGMOID ? dsigmoid(ddiv(dscale(phi, -1.0), D->sigma)) : dpow(ratio, D->sigma);
    dual a = dmul(D->o, I);
    if (a.v > K->alpha_max) a = dcst(K->alpha_max);
    return a;
}

/* ------------------------------------------------------------------ */
/* rendering                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int pix, id;
    double depth, alpha, ratio;
    int kept;       /* alpha >= ALPHA_MIN */
    int argmax;
} ent_t;

static int ent_cmp(const void *a, const void *b) {
    const ent_t *x = (const ent_t *)a, *y = (const ent_t *)b;
    if (x->pix != y->pix) return x->pix < y->pix ? -1 : 1;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

typedef struct { ent_t *e; size_t n, cap; } vec_t;

static void vec_push(vec_t *v, ent_t x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->e = (ent_t *)realloc(v->e, v->cap * sizeof(ent_t));
    }
    v->e[v->n++] = x;
}

/* camera depth of the plane of triangle t along the ray through pixel point (px, py):
 * z = (n . x0) / (n . d), n = (x1 - x0) x (x2 - x0), d = ((px - cx) / fx, (py - cy) / fy, 1) */
static double pixel_depth(const tri_t *t, const cam_t *C, double px, double py) {
    const double *a = t->xc[0], *b = t->xc[1], *c = t->xc[2];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double d[3] = {(px - C->cx) / C->fx, (py - C->cy) / C->fy, 1.0};
    return (n[0] * a[0] + n[1] * a[1] + n[2] * a[2]) / (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]);
}

/* window value of triangle t at window ratio `ratio` (FP64) */
static double window_I(const consts_t *K, const tri_t *t, double ratio) {
    if (K->window == WIN_SIGMOID) return 1.0 / (1.0 + exp(-t->g.r * ratio / t->sigma));
    return ratio > 0 ? pow(ratio, t->sigma) : 0.0;
}

/* relative error of the FP32 window evaluation (approximate lg2 / ex2 / rcp) */
static double window_rel(const consts_t *K, const tri_t *t, double ratio) {
    if (K->window == WIN_SIGMOID) return EPS_MUFU * (2.0 + fabs(t->g.r * ratio / t->sigma));
    return EPS_MUFU * (1.0 + t->sigma * fabs(log2(fmax(ratio, 1e-300))));
}

static double ulp32(double x) {
    int e;
    frexp(fabs(x), &e);   /* x = m 2^e, m in [0.5, 1) */
    return ldexp(1.0, e - 24);
}

/* FP32 error band of the window ratio at p (classifier only) */
static double ratio_band(const tri2d_t *g, int am, double px, double py) {
    double ax = fabs(g->n[am][0] * (px - g->s[0])) / g->r;
    double ay = fabs(g->n[am][1] * (py - g->s[1])) / g->r;
    return EPS_LINE * (1.0 + ax + ay);
}

/* Relative FP32 uncertainty of a composited fragment's contribution to the gradient
 * (classifier only). The window's derivative, sigma ratio^(sigma-1) for
 * Eq. indicator1 or kappa I (1 - I) for Eq. indicator2, and the vertex derivative of
 * the active edge's value (which vanishes with the ratio for the opposite vertex)
 * carry the ratio's absolute error `band` relative to the ratio itself; and where two
 * edges are within the band of the maximum, FP32 may take the other one, whose
 * derivative differs (Sec. 3.1: phi is a max over the edges). */
static double grad_sens(const consts_t *K, const tri_t *t, const ent_t *f, double band, double px, double py) {
    const tri2d_t *g = &t->g;
    double second = -INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (i == f->argmax) continue;
        double L = (g->n[i][0] * px + g->n[i][1] * py + g->d[i]) / g->r;
        if (L > second) second = L;
    }
    /* -ratio is the largest scaled edge value */
    if (-f->ratio - second <= 2.0 * band) return INFINITY;
    const double ar = fabs(f->ratio);
    if (K->window == WIN_SIGMOID) {
        const double kap = g->r / t->sigma;
        const double I = 1.0 / (1.0 + exp(-kap * f->ratio));
        return band * (kap * fabs(1.0 - 2.0 * I) + (ar > 0 ? 1.0 / ar : INFINITY));
    }
    return band * (1.0 + fmax(t->sigma, fabs(t->sigma - 1.0))) / ar;
}

typedef struct {
    int n, sh_deg, nk;
    const double *verts, *sh, *opac, *sigma;
    cam_t C;
    consts_t K;
    tri_t *tris;
    int brute;
    const uint8_t *pix_mask;
    /* forward outputs (nullable) */
    double *image, *T_final;
    int32_t *n_kept;
    uint8_t *flags;
    double *err_est;
    /* alternative outcomes of pixels with a decision in the FP32 band (nullable):
     * a shared list of capacity alt_cap, its fill count at *alt_n */
    struct alt_s *alts;
    size_t alt_cap;
    size_t *alt_n;
    /* pruning statistics per triangle (nullable, Sec. 3.3 "Pruning"): largest
     * blending weight T o over its composited fragments, number of pixels where it
     * was composited, and 1 when a pixel it took part in is flagged */
    double *max_weight;
    int32_t *n_pix;
    uint8_t *tri_amb;
    /* adjoint (nullable) */
    const double *dL;
    const int32_t *track;        /* triangle id -> dual slot, or -1 */
    const tri_dual_t *duals;
    double *dverts, *dsh, *dopac, *dsigma;
} job_t;

#define BAND 8

static void atomic_add(double *p, double v) {
#ifdef _OPENMP
#pragma omp atomic
#endif
    *p += v;
}

/* ------------------------------------------------------------------ */
/* alternative outcomes of a pixel whose decisions lie in the FP32 band */
/* ------------------------------------------------------------------ */
/* One outcome: the pixel's colour (background included), final transmittance and
 * number of composited fragments. */
typedef struct alt_s {
    int32_t pix, nk;
    double C[3], T;
} alt_t;

#define ALT_PER_PIX 64   /* outcomes listed per pixel at most */
#define ALT_RUN_MAX 3    /* longest run of depths within the band that is permuted */

typedef struct {
    const job_t *J;
    const ent_t **ord;   /* the pixel's candidate fragments in one admissible order */
    size_t cnt;
    double px, py;
    alt_t leaf[ALT_PER_PIX];
    int nleaf, over;
} walk_t;

static void alt_leaf(walk_t *W, double T, const double C[3], int nk) {
    if (W->nleaf == ALT_PER_PIX) { W->over = 1; return; }
    alt_t *a = &W->leaf[W->nleaf++];
    for (int c = 0; c < 3; ++c) a->C[c] = C[c] + T * W->J->C.bg[c];
    a->T = T;
    a->nk = nk;
}

/* the alpha band [alo, ahi] of fragment f, as the classifier of shade_pixel bounds it */
static void alpha_band(const job_t *J, const ent_t *f, double px, double py, double *alo, double *ahi) {
    const consts_t *K = &J->K;
    const tri_t *t = &J->tris[f->id];
    double band = ratio_band(&t->g, f->argmax, px, py);
    double wrel = window_rel(K, t, f->ratio);
    *ahi = t->o * window_I(K, t, f->ratio + band) * (1.0 + wrel);
    double rlo = f->ratio - band;
    *alo = (rlo > 0 || K->window == WIN_SIGMOID) ? t->o * window_I(K, t, rlo) * (1.0 - wrel) : 0.0;
}

/* Composite W->ord[i..] front to back from the state (T, C, nk, dTrel), taking every
 * keep/skip and stop/continue decision that lies in the FP32 band both ways and every
 * other decision as FP64 takes it; each path ends in one outcome. */
static void alt_walk(walk_t *W, size_t i, double T, const double C0[3], int nk, double dTrel) {
    const job_t *J = W->J;
    const consts_t *K = &J->K;
    double C[3] = {C0[0], C0[1], C0[2]};
    for (; i < W->cnt && !W->over; ++i) {
        const ent_t *f = W->ord[i];
        const tri_t *t = &J->tris[f->id];
        double alo, ahi;
        alpha_band(J, f, W->px, W->py, &alo, &ahi);
        const int can_keep = f->kept || ahi >= K->alpha_min;
        const int can_skip = !f->kept || alo < K->alpha_min;
        if (!can_keep) continue;
        if (can_skip) alt_walk(W, i + 1, T, C, nk, dTrel);   /* the fragment skipped */
        /* the fragment kept: its FP64 alpha (below ALPHA_MIN by rounding when FP64 skips it) */
        const double a = f->alpha;
        const double da = alo >= K->alpha_max ? 0.0 : fmax(fmin(ahi, K->alpha_max) - a, a - alo);
        const double test = T * (1.0 - a);
        if (K->t_eps > 0) {
            const double rel = dTrel + da / (1.0 - a) + (nk + 1) * EPS_ACC;
            const int amb = fabs(test - K->t_eps) <= 2.0 * test * rel;
            if (test < K->t_eps || amb) alt_leaf(W, T, C, nk);   /* stopped before it */
            if (test < K->t_eps && !amb) return;
        }
        for (int c = 0; c < 3; ++c) C[c] += t->rgb[c] * a * T;
        T = test;
        dTrel += da / (1.0 - a);
        ++nk;
    }
    if (!W->over) alt_leaf(W, T, C, nk);
}

/* next permutation of p[0..n) in lexicographic order; 0 after the last one */
static int next_perm(int *p, int n) {
    int i = n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int j = n - 1;
    while (p[j] <= p[i]) --j;
    int tmp = p[i]; p[i] = p[j]; p[j] = tmp;
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) { tmp = p[a]; p[a] = p[b]; p[b] = tmp; }
    return 1;
}

/* List the outcomes of pixel pix into J->alts. The candidates are the fragments that
 * FP32 may keep; runs of consecutive candidates whose depths lie within the band of
 * one another may be composited in any order (runs longer than ALT_RUN_MAX are not
 * enumerated). Returns AMB_UNRES when the outcomes could not all be listed: a cull
 * decision in the band, a longer run, more than ALT_PER_PIX outcomes, or a full list. */
static int pixel_alternatives(const job_t *J, const ent_t *e, size_t cnt, int pix, double px, double py) {
    const consts_t *K = &J->K;
    const ent_t **cand = (const ent_t **)malloc(sizeof(*cand) * (cnt > 0 ? cnt : 1));
    size_t nc = 0;
    for (size_t i = 0; i < cnt; ++i) {
        if (e[i].kept < 0) { free(cand); return AMB_UNRES; }
        double alo, ahi;
        alpha_band(J, &e[i], px, py, &alo, &ahi);
        if (e[i].kept || ahi >= K->alpha_min) cand[nc++] = &e[i];
    }
    /* runs of depths within the band, as run start and length */
    size_t *rs = (size_t *)malloc(sizeof(size_t) * (nc > 0 ? nc : 1));
    int *rl = (int *)malloc(sizeof(int) * (nc > 0 ? nc : 1));
    size_t nr = 0;
    for (size_t i = 0; i < nc;) {
        size_t j = i + 1;
        while (j < nc) {
            const double dband = (K->sort == SORT_PIXEL ? 64.0 : 4.0) * ulp32(cand[j - 1]->depth);
            if (fabs(cand[j]->depth - cand[j - 1]->depth) > dband) break;
            ++j;
        }
        if (j - i > 1) { rs[nr] = i; rl[nr] = (int)(j - i); ++nr; }
        i = j;
    }
    walk_t *W = (walk_t *)malloc(sizeof(walk_t));
    W->J = J; W->cnt = nc; W->px = px; W->py = py; W->nleaf = 0; W->over = 0;
    W->ord = (const ent_t **)malloc(sizeof(*W->ord) * (nc > 0 ? nc : 1));
    int unres = 0;
    for (size_t r = 0; r < nr; ++r)
        if (rl[r] > ALT_RUN_MAX) unres = 1;
    /* every combination of one permutation per run (odometer over the runs) */
    int perm[64][ALT_RUN_MAX];
    if (nr > 64) unres = 1;
    for (size_t r = 0; r < nr && !unres; ++r)
        for (int k = 0; k < rl[r]; ++k) perm[r][k] = k;
    const double C0[3] = {0.0, 0.0, 0.0};
    while (!unres && !W->over) {
        for (size_t i = 0; i < nc; ++i) W->ord[i] = cand[i];
        for (size_t r = 0; r < nr; ++r)
            for (int k = 0; k < rl[r]; ++k) W->ord[rs[r] + k] = cand[rs[r] + perm[r][k]];
        alt_walk(W, 0, 1.0, C0, 0, 0.0);
        size_t r = 0;
        while (r < nr && !next_perm(perm[r], rl[r])) ++r;   /* wrapped runs restart at identity */
        if (r == nr) break;
    }
    if (W->over) unres = 1;
    if (!unres) {
        size_t base;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
        { base = *J->alt_n; *J->alt_n += (size_t)W->nleaf; }
        if (base + (size_t)W->nleaf > J->alt_cap) unres = 1;
        else
            for (int k = 0; k < W->nleaf; ++k) {
                J->alts[base + k] = W->leaf[k];
                J->alts[base + k].pix = pix;
            }
    }
    free(W->ord);
    free(W);
    free(rs);
    free(rl);
    free(cand);
    return unres ? AMB_UNRES : 0;
}

/* composite one pixel's sorted entries [e0, e1) */
static void shade_pixel(const job_t *J, const ent_t *e, size_t cnt, int x, int y) {
    const consts_t *K = &J->K;
    const int W = J->C.W, H = J->C.H;
    const size_t pix = (size_t)y * W + x;
    double px = x + 0.5, py = y + 0.5;
    double T = 1.0, C[3] = {0, 0, 0};
    int amb = 0, nk = 0;
    double dTrel = 0.0;
    /* kept fragments, for the suffix pass */
    enum { MAXK = 4096 };
    static __thread int kid[MAXK];
    static __thread double ka[MAXK], kT[MAXK], kda[MAXK];
    double prev_depth = NAN;
    for (size_t i = 0; i < cnt; ++i) {
        const ent_t *f = &e[i];
        const tri_t *t = &J->tris[f->id];
        if (f->kept < 0) { amb |= AMB_CULL; continue; }
        double band = ratio_band(&t->g, f->argmax, px, py);
        double wrel = window_rel(K, t, f->ratio);
        double ahi = t->o * window_I(K, t, f->ratio + band) * (1.0 + wrel);
        double rlo = f->ratio - band;
        double alo = (rlo > 0 || K->window == WIN_SIGMOID) ? t->o * window_I(K, t, rlo) * (1.0 - wrel) : 0.0;
        if (!f->kept) {
            if (ahi >= K->alpha_min) amb |= AMB_SKIP;
            continue;
        }
        if (alo < K->alpha_min) amb |= AMB_SKIP;
        double a = f->alpha;
        double da;
        if (alo >= K->alpha_max) da = 0.0;
        else da = fmax(fmin(ahi, K->alpha_max) - a, a - alo);
        /* FP32 depth keys that may swap: the centroid depth (a few roundings), or the
         * per-pixel plane depth (a plane evaluation and a reciprocal) */
        const double dband = (K->sort == SORT_PIXEL ? 64.0 : 4.0) * ulp32(f->depth);
        if (!isnan(prev_depth) && fabs(f->depth - prev_depth) <= dband) amb |= AMB_ORDER;
        prev_depth = f->depth;
        double test = T * (1.0 - a);
        if (K->t_eps > 0) {
            double rel = dTrel + da / (1.0 - a) + (nk + 1) * EPS_ACC;
            if (fabs(test - K->t_eps) <= 2.0 * test * rel) amb |= AMB_STOP;
        }
        if (test < K->t_eps) break;
        if (grad_sens(K, t, f, band, px, py) > GRAD_TOL) amb |= AMB_GRAD;
        if (J->n_pix) {
            const double wgt = T * t->o;
#ifdef _OPENMP
#pragma omp atomic
#endif
            J->n_pix[f->id] += 1;
#ifdef _OPENMP
#pragma omp critical(orc_max_weight)
#endif
            if (J->max_weight[f->id] < wgt) J->max_weight[f->id] = wgt;
        }
        for (int c = 0; c < 3; ++c) C[c] += t->rgb[c] * a * T;
        if (nk < MAXK) { kid[nk] = f->id; ka[nk] = a; kT[nk] = T; kda[nk] = da; }
        T = test;
        dTrel += da / (1.0 - a);
        ++nk;
    }
    if (nk > MAXK) nk = MAXK;  /* never reached at the sizes used */
    for (int c = 0; c < 3; ++c) C[c] += T * J->C.bg[c];
    if (J->image)
        for (int c = 0; c < 3; ++c) J->image[(size_t)c * W * H + pix] = C[c];
    if (J->T_final) J->T_final[pix] = T;
    if (J->n_kept) J->n_kept[pix] = nk;

    /* suffix pass: B = colour from fragment k+1 on, plus the background term */
    double B[3];
    for (int c = 0; c < 3; ++c) B[c] = T * J->C.bg[c];
    double E = 0.0;
    const double *g = J->dL ? J->dL : NULL;
    for (int k = nk - 1; k >= 0; --k) {
        const tri_t *t = &J->tris[kid[k]];
        double a = ka[k], Tk = kT[k];
        double dCda = 0.0, gal = 0.0;
        for (int c = 0; c < 3; ++c) {
            double dc = t->rgb[c] * Tk - B[c] / (1.0 - a);
            if (fabs(dc) > dCda) dCda = fabs(dc);
            if (g) gal += g[(size_t)c * W * H + pix] * dc;
        }
        E += dCda * kda[k] + a * Tk * 1e-6 * (1.0 + fabs(t->rgb[0]) + fabs(t->rgb[1]) + fabs(t->rgb[2]));
        if (g && J->track && J->track[kid[k]] >= 0) {
            const tri_dual_t *D = &J->duals[J->track[kid[k]]];
            dual ad = frag_alpha_dual(D, px, py, K);
            int id = kid[k];
            double grgb[3];
            for (int c = 0; c < 3; ++c)
                grgb[c] = (D->rgb_raw[c].v > 0) ? g[(size_t)c * W * H + pix] * a * Tk : 0.0;
            for (int j = 0; j < 9; ++j) {
                double acc = gal * ad.d[j];
                for (int c = 0; c < 3; ++c) acc += grgb[c] * D->rgb_raw[c].d[j];
                atomic_add(&J->dverts[(size_t)id * 9 + j], acc);
            }
            atomic_add(&J->dopac[id], gal * ad.d[9]);
            atomic_add(&J->dsigma[id], gal * ad.d[10]);
            for (int kk = 0; kk < J->nk; ++kk)
                for (int c = 0; c < 3; ++c)
                    if (grgb[c] != 0.0) atomic_add(&J->dsh[((size_t)id * J->nk + kk) * 3 + c], grgb[c] * D->Y[kk]);
        }
        for (int c = 0; c < 3; ++c) B[c] += t->rgb[c] * a * Tk;
    }
    E += nk * 4.0 * EPS_ACC;
    if (E > FLAG_TOL) amb |= AMB_SENS;
    if (J->alts && (amb & (AMB_SKIP | AMB_STOP | AMB_ORDER | AMB_CULL)))
        amb |= pixel_alternatives(J, e, cnt, (int)pix, px, py);
    if (J->flags) J->flags[pix] = (uint8_t)amb;
    if (J->err_est) J->err_est[pix] = E;
    if (J->tri_amb && (amb & ~AMB_GRAD))
        for (size_t i = 0; i < cnt; ++i) J->tri_amb[e[i].id] = 1;   /* benign race: all write 1 */
}

static void render_band(const job_t *J, int y0, int y1, const int *cand, int ncand) {
    const int W = J->C.W;
    const consts_t *K = &J->K;
    vec_t v = {0};
    int want_flags = J->flags != NULL || J->err_est != NULL;
    for (int ci = 0; ci < ncand; ++ci) {
        int id = cand[ci];
        const tri_t *t = &J->tris[id];
        if (t->cull) {
            /* a culled triangle whose cull decision is within the FP32 band: its
             * pixels are marked, provided its projection exists (all z > 0) */
            if (!(want_flags && t->amb_cull && t->z[0] > 0 && t->z[1] > 0 && t->z[2] > 0)) continue;
        }
        int xa, xb, ya, yb;
        if (J->brute) { xa = 0; xb = W - 1; ya = y0; yb = y1 - 1; }
        else {
            pix_range(t->ext[0] - 1.0, t->ext[2] + 1.0, W, &xa, &xb);
            pix_range(t->ext[1] - 1.0, t->ext[3] + 1.0, J->C.H, &ya, &yb);
            if (ya < y0) ya = y0;
            if (yb > y1 - 1) yb = y1 - 1;
        }
        for (int y = ya; y <= yb; ++y)
            for (int x = xa; x <= xb; ++x) {
                size_t pix = (size_t)y * W + x;
                if (J->pix_mask && !J->pix_mask[pix]) continue;
                double px = x + 0.5, py = y + 0.5;
                if (t->cull) {
                    /* ambiguous degenerate triangle: mark the pixels around it */
                    if (px >= t->bbox[0] - 1 && px <= t->bbox[2] + 1 && py >= t->bbox[1] - 1 && py <= t->bbox[3] + 1) {
                        ent_t e = {(int)pix, id, t->depth, 0.0, 0.0, -1, 0};
                        vec_push(&v, e);
                    }
                    continue;
                }
                int am;
                double ratio = tri2d_ratio(&t->g, px, py, &am);
                const int sig = K->window == WIN_SIGMOID;
                double araw = (ratio > 0 || sig) ? t->o * window_I(K, t, ratio) : 0.0;
                /* a fragment needs alpha >= ALPHA_MIN (and, for the power window, a
                 * positive window ratio) */
                int kept = (ratio > 0 || sig) && araw >= K->alpha_min;
                if (!kept) {
                    if (!want_flags) continue;
                    double band = ratio_band(&t->g, am, px, py);
                    if (!sig && ratio + band <= 0) continue;
                    double ahi = t->o * window_I(K, t, ratio + band) * (1.0 + 4.0 * window_rel(K, t, ratio));
                    if (ahi < K->alpha_min) continue;
                }
                ent_t e;
                e.pix = (int)pix; e.id = id;
                e.depth = K->sort == SORT_PIXEL ? pixel_depth(t, &J->C, px, py) : t->depth;
                e.alpha = araw < K->alpha_max ? araw : K->alpha_max;
                e.ratio = ratio; e.kept = kept; e.argmax = am;
                vec_push(&v, e);
                if (t->amb_cull && want_flags) {
                    ent_t m = e; m.kept = -1;
                    vec_push(&v, m);
                }
            }
    }
    qsort(v.e, v.n, sizeof(ent_t), ent_cmp);
    /* every pixel of the band gets written, with or without fragments */
    size_t i = 0;
    for (int y = y0; y < y1; ++y)
        for (int x = 0; x < W; ++x) {
            int pix = y * W + x;
            size_t j = i;
            while (j < v.n && v.e[j].pix == pix) ++j;
            if (!J->pix_mask || J->pix_mask[pix]) shade_pixel(J, v.e + i, j - i, x, y);
            i = j;
        }
    free(v.e);
}

static void run_job(job_t *J) {
    const int H = J->C.H;
    int nb = (H + BAND - 1) / BAND;
    /* candidate lists per band */
    int *cnt = (int *)calloc((size_t)nb + 1, sizeof(int));
    int *all = NULL;
    if (!J->brute) {
        for (int id = 0; id < J->n; ++id) {
            const tri_t *t = &J->tris[id];
            if (t->cull && !t->amb_cull) continue;
            int ya, yb;
            pix_range(t->ext[1] - 1.0, t->ext[3] + 1.0, H, &ya, &yb);
            if (ya > yb) continue;
            for (int b = ya / BAND; b <= yb / BAND; ++b) cnt[b + 1]++;
        }
        for (int b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
        all = (int *)malloc(sizeof(int) * ((size_t)cnt[nb] + 1));
        int *fill = (int *)calloc((size_t)nb, sizeof(int));
        for (int id = 0; id < J->n; ++id) {
            const tri_t *t = &J->tris[id];
            if (t->cull && !t->amb_cull) continue;
            int ya, yb;
            pix_range(t->ext[1] - 1.0, t->ext[3] + 1.0, H, &ya, &yb);
            if (ya > yb) continue;
            for (int b = ya / BAND; b <= yb / BAND; ++b) all[cnt[b] + fill[b]++] = id;
        }
        free(fill);
    } else {
        all = (int *)malloc(sizeof(int) * ((size_t)J->n + 1));
        for (int id = 0; id < J->n; ++id) all[id] = id;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < nb; ++b) {
        int y0 = b * BAND, y1 = y0 + BAND < H ? y0 + BAND : H;
        if (J->pix_mask) {
            int any = 0;
            for (size_t p = (size_t)y0 * J->C.W; p < (size_t)y1 * J->C.W && !any; ++p) any = J->pix_mask[p];
            if (!any) continue;
        }
        if (J->brute) render_band(J, y0, y1, all, J->n);
        else render_band(J, y0, y1, all + cnt[b], cnt[b + 1] - cnt[b]);
    }
    free(all);
    free(cnt);
}

static tri_t *setup_all(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                        const double *sigma, const cam_t *C, const consts_t *K) {
    tri_t *tris = (tri_t *)malloc(sizeof(tri_t) * (size_t)(n > 0 ? n : 1));
    sh_init();
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int id = 0; id < n; ++id) tri_setup(id, verts, sh, sh_deg, opac, sigma, C, K, &tris[id]);
    return tris;
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                               */
/* ------------------------------------------------------------------ */
int orc_version(void) { return 1; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Forward render. image [3,H,W], T_final [H,W], n_kept [H,W]; flags / err_est nullable.
 * alts (nullable, capacity alt_cap records of {int32 pix, int32 n_kept, double
 * colour[3], double T}): every outcome of each pixel with a decision in the FP32
 * band, listed in any order, their number in *alt_n (which may exceed alt_cap, the
 * excess pixels then carry AMB_UNRES). */
static int render_impl(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                       const double *sigma, const double *cam, const double *consts, int brute,
                       const uint8_t *pix_mask, double *image, double *T_final, int32_t *n_kept,
                       uint8_t *flags, double *err_est, alt_t *alts, size_t alt_cap, size_t *alt_n) {
    if (n < 0 || sh_deg < 0 || sh_deg > 3) return 1;
    if (alts && (!alt_n || !flags)) return 1;
    job_t J;
    memset(&J, 0, sizeof J);
    J.n = n; J.sh_deg = sh_deg; J.nk = (sh_deg + 1) * (sh_deg + 1);
    J.verts = verts; J.sh = sh; J.opac = opac; J.sigma = sigma;
    J.C = load_cam(cam); J.K = load_consts(consts);
    J.brute = brute; J.pix_mask = pix_mask;
    J.image = image; J.T_final = T_final; J.n_kept = n_kept; J.flags = flags; J.err_est = err_est;
    if (alts) { J.alts = alts; J.alt_cap = alt_cap; J.alt_n = alt_n; *alt_n = 0; }
    J.tris = setup_all(n, verts, sh, sh_deg, opac, sigma, &J.C, &J.K);
    run_job(&J);
    free(J.tris);
    return 0;
}

int orc_render(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
               const double *sigma, const double *cam, const double *consts, int brute,
               const uint8_t *pix_mask, double *image, double *T_final, int32_t *n_kept,
               uint8_t *flags, double *err_est) {
    return render_impl(n, verts, sh, sh_deg, opac, sigma, cam, consts, brute, pix_mask, image, T_final, n_kept,
                       flags, err_est, NULL, 0, NULL);
}

int orc_render_alts(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                    const double *sigma, const double *cam, const double *consts, int brute,
                    const uint8_t *pix_mask, double *image, double *T_final, int32_t *n_kept,
                    uint8_t *flags, double *err_est, void *alts, size_t alt_cap, size_t *alt_n) {
    return render_impl(n, verts, sh, sh_deg, opac, sigma, cam, consts, brute, pix_mask, image, T_final, n_kept,
                       flags, err_est, (alt_t *)alts, alt_cap, alt_n);
}

/* Pruning statistics (Sec. 3.3 "Pruning"), per triangle: max_weight = largest T o over
 * its composited fragments (0 if none), n_pix = number of pixels where it was
 * composited, tri_amb = 1 if it took part in a pixel whose result is within the FP32
 * band (flags != 0). Outputs are overwritten. */
int orc_render_stats(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                     const double *sigma, const double *cam, const double *consts, double *max_weight,
                     int32_t *n_pix, uint8_t *tri_amb) {
    if (n < 0 || sh_deg < 0 || sh_deg > 3 || !max_weight || !n_pix || !tri_amb) return 1;
    job_t J;
    memset(&J, 0, sizeof J);
    J.n = n; J.sh_deg = sh_deg; J.nk = (sh_deg + 1) * (sh_deg + 1);
    J.verts = verts; J.sh = sh; J.opac = opac; J.sigma = sigma;
    J.C = load_cam(cam); J.K = load_consts(consts);
    for (int i = 0; i < n; ++i) { max_weight[i] = 0.0; n_pix[i] = 0; tri_amb[i] = 0; }
    J.max_weight = max_weight; J.n_pix = n_pix; J.tri_amb = tri_amb;
    /* flags are needed for tri_amb: a scratch image of flags */
    uint8_t *fl = (uint8_t *)calloc((size_t)J.C.W * J.C.H, 1);
    J.flags = fl;
    J.tris = setup_all(n, verts, sh, sh_deg, opac, sigma, &J.C, &J.K);
    run_job(&J);
    free(J.tris);
    free(fl);
    return 0;
}

/* Solid-triangle render: the limit of the splat render for sigma -> 0 and o = 1
 * (Sec. 5 converts the soup into opaque triangles for game engines): every pixel
 * takes the colour of the nearest triangle, by (centroid depth, id), whose window
 * ratio at the pixel centre is positive, else the background. Opacity and sigma are
 * ignored and only near-plane and degenerate triangles are culled. image [3,H,W],
 * id [H,W] (-1: background). pix_mask (nullable) limits the work to the pixels where
 * it is non-zero; the others get the background and id -1. flags (nullable) marks
 * pixels whose winner is within
 * the FP32 band: a ratio within EPS_LINE of zero for the winner or a nearer
 * triangle, or a depth within 4 FP32 ulps of the winner's. */
int orc_render_solid(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                     const double *sigma, const double *cam, const double *consts, const uint8_t *pix_mask,
                     double *image, int32_t *id_out, uint8_t *flags) {
    if (n < 0 || sh_deg < 0 || sh_deg > 3 || !image || !id_out) return 1;
    cam_t C = load_cam(cam);
    consts_t K = load_consts(consts);
    tri_t *tris = setup_all(n, verts, sh, sh_deg, opac, sigma, &C, &K);
    const int W = C.W, H = C.H;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int y = 0; y < H; ++y) {
        const double py = y + 0.5;
        for (int x = 0; x < W; ++x) {
            const double px = x + 0.5;
            int best = -1;
            double bd = 0.0;
            const size_t pix = (size_t)y * W + x;
            if (pix_mask && !pix_mask[pix]) {          /* not sampled: background, id -1 */
                id_out[pix] = -1;
                for (int c = 0; c < 3; ++c) image[(size_t)c * W * H + pix] = C.bg[c];
                if (flags) flags[pix] = 0;
                continue;
            }
            for (int id = 0; id < n; ++id) {
                const tri_t *t = &tris[id];
                if (t->cull) continue;
                if (px < t->bbox[0] - 1.0 || px > t->bbox[2] + 1.0 || py < t->bbox[1] - 1.0 || py > t->bbox[3] + 1.0)
                    continue;
                if (tri2d_ratio(&t->g, px, py, NULL) <= 0.0) continue;
                if (best < 0 || t->depth < bd || (t->depth == bd && id < best)) { best = id; bd = t->depth; }
            }
            id_out[pix] = best;
            for (int c = 0; c < 3; ++c)
                image[(size_t)c * W * H + pix] = best >= 0 ? tris[best].rgb[c] : C.bg[c];
            if (!flags) continue;
            uint8_t amb = 0;
            for (int id = 0; id < n; ++id) {
                const tri_t *t = &tris[id];
                if (t->cull) {
                    /* a cull within the FP32 band can only change the pixels the
                     * triangle covers: those of its bounding box, when it projects */
                    if (t->amb_cull && t->z[0] > 0 && t->z[1] > 0 && t->z[2] > 0 && px >= t->bbox[0] - 1.0 &&
                        px <= t->bbox[2] + 1.0 && py >= t->bbox[1] - 1.0 && py <= t->bbox[3] + 1.0)
                        amb |= AMB_CULL;
                    continue;
                }
                if (px < t->bbox[0] - 1.0 || px > t->bbox[2] + 1.0 || py < t->bbox[1] - 1.0 || py > t->bbox[3] + 1.0)
                    continue;
                int am;
                const double ratio = tri2d_ratio(&t->g, px, py, &am);
                const int nearer = best < 0 || t->depth < bd || (t->depth == bd && id <= best);
                if (nearer && fabs(ratio) <= ratio_band(&t->g, am, px, py)) amb |= AMB_SKIP;
                if (best >= 0 && id != best && ratio > 0.0 && fabs(t->depth - bd) <= 4.0 * ulp32(bd)) amb |= AMB_ORDER;
            }
            flags[pix] = amb;
        }
    }
    free(tris);
    return 0;
}

/* Adjoint: given dL/dimage [3,H,W], accumulate parameter gradients of the triangles
 * with tri_mask[id] != 0 (all when NULL) from the pixels with pix_mask != 0 (all when
 * NULL). Outputs are overwritten: dverts [n,9], dsh [n,K,3], dopac [n], dsigma [n]. */
int orc_render_grad(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                    const double *sigma, const double *cam, const double *consts,
                    const double *dL_dimage, const uint8_t *pix_mask, const uint8_t *tri_mask,
                    double *dverts, double *dsh, double *dopac, double *dsigma) {
    if (n < 0 || sh_deg < 0 || sh_deg > 3) return 1;
    job_t J;
    memset(&J, 0, sizeof J);
    J.n = n; J.sh_deg = sh_deg; J.nk = (sh_deg + 1) * (sh_deg + 1);
    J.verts = verts; J.sh = sh; J.opac = opac; J.sigma = sigma;
    J.C = load_cam(cam); J.K = load_consts(consts);
    J.brute = 0; J.pix_mask = pix_mask;
    J.dL = dL_dimage;
    J.dverts = dverts; J.dsh = dsh; J.dopac = dopac; J.dsigma = dsigma;
    memset(dverts, 0, sizeof(double) * 9 * (size_t)n);
    memset(dsh, 0, sizeof(double) * 3 * (size_t)J.nk * n);
    memset(dopac, 0, sizeof(double) * (size_t)n);
    memset(dsigma, 0, sizeof(double) * (size_t)n);
    J.tris = setup_all(n, verts, sh, sh_deg, opac, sigma, &J.C, &J.K);
    int32_t *track = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int nt = 0;
    for (int id = 0; id < n; ++id) {
        int want = (!tri_mask || tri_mask[id]) && J.tris[id].cull == CULL_NONE;
        track[id] = want ? nt++ : -1;
    }
    tri_dual_t *duals = (tri_dual_t *)malloc(sizeof(tri_dual_t) * (size_t)(nt > 0 ? nt : 1));
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int id = 0; id < n; ++id)
        if (track[id] >= 0) tri_dual_setup(id, verts, sh, sh_deg, &J.C, &J.tris[id], &duals[track[id]]);
    J.track = track;
    J.duals = duals;
    run_job(&J);
    free(duals);
    free(track);
    free(J.tris);
    return 0;
}

/* Per-triangle quantities.
 * f64 [n, 24]: q (6), z (3), depth, s (2), r, f, rect (4), rgb (3), dir (3)
 * i32 [n, 12]: cull, rect_state, pix (4), tiles (4), amb (bit0 cull band, bit1 rect band), ntiles */
int orc_tri_info(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                 const double *sigma, const double *cam, const double *consts,
                 double *out_f, int32_t *out_i) {
    if (n < 0 || sh_deg < 0 || sh_deg > 3) return 1;
    cam_t C = load_cam(cam);
    consts_t K = load_consts(consts);
    tri_t *tris = setup_all(n, verts, sh, sh_deg, opac, sigma, &C, &K);
    for (int id = 0; id < n; ++id) {
        const tri_t *t = &tris[id];
        double *f = out_f + 24 * (size_t)id;
        int32_t *o = out_i + 12 * (size_t)id;
        for (int i = 0; i < 3; ++i) { f[2 * i] = t->g.q[i][0]; f[2 * i + 1] = t->g.q[i][1]; }
        for (int i = 0; i < 3; ++i) f[6 + i] = t->z[i];
        f[9] = t->depth; f[10] = t->g.s[0]; f[11] = t->g.s[1]; f[12] = t->g.r; f[13] = t->f;
        for (int i = 0; i < 4; ++i) f[14 + i] = t->rect[i];
        for (int i = 0; i < 3; ++i) { f[18 + i] = t->rgb[i]; f[21 + i] = t->dir[i]; }
        o[0] = t->cull; o[1] = t->rect_state;
        for (int i = 0; i < 4; ++i) { o[2 + i] = t->pix[i]; o[6 + i] = t->tiles[i]; }
        o[10] = (t->amb_cull ? 1 : 0) | (t->amb_rect ? 2 : 0);
        o[11] = (t->cull == CULL_NONE && t->rect_state == RECT_OK) ? t->ntiles : 0;
    }
    free(tris);
    return 0;
}

/* 2D triangle geometry. out [15]: n (6), d (3), s (2), r, ell (3) */
int orc_tri2d(const double *q6, double *out) {
    double q[3][2] = {{q6[0], q6[1]}, {q6[2], q6[3]}, {q6[4], q6[5]}};
    tri2d_t T;
    tri2d_setup(q, &T);
    for (int i = 0; i < 3; ++i) { out[2 * i] = T.n[i][0]; out[2 * i + 1] = T.n[i][1]; out[6 + i] = T.d[i]; }
    out[9] = T.s[0]; out[10] = T.s[1]; out[11] = T.r;
    for (int i = 0; i < 3; ++i) out[12 + i] = T.ell[i];
    return 0;
}

/* Window at points: ratio = phi(p)/phi(s), I = ReLU(ratio)^sigma. */
int orc_window(const double *q6, double sigma, int npts, const double *pts, double *ratio, double *I) {
    double q[3][2] = {{q6[0], q6[1]}, {q6[2], q6[3]}, {q6[4], q6[5]}};
    tri2d_t T;
    tri2d_setup(q, &T);
    for (int i = 0; i < npts; ++i) {
        double r = tri2d_ratio(&T, pts[2 * i], pts[2 * i + 1], NULL);
        if (ratio) ratio[i] = r;
        if (I) I[i] = r > 0 ? pow(r, sigma) : 0.0;
    }
    return 0;
}

/* Eq. indicator2: I = sigmoid(-phi(p) / sigma) with phi the signed distance field
 * max_i L_i(p) (pixels); also returns phi. */
int orc_window_sigmoid(const double *q6, double sigma, int npts, const double *pts, double *phi, double *I) {
    double q[3][2] = {{q6[0], q6[1]}, {q6[2], q6[3]}, {q6[4], q6[5]}};
    tri2d_t T;
    tri2d_setup(q, &T);
    for (int i = 0; i < npts; ++i) {
        double ph = -INFINITY;
        for (int k = 0; k < 3; ++k) {
            double L = T.n[k][0] * pts[2 * i] + T.n[k][1] * pts[2 * i + 1] + T.d[k];
            if (L > ph) ph = L;
        }
        if (phi) phi[i] = ph;
        if (I) I[i] = 1.0 / (1.0 + exp(ph / sigma));
    }
    return 0;
}

/* Real SH basis at unit directions: out [ndir, (deg+1)^2]. */
int orc_sh_eval(int deg, int ndir, const double *dirs, double *out) {
    if (deg < 0 || deg > 3) return 1;
    int nk = (deg + 1) * (deg + 1);
    for (int i = 0; i < ndir; ++i) sh_eval_val(deg, dirs + 3 * i, out + (size_t)nk * i);
    return 0;
}
