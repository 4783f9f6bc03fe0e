/*
 * Address / undefined-behaviour sanitizer run of the oracle (TEST INFRASTRUCTURE ONLY):
 * built together with trisplat_oracle.c by tests/test_oracle_sanitize.py with
 * -fsanitize=address,undefined and run on the CPU. It renders a small seeded scene of
 * random triangles (some behind the near plane, some degenerate, some off screen)
 * forward, with flags, alternative outcomes and statistics, and its adjoint, in both compositing orders and
 * both windows, and exits 0; a sanitizer report fails the run.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int orc_render(int n, const double *verts, const double *sh, int sh_deg, const double *opac, const double *sigma,
               const double *cam, const double *consts, int brute, const uint8_t *pix_mask, double *image,
               double *T_final, int32_t *n_kept, uint8_t *flags, double *err_est);
int orc_render_alts(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                    const double *sigma, const double *cam, const double *consts, int brute,
                    const uint8_t *pix_mask, double *image, double *T_final, int32_t *n_kept, uint8_t *flags,
                    double *err_est, void *alts, size_t alt_cap, size_t *alt_n);
int orc_render_grad(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                    const double *sigma, const double *cam, const double *consts, const double *dL_dimage,
                    const uint8_t *pix_mask, const uint8_t *tri_mask, double *dverts, double *dsh, double *dopac,
                    double *dsigma);
int orc_render_stats(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                     const double *sigma, const double *cam, const double *consts, double *max_weight,
                     int32_t *n_pix, uint8_t *amb);
int orc_render_solid(int n, const double *verts, const double *sh, int sh_deg, const double *opac,
                     const double *sigma, const double *cam, const double *consts, const uint8_t *pix_mask,
                     double *image, int32_t *ids, uint8_t *flags);

static uint64_t state = 88172645463325252ull;
static double rnd(void) {   /* xorshift64, uniform [0, 1) */
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return (double)(state >> 11) / 9007199254740992.0;
}

int main(void) {
    enum { N = 60, W = 40, H = 32, DEG = 2, NK = (DEG + 1) * (DEG + 1) };
    static double verts[N * 9], sh[N * NK * 3], opac[N], sigma[N];
    for (int i = 0; i < N; ++i) {
        const double cx = rnd() * 2.4 - 1.2, cy = rnd() * 1.8 - 0.9, cz = (i % 13 == 0) ? 0.1 : 1.5 + 3.0 * rnd();
        const double s = (i % 17 == 0) ? 0.0 : 0.05 + 0.4 * rnd();   /* a few degenerate */
        for (int k = 0; k < 3; ++k) {
            verts[i * 9 + 3 * k] = cx + s * (rnd() - 0.5);
            verts[i * 9 + 3 * k + 1] = cy + s * (rnd() - 0.5);
            verts[i * 9 + 3 * k + 2] = cz + 0.2 * s * (rnd() - 0.5);
        }
        for (int k = 0; k < NK * 3; ++k) sh[i * NK * 3 + k] = 0.3 * (rnd() - 0.5);
        opac[i] = 0.02 + 0.9 * rnd();
        sigma[i] = 0.3 + 2.5 * rnd();
    }
    double cam[21] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 36.0, 36.0, W / 2.0, H / 2.0, W, H, 0.1, 0.2, 0.3};
    static double image[3 * W * H], T[W * H], err[W * H], dL[3 * W * H];
    static int32_t n_kept[W * H], ids[W * H], n_pix[N];
    static uint8_t flags[W * H], amb[N];
    static double dverts[N * 9], dsh[N * NK * 3], dopac[N], dsigma[N], mw[N];
    static double alts[5 * 256];   /* 256 outcome records of 40 bytes */
    for (int k = 0; k < 3 * W * H; ++k) dL[k] = rnd() - 0.5;
    int rc = 0;
    for (int window = 0; window < 2; ++window)
        for (int sort = 0; sort < 2; ++sort) {
            double consts[9] = {0.99, 1.0 / 255.0, 1e-4, 0.2, 1e-4, 16, 1.0 / 512.0, (double)window, (double)sort};
            rc |= orc_render(N, verts, sh, DEG, opac, sigma, cam, consts, 0, NULL, image, T, n_kept, flags, err);
            rc |= orc_render(N, verts, sh, DEG, opac, sigma, cam, consts, 1, NULL, image, T, n_kept, flags, err);
            /* alternative outcomes, with a list too small for them all */
            size_t nalt = 0;
            rc |= orc_render_alts(N, verts, sh, DEG, opac, sigma, cam, consts, 0, NULL, image, T, n_kept, flags, err,
                                  alts, sizeof alts / 40, &nalt);
            rc |= orc_render_alts(N, verts, sh, DEG, opac, sigma, cam, consts, 0, NULL, image, T, n_kept, flags, err,
                                  alts, 1, &nalt);
            rc |= orc_render_grad(N, verts, sh, DEG, opac, sigma, cam, consts, dL, NULL, NULL, dverts, dsh, dopac,
                                  dsigma);
            if (window == 0 && sort == 0) {
                rc |= orc_render_stats(N, verts, sh, DEG, opac, sigma, cam, consts, mw, n_pix, amb);
                rc |= orc_render_solid(N, verts, sh, DEG, opac, sigma, cam, consts, NULL, image, ids, flags);
            }
        }
    printf("sanitize check rc=%d\n", rc);
    return rc;
}
