/*
 * fse_oracle.c -- plain FP64 CPU oracle for Frequency Selective Extrapolation
 * (FSE) block-loss concealment with the line-scan or the optimized
 * processing order of Seiler & Kaup, "Optimized and Parallelized Processing
 * Order for Improved Frequency Selective Signal Extrapolation".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  It is linked by the tests, by
 * the smoke check and by the CPU-baseline leg of the benchmark, never by the
 * product library, and it shares no code, header or table with the GPU path.
 *
 * Everything is double precision.  Loops follow the definitions directly:
 *   - processing order: Algorithm 1 (Sec. 3) and the line-scan order (Sec. 2);
 *   - extrapolation area L and its sub-areas A, R, B_i, B_o (Sec. 2, Fig. 1);
 *   - weighting function, Eq. (2);
 *   - model g = sum_k c_k phi_k, Eq. (1), with 2-D DFT basis functions
 *     (Sec. 4) phi_k[m,n] = exp(+j 2 pi (k_m m + k_n n) / F);
 *   - per iteration: select the basis function with the largest decrease of
 *     the weighted residual energy, add gamma times its projection
 *     coefficient (orthogonality deficiency compensation, Sec. 4), and update
 *     the weighted residual spectrum (transform-domain form, Sec. 4).
 *
 * Readings of points the paper leaves open (each one is listed with its
 * justification in the design notes of the repository):
 *   - the weighted residual energy is E = sum w |f - g|^2; adding
 *     gamma * p * phi_u with p = R_w[u] / W[0] lowers E by
 *     (2 gamma - gamma^2) |R_w[u]|^2 / W[0], so the selected index is the
 *     argmax of |R_w[k]|^2; ties go to the smallest linear index
 *     kappa = F * k_m + k_n (or to the largest, for the symmetry test);
 *   - the residual update R_w[k] -= dc * W[(k - u) mod F] is the DFT of
 *     w * (r - dc * phi_u), exact because phi is F-periodic;
 *   - the extrapolated value is the real part of the model, clamped to
 *     [0, 255]; later blocks read the clamped unrounded value, the final
 *     8-bit output is rounded half to even;
 *   - N_min of Eq. (3) is the minimum over blocks with N >= 0;
 *     neighbours are the 8-neighbourhood (consistent with the +3 margin /
 *     +5 corner penalties); the set S is built by a raster scan;
 *   - blocks of one group read the frame as of the start of the group;
 *   - an area without any support sample (W[0] = 0) yields the zero model.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "fse_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Processing order: line scan (Sec. 2) and Algorithm 1 (Sec. 3).            */
/* ------------------------------------------------------------------------ */

static int is_corner(int by, int bx, int bh, int bw)
{
    int row_edge = (by == 0) || (by == bh - 1);
    int col_edge = (bx == 0) || (bx == bw - 1);
    return row_edge && col_edge;
}

static int is_margin(int by, int bx, int bh, int bw)
{
    int edge = (by == 0) || (by == bh - 1) || (bx == 0) || (bx == bw - 1);
    return edge && !is_corner(by, bx, bh, bw);
}

int oracle_plan(int bw, int bh, const uint8_t *lost, int order,
                int32_t *group_of_block, int32_t *group_ptr,
                int32_t *block_ids, int32_t *n_groups)
{
    if (bw <= 0 || bh <= 0 || !lost || !group_of_block || !group_ptr ||
        !block_ids || !n_groups)
        return -1;
    const int nb = bw * bh;
    for (int b = 0; b < nb; ++b)
        group_of_block[b] = -1;

    if (order == 0) {
        /* Line scan: every lost block alone, in raster order. */
        int g = 0;
        group_ptr[0] = 0;
        for (int b = 0; b < nb; ++b) {
            if (!lost[b])
                continue;
            group_of_block[b] = g;
            block_ids[g] = b;
            group_ptr[g + 1] = g + 1;
            ++g;
        }
        *n_groups = g;
        return 0;
    }
    if (order != 1)
        return -1;

    /* Algorithm 1, initialisation: N(b) counts the lost 8-neighbours, plus
     * 5 for a corner block or 3 for a margin block; blocks without loss get
     * N = -1. */
    int *N = (int *)calloc((size_t)nb, sizeof(int));
    uint8_t *in_s = (uint8_t *)calloc((size_t)nb, 1);
    if (!N || !in_s) {
        free(N);
        free(in_s);
        return -2;
    }
    for (int by = 0; by < bh; ++by) {
        for (int bx = 0; bx < bw; ++bx) {
            int b = by * bw + bx;
            if (lost[b]) {
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dy == 0 && dx == 0)
                            continue;
                        int ny = by + dy, nx = bx + dx;
                        if (ny < 0 || ny >= bh || nx < 0 || nx >= bw)
                            continue;
                        N[ny * bw + nx] += 1;
                    }
            }
            if (is_margin(by, bx, bh, bw))
                N[b] += 3;
            if (is_corner(by, bx, bh, bw))
                N[b] += 5;
        }
    }
    for (int b = 0; b < nb; ++b)
        if (!lost[b])
            N[b] = -1;

    /* Algorithm 1, extrapolation loop. */
    int ng = 0, pos = 0;
    group_ptr[0] = 0;
    for (;;) {
        int nmin = -1;
        for (int b = 0; b < nb; ++b)
            if (N[b] >= 0 && (nmin < 0 || N[b] < nmin))
                nmin = N[b];
        if (nmin < 0)
            break; /* N(b) < 0 for all blocks: finished */

        memset(in_s, 0, (size_t)nb);
        int start = pos;
        for (int by = 0; by < bh; ++by) {
            for (int bx = 0; bx < bw; ++bx) {
                int b = by * bw + bx;
                if (N[b] != nmin)
                    continue;
                int blocked = 0;
                for (int dy = -1; dy <= 1 && !blocked; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dy == 0 && dx == 0)
                            continue;
                        int ny = by + dy, nx = bx + dx;
                        if (ny < 0 || ny >= bh || nx < 0 || nx >= bw)
                            continue;
                        if (in_s[ny * bw + nx]) {
                            blocked = 1;
                            break;
                        }
                    }
                if (blocked)
                    continue;
                in_s[b] = 1;
                block_ids[pos++] = b;
                group_of_block[b] = ng;
            }
        }
        /* After extrapolation of S: N(b) = -1, and every neighbour that is
         * still pending loses one not-extrapolated neighbour. */
        for (int i = start; i < pos; ++i) {
            int b = block_ids[i];
            int by = b / bw, bx = b % bw;
            N[b] = -1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dy == 0 && dx == 0)
                        continue;
                    int ny = by + dy, nx = bx + dx;
                    if (ny < 0 || ny >= bh || nx < 0 || nx >= bw)
                        continue;
                    if (N[ny * bw + nx] >= 0)
                        N[ny * bw + nx] -= 1;
                }
        }
        ++ng;
        group_ptr[ng] = pos;
    }
    *n_groups = ng;
    free(N);
    free(in_s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FSE for one extrapolation area (Sec. 2, Eq. (1), Eq. (2)).                */
/* ------------------------------------------------------------------------ */

/* cos / sin of 2 pi t / F for t in [0, F).  Values for t > F/2 are the
 * mirror of t' = F - t (cos even, sin odd), so that a real input has an
 * exactly conjugate-symmetric spectrum; mathematically zero entries are
 * stored as exact zeros. */
static void twiddle_table(int F, double *c, double *s)
{
    for (int t = 0; t <= F / 2; ++t) {
        c[t] = cos(2.0 * M_PI * (double)t / (double)F);
        s[t] = sin(2.0 * M_PI * (double)t / (double)F);
        if (4 * t == F)
            c[t] = 0.0;
        if (t == 0 || 2 * t == F)
            s[t] = 0.0;
    }
    for (int t = F / 2 + 1; t < F; ++t) {
        c[t] = c[F - t];
        s[t] = -s[F - t];
    }
}

/* Eq. (2): rho^dist for A, delta * rho^dist for R, 0 for B_i, B_o and
 * samples outside the image; dist is measured from ((M-1)/2, (N-1)/2). */
void oracle_weights(int M, int N, const uint8_t *cls, double rho, double delta,
                    double *w)
{
    const double cm = 0.5 * (double)(M - 1), cn = 0.5 * (double)(N - 1);
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            double dm = (double)m - cm, dn = (double)n - cn;
            double dist = sqrt(dm * dm + dn * dn);
            double v;
            switch (cls[m * N + n]) {
            case ORACLE_CLS_A:
                v = pow(rho, dist);
                break;
            case ORACLE_CLS_R:
                v = delta * pow(rho, dist);
                break;
            default:
                v = 0.0;
                break;
            }
            w[m * N + n] = v;
        }
}

/* 2-D DFT of an M x N real array zero-extended to F x F:
 * X[k_m, k_n] = sum_m sum_n x[m,n] exp(-j 2 pi (k_m m + k_n n) / F),
 * summed along n first, then along m (the exponential factorises).
 * Output interleaved (re, im), row-major in (k_m, k_n). */
static void dft2_real(int M, int N, int F, const double *x, const double *c,
                      const double *s, double *X)
{
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)M * (size_t)F);
    for (int m = 0; m < M; ++m)
        for (int kn = 0; kn < F; ++kn) {
            double re = 0.0, im = 0.0;
            for (int n = 0; n < N; ++n) {
                int t = (int)(((long)kn * n) % F);
                re += x[m * N + n] * c[t];
                im -= x[m * N + n] * s[t];
            }
            Y[2 * ((size_t)m * F + kn)] = re;
            Y[2 * ((size_t)m * F + kn) + 1] = im;
        }
    for (int km = 0; km < F; ++km)
        for (int kn = 0; kn < F; ++kn) {
            double re = 0.0, im = 0.0;
            for (int m = 0; m < M; ++m) {
                int t = (int)(((long)km * m) % F);
                double yr = Y[2 * ((size_t)m * F + kn)];
                double yi = Y[2 * ((size_t)m * F + kn) + 1];
                /* (c - j s) * (yr + j yi) */
                re += c[t] * yr + s[t] * yi;
                im += c[t] * yi - s[t] * yr;
            }
            X[2 * ((size_t)km * F + kn)] = re;
            X[2 * ((size_t)km * F + kn) + 1] = im;
        }
    free(Y);
}

int oracle_extrapolate_area(int M, int N, int F, const double *f,
                            const uint8_t *cls, double rho, double delta,
                            double gamma, int K, int tie_largest,
                            const uint8_t *want_g, double *g_out,
                            double *w_out, double *R0_out, double *W_out,
                            int32_t *u_out, double *dc_out, double *R_out,
                            double *coef_out, double *margin_out)
{
    if (M <= 0 || N <= 0 || F <= 0 || M > F || N > F || K < 0 || !f || !cls)
        return -1;
    const size_t FF = (size_t)F * (size_t)F;
    double *c = (double *)malloc(sizeof(double) * (size_t)F);
    double *s = (double *)malloc(sizeof(double) * (size_t)F);
    double *w = (double *)malloc(sizeof(double) * (size_t)M * N);
    double *x = (double *)malloc(sizeof(double) * (size_t)M * N);
    double *R = (double *)malloc(sizeof(double) * 2 * FF);
    double *W = (double *)malloc(sizeof(double) * 2 * FF);
    double *coef = (double *)calloc(2 * FF, sizeof(double));
    if (!c || !s || !w || !x || !R || !W || !coef) {
        free(c); free(s); free(w); free(x); free(R); free(W); free(coef);
        return -2;
    }
    twiddle_table(F, c, s);
    oracle_weights(M, N, cls, rho, delta, w);

    /* Weighted signal: samples with zero weight do not contribute. */
    for (int i = 0; i < M * N; ++i)
        x[i] = (w[i] != 0.0) ? w[i] * f[i] : 0.0;

    /* Initial weighted residual spectrum (the model starts at g = 0) and
     * the spectrum of the weighting function. */
    dft2_real(M, N, F, x, c, s, R);
    dft2_real(M, N, F, w, c, s, W);
    if (R0_out)
        memcpy(R0_out, R, sizeof(double) * 2 * FF);
    if (W_out)
        memcpy(W_out, W, sizeof(double) * 2 * FF);
    if (w_out)
        memcpy(w_out, w, sizeof(double) * (size_t)M * N);

    /* W[0] = sum of the weights; every basis function has weighted energy
     * sum w |phi_k|^2 = W[0]. */
    const double W0 = W[0];
    /* Scale of the selection margins: sum |w f| + W[0] * sum |dc| so far. */
    double scale = 0.0;
    for (int i = 0; i < M * N; ++i)
        scale += fabs(x[i]);

    for (int it = 0; it < K; ++it) {
        if (!(W0 > 0.0)) {
            if (u_out) u_out[it] = -1;
            if (dc_out) { dc_out[2 * it] = 0.0; dc_out[2 * it + 1] = 0.0; }
            if (margin_out) margin_out[it] = HUGE_VAL;
            continue;
        }
        /* Selection: largest decrease of the weighted residual energy,
         * i.e. largest |R_w[k]|^2. */
        size_t u = 0;
        double best = -1.0;
        for (size_t k = 0; k < FF; ++k) {
            double e = R[2 * k] * R[2 * k] + R[2 * k + 1] * R[2 * k + 1];
            if (e > best || (tie_largest && e == best)) {
                best = e;
                u = k;
            }
        }
        /* Margin of the choice: |R_w[u]| minus the largest magnitude among
         * the other entries, in units of the scale above.  A small margin is
         * a near-tie that a lower precision may resolve the other way.  An
         * exact tie counts as margin 0 (a lower precision rounds the tied
         * magnitudes apart), except an exact tie with the conjugate partner
         * R_w[-u]: R_w[-u] = conj R_w[u] holds in any precision that keeps
         * a real input's symmetry, and the index rule then decides alike. */
        if (margin_out) {
            const size_t um = u / (size_t)F, un = u % (size_t)F;
            const size_t up = ((F - um) % F) * (size_t)F + (F - un) % F;
            double second = -1.0;
            for (size_t k = 0; k < FF; ++k) {
                if (k == u)
                    continue;
                double e = R[2 * k] * R[2 * k] + R[2 * k + 1] * R[2 * k + 1];
                if (k == up && e == best)
                    continue;
                if (e > second)
                    second = e;
            }
            margin_out[it] = (second < 0.0 || !(scale > 0.0))
                                 ? HUGE_VAL
                                 : (sqrt(best) - sqrt(second)) / scale;
        }
        /* Orthogonality deficiency compensation: add gamma times the
         * projection coefficient R_w[u] / W[0]. */
        const double dcr = gamma * R[2 * u] / W0;
        const double dci = gamma * R[2 * u + 1] / W0;
        coef[2 * u] += dcr;
        coef[2 * u + 1] += dci;
        if (u_out) u_out[it] = (int32_t)u;
        if (dc_out) { dc_out[2 * it] = dcr; dc_out[2 * it + 1] = dci; }
        scale += W0 * sqrt(dcr * dcr + dci * dci);

        /* Weighted residual update in the transform domain:
         * R_w[k] -= dc * W[(k - u) mod F] for every k. */
        const int um = (int)(u / (size_t)F), un = (int)(u % (size_t)F);
        for (int km = 0; km < F; ++km) {
            int sm = (km - um + F) % F;
            for (int kn = 0; kn < F; ++kn) {
                int sn = (kn - un + F) % F;
                size_t k = (size_t)km * F + kn;
                size_t j = (size_t)sm * F + sn;
                double wr = W[2 * j], wi = W[2 * j + 1];
                R[2 * k] -= dcr * wr - dci * wi;
                R[2 * k + 1] -= dcr * wi + dci * wr;
            }
        }
    }
    if (R_out)
        memcpy(R_out, R, sizeof(double) * 2 * FF);
    if (coef_out)
        memcpy(coef_out, coef, sizeof(double) * 2 * FF);

    /* Eq. (1), real part: g[m,n] = Re sum_k c_k exp(+j 2 pi (k_m m + k_n n)/F).
     * Terms with c_k = 0 add nothing and are skipped. */
    if (g_out) {
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                if (want_g && !want_g[m * N + n])
                    continue;
                double acc = 0.0;
                for (size_t k = 0; k < FF; ++k) {
                    double cr = coef[2 * k], ci = coef[2 * k + 1];
                    if (cr == 0.0 && ci == 0.0)
                        continue;
                    int km = (int)(k / (size_t)F), kn = (int)(k % (size_t)F);
                    int t = (int)(((long)km * m + (long)kn * n) % F);
                    acc += cr * c[t] - ci * s[t];
                }
                g_out[m * N + n] = acc;
            }
    }
    free(c); free(s); free(w); free(x); free(R); free(W); free(coef);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole frame: schedule, then per group the extrapolation of every block    */
/* of the group from the frame state at the start of the group (Alg. 1).     */
/* ------------------------------------------------------------------------ */

int oracle_conceal_frame(int H, int Wd, const uint8_t *img,
                         const uint8_t *mask, int B, int d, int F, int K,
                         double rho, double delta, double gamma, int order,
                         int threads, double *work, uint8_t *out,
                         int32_t *group_of_block_out, int32_t *u_trace)
{
    return oracle_conceal_frame_ex(H, Wd, img, mask, B, d, F, K, rho, delta,
                                   gamma, order, threads, work, out,
                                   group_of_block_out, u_trace, NULL, NULL);
}

int oracle_conceal_frame_ex(int H, int Wd, const uint8_t *img,
                            const uint8_t *mask, int B, int d, int F, int K,
                            double rho, double delta, double gamma, int order,
                            int threads, double *work, uint8_t *out,
                            int32_t *group_of_block_out, int32_t *u_trace,
                            uint8_t *cls_trace, double *margin_trace)
{
    if (H <= 0 || Wd <= 0 || B <= 0 || d < 0 || !img || !mask || !work || !out)
        return -1;
    const int M = B + 2 * d;
    if (M > F)
        return -1;
    const int bh = (H + B - 1) / B, bw = (Wd + B - 1) / B, nb = bh * bw;

    uint8_t *lost = (uint8_t *)calloc((size_t)nb, 1);
    uint8_t *done = (uint8_t *)calloc((size_t)nb, 1);
    int32_t *gob = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *gptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nb + 1));
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
    if (!lost || !done || !gob || !gptr || !ids) {
        free(lost); free(done); free(gob); free(gptr); free(ids);
        return -2;
    }
    /* A block is lost when any of its in-image samples is lost. */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < Wd; ++x)
            if (mask[(size_t)y * Wd + x])
                lost[(y / B) * bw + (x / B)] = 1;
    int32_t ng = 0;
    int rc = oracle_plan(bw, bh, lost, order, gob, gptr, ids, &ng);
    if (rc) {
        free(lost); free(done); free(gob); free(gptr); free(ids);
        return rc;
    }
    if (group_of_block_out)
        memcpy(group_of_block_out, gob, sizeof(int32_t) * (size_t)nb);

    for (size_t i = 0; i < (size_t)H * Wd; ++i)
        work[i] = mask[i] ? 0.0 : (double)img[i];

    for (int g = 0; g < ng; ++g) {
        const int first = gptr[g], count = gptr[g + 1] - gptr[g];
        double *stage = (double *)malloc(sizeof(double) * (size_t)count * B * B);
        int err = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1) reduction(| : err)
#endif
        for (int i = 0; i < count; ++i) {
            const int b = ids[first + i];
            const int by = b / bw, bx = b % bw;
            const int y0 = by * B - d, x0 = bx * B - d;
            double *f = (double *)malloc(sizeof(double) * (size_t)M * M);
            uint8_t *cls = (uint8_t *)malloc((size_t)M * M);
            uint8_t *want = (uint8_t *)calloc((size_t)M * M, 1);
            double *gv = (double *)calloc((size_t)M * M, sizeof(double));
            /* Sub-areas of L (Sec. 2, Fig. 1). */
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < M; ++n) {
                    int y = y0 + m, x = x0 + n;
                    int idx = m * M + n;
                    f[idx] = 0.0;
                    if (y < 0 || y >= H || x < 0 || x >= Wd) {
                        cls[idx] = ORACLE_CLS_OUT;
                        continue;
                    }
                    size_t p = (size_t)y * Wd + x;
                    int pb = (y / B) * bw + (x / B);
                    if (!mask[p]) {
                        cls[idx] = ORACLE_CLS_A;
                        f[idx] = work[p];
                    } else if (pb == b) {
                        cls[idx] = ORACLE_CLS_BI;
                        want[idx] = 1;
                    } else if (done[pb]) {
                        cls[idx] = ORACLE_CLS_R;
                        f[idx] = work[p];
                    } else {
                        cls[idx] = ORACLE_CLS_BO;
                    }
                }
            int32_t *ut = u_trace ? u_trace + (size_t)b * (size_t)K : NULL;
            double *mt = margin_trace ? margin_trace + (size_t)b * (size_t)K : NULL;
            if (cls_trace)
                memcpy(cls_trace + (size_t)b * M * M, cls, (size_t)M * M);
            int r = oracle_extrapolate_area(M, M, F, f, cls, rho, delta, gamma, K,
                                            0, want, gv, NULL, NULL, NULL, ut,
                                            NULL, NULL, NULL, mt);
            if (r)
                err |= 1;
            /* Insert the model samples of B_i, clamped to the 8-bit range. */
            for (int m = 0; m < B; ++m)
                for (int n = 0; n < B; ++n) {
                    double v = gv[(m + d) * M + (n + d)];
                    if (v < 0.0) v = 0.0;
                    if (v > 255.0) v = 255.0;
                    stage[(size_t)i * B * B + m * B + n] = v;
                }
            free(f); free(cls); free(want); free(gv);
        }
        /* Commit the group: all its blocks read the pre-group state. */
        for (int i = 0; i < count; ++i) {
            const int b = ids[first + i];
            const int by = b / bw, bx = b % bw;
            for (int m = 0; m < B; ++m)
                for (int n = 0; n < B; ++n) {
                    int y = by * B + m, x = bx * B + n;
                    if (y >= H || x >= Wd)
                        continue;
                    size_t p = (size_t)y * Wd + x;
                    if (mask[p])
                        work[p] = stage[(size_t)i * B * B + m * B + n];
                }
            done[b] = 1;
        }
        free(stage);
        if (err) {
            free(lost); free(done); free(gob); free(gptr); free(ids);
            return -3;
        }
    }

    for (size_t i = 0; i < (size_t)H * Wd; ++i)
        out[i] = mask[i] ? (uint8_t)rint(work[i]) : img[i];

    free(lost); free(done); free(gob); free(gptr); free(ids);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
