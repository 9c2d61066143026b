/*
 * FP64 CPU oracle for the non-gridding MEM measurement operator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the CUDA library computes.  It shares no code with the
 * library; only tests, the smoke check and the benchmark's CPU baseline load it.
 *
 * Operator (Eq. 1 discretised on the regular pixel grid, Section 2 "Data
 * description"; pixel coordinates as in the gradient kernel of Section 2.5:
 * x = (j - x_c) dx, y = (i - y_c) dy with the centre pixel x_c = y_c = N/2):
 *
 *   forward:  V_k = sum_{n,m} B[n][m] exp(-2 pi i (u_k x_m + v_k y_n)),  B = A * I
 *   adjoint:  G[n][m] = sum_k Re( y_k exp(+2 pi i (u_k x_m + v_k y_n)) )
 *
 * With y_k = w_k r_k (w = 1/sigma^2, r = V^m - V^o) the adjoint times A is the
 * chi^2 gradient of Eq. (chi2gradient) / Appendix C, with the primary-beam
 * factor of the model kept (the derivative of V^m with respect to I_l carries
 * A_l).
 *
 * Two evaluation orders are given for each operator:
 *   *_direct   : one complex exponential per (visibility, pixel) pair, the sum
 *                written exactly as above;
 *   *_factored : exp(-2 pi i (u x + v y)) = exp(-2 pi i u x) exp(-2 pi i v y)
 *                (exact identity on the grid), row sums first.  Used where the
 *                direct order is too slow; tests pin it to the direct order.
 * Phases are reduced modulo one turn in FP64 before the trigonometric call.
 * OpenMP parallelises over independent outputs only; every individual sum is
 * accumulated serially in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static inline void turn_cis(double turns, double *c, double *s)
{
    double t = turns - nearbyint(turns);  /* in [-0.5, 0.5] */
    *c = cos(2.0 * M_PI * t);
    *s = sin(2.0 * M_PI * t);
}

static inline double coord(int idx, int N, double d) { return (double)(idx - N / 2) * d; }

/* V: 2*Z doubles (re, im).  B: N*N row-major [n][m]. */
void orc_forward_direct(int N, double dx, double dy, int64_t Z, const double *u,
                        const double *v, const double *B, double *V)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < Z; ++k) {
        double re = 0.0, im = 0.0;
        for (int n = 0; n < N; ++n) {
            double yn = coord(n, N, dy);
            for (int m = 0; m < N; ++m) {
                double xm = coord(m, N, dx);
                double c, s;
                turn_cis(u[k] * xm + v[k] * yn, &c, &s);
                double b = B[(int64_t)n * N + m];
                re += b * c;       /* exp(-i a) = cos a - i sin a */
                im -= b * s;
            }
        }
        V[2 * k] = re;
        V[2 * k + 1] = im;
    }
}

void orc_forward_factored(int N, double dx, double dy, int64_t Z, const double *u,
                          const double *v, const double *B, double *V)
{
#pragma omp parallel
    {
        double *ex = (double *)malloc(sizeof(double) * 2 * N);
        double *ey = (double *)malloc(sizeof(double) * 2 * N);
#pragma omp for schedule(static)
        for (int64_t k = 0; k < Z; ++k) {
            for (int m = 0; m < N; ++m) {
                double c, s;
                turn_cis(u[k] * coord(m, N, dx), &c, &s);
                ex[2 * m] = c; ex[2 * m + 1] = -s;
            }
            for (int n = 0; n < N; ++n) {
                double c, s;
                turn_cis(v[k] * coord(n, N, dy), &c, &s);
                ey[2 * n] = c; ey[2 * n + 1] = -s;
            }
            double re = 0.0, im = 0.0;
            for (int n = 0; n < N; ++n) {
                /* row sum t_n = sum_m B[n][m] ex_m */
                double tr = 0.0, ti = 0.0;
                for (int m = 0; m < N; ++m) {
                    double b = B[(int64_t)n * N + m];
                    tr += b * ex[2 * m];
                    ti += b * ex[2 * m + 1];
                }
                re += ey[2 * n] * tr - ey[2 * n + 1] * ti;
                im += ey[2 * n] * ti + ey[2 * n + 1] * tr;
            }
            V[2 * k] = re;
            V[2 * k + 1] = im;
        }
        free(ex);
        free(ey);
    }
}

/* G: nn*nm doubles for the crop rows [n0, n0+nn), columns [m0, m0+nm).
 * y: 2*Z doubles (re, im). */
void orc_adjoint_direct(int N, double dx, double dy, int64_t Z, const double *u,
                        const double *v, const double *y, int n0, int nn, int m0,
                        int nm, double *G)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < nn; ++a) {
        for (int b = 0; b < nm; ++b) {
            double yn = coord(n0 + a, N, dy);
            double xm = coord(m0 + b, N, dx);
            double acc = 0.0;
            for (int64_t k = 0; k < Z; ++k) {
                double c, s;
                turn_cis(u[k] * xm + v[k] * yn, &c, &s);
                /* Re((yr + i yi)(c + i s)) */
                acc += y[2 * k] * c - y[2 * k + 1] * s;
            }
            G[(int64_t)a * nm + b] = acc;
        }
    }
}

void orc_adjoint_factored(int N, double dx, double dy, int64_t Z, const double *u,
                          const double *v, const double *y, int n0, int nn, int m0,
                          int nm, double *G)
{
    /* Per output pixel the sum over k runs in index order, as in the direct
     * form; the exponential is the product of its two separable factors. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < nn; ++a) {
        for (int b = 0; b < nm; ++b) {
            double yn = coord(n0 + a, N, dy);
            double xm = coord(m0 + b, N, dx);
            double acc = 0.0;
            for (int64_t k = 0; k < Z; ++k) {
                double cx, sx, cy, sy;
                turn_cis(u[k] * xm, &cx, &sx);
                turn_cis(v[k] * yn, &cy, &sy);
                double c = cx * cy - sx * sy;   /* cos(ax + ay) */
                double s = sx * cy + cx * sy;   /* sin(ax + ay) */
                acc += y[2 * k] * c - y[2 * k + 1] * s;
            }
            G[(int64_t)a * nm + b] = acc;
        }
    }
}

/* Full-image adjoint in the factored order: for each image row n the terms
 * are added to G[n][m] for k = 0, 1, ..., Z-1 in index order, with
 * Re(y_k e^{+i(ax+ay)}) = cos(ax) Re(p) - sin(ax) Im(p),  p = y_k e^{+i ay}.
 * Parallel over image rows only. */
void orc_adjoint_factored_full(int N, double dx, double dy, int64_t Z, const double *u,
                               const double *v, const double *y, double *G)
{
    double *ex = (double *)malloc(sizeof(double) * 2 * (size_t)N * (size_t)Z);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < Z; ++k) {
        for (int m = 0; m < N; ++m) {
            double c, s;
            turn_cis(u[k] * coord(m, N, dx), &c, &s);
            ex[(2 * k) * N + 2 * m] = c;
            ex[(2 * k) * N + 2 * m + 1] = s;
        }
    }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; ++n) {
        double *row = G + (int64_t)n * N;
        double yn = coord(n, N, dy);
        for (int m = 0; m < N; ++m) row[m] = 0.0;
        for (int64_t k = 0; k < Z; ++k) {
            double cy, sy;
            turn_cis(v[k] * yn, &cy, &sy);
            double pr = y[2 * k] * cy - y[2 * k + 1] * sy;
            double pi = y[2 * k] * sy + y[2 * k + 1] * cy;
            const double *e = ex + (2 * k) * N;
            for (int m = 0; m < N; ++m) row[m] += e[2 * m] * pr - e[2 * m + 1] * pi;
        }
    }
    free(ex);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by the following calls (n >= 1); for timing the oracle on one
 * core beside all of them.  The sums do not depend on it: every output is
 * summed by one thread in index order. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
