/*
 * Oracle: the exact solution of the discrete homogeneous diffusion inpainting
 * problem, by FP64 conjugate gradients on the reduced system.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (Section 2.2, eq. (2.6) and the "Practical Considerations"
 * paragraph): the solution u of (C + (I - C) L) u = C f per channel, where c is
 * the binary mask, L the 5-point negated Laplacian with reflecting boundaries
 * and h = 1:  L_ii = |N(i)|, L_ij = -1 for the in-image 4-neighbours j of i.
 * Removing the mask pixels (where u = f) leaves, for every unknown pixel i,
 *     |N(i)| u_i - sum_{j in N(i), c_j = 0} u_j = sum_{j in N(i), c_j = 1} f_j,
 * a symmetric positive definite system (Section 2.2), solved here by
 * Jacobi-preconditioned CG (Hestenes-Stiefel) from u = 0 until
 * ||r||_2 <= rel_tol * ||b_red||_2.  Channels are independent and run one
 * after another; each matrix-vector product and dot product is split over
 * rows with OpenMP.
 *
 * Values of f at unknown pixels are never read into the arithmetic (they may
 * be NaN or Inf).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_INVALID 1
#define ORACLE_EMPTY_MASK 2
#define ORACLE_OOM 3
#define ORACLE_NOT_CONVERGED 4

/* y = A_red x on unknown pixels (0 on mask pixels). */
static void apply_reduced(const uint8_t *c, int W, int H, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int yy = 0; yy < H; ++yy) {
        for (int xx = 0; xx < W; ++xx) {
            size_t i = (size_t)yy * W + xx;
            if (c[i]) { y[i] = 0.0; continue; }
            double acc = 0.0;
            int deg = 0;
            if (xx > 0)     { ++deg; if (!c[i - 1]) acc -= x[i - 1]; }
            if (xx < W - 1) { ++deg; if (!c[i + 1]) acc -= x[i + 1]; }
            if (yy > 0)     { ++deg; if (!c[i - W]) acc -= x[i - W]; }
            if (yy < H - 1) { ++deg; if (!c[i + W]) acc -= x[i + W]; }
            y[i] = (double)deg * x[i] + acc;
        }
    }
}

static double dot(const double *a, const double *b, size_t n)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static int degree(int xx, int yy, int W, int H)
{
    return (xx > 0) + (xx < W - 1) + (yy > 0) + (yy < H - 1);
}

/*
 * f: float32 planar [C][H][W]; c: uint8 [H][W] (nonzero = known);
 * u: float64 planar [C][H][W] output.  iters / relres (may be NULL): per
 * channel CG iteration counts and final relative residuals.
 * Returns ORACLE_* codes.  A 1x1 ... WxH image with at least one mask pixel is
 * valid.  A degree-0 pixel (1x1 image) is necessarily a mask pixel.
 */
int oracle_cg_inpaint(const float *f, const uint8_t *c, int W, int H, int C,
                      double rel_tol, int max_iter, double *u, int *iters,
                      double *relres)
{
    if (!f || !c || !u || W < 1 || H < 1 || C < 1 || !(rel_tol > 0.0) || max_iter < 0)
        return ORACLE_INVALID;
    size_t n = (size_t)W * H;
    size_t nmask = 0;
    for (size_t i = 0; i < n; ++i) nmask += c[i] != 0;
    if (nmask == 0) return ORACLE_EMPTY_MASK;

    double *b = malloc(n * sizeof(double));
    double *x = malloc(n * sizeof(double));
    double *r = malloc(n * sizeof(double));
    double *z = malloc(n * sizeof(double));
    double *p = malloc(n * sizeof(double));
    double *q = malloc(n * sizeof(double));
    double *dinv = malloc(n * sizeof(double));
    if (!b || !x || !r || !z || !p || !q || !dinv) {
        free(b); free(x); free(r); free(z); free(p); free(q); free(dinv);
        return ORACLE_OOM;
    }
    for (int yy = 0; yy < H; ++yy)
        for (int xx = 0; xx < W; ++xx) {
            size_t i = (size_t)yy * W + xx;
            int d = degree(xx, yy, W, H);
            dinv[i] = (c[i] || d == 0) ? 0.0 : 1.0 / (double)d;
        }

    int status = ORACLE_OK;
    for (int ch = 0; ch < C; ++ch) {
        const float *fc = f + (size_t)ch * n;
        double *uc = u + (size_t)ch * n;
        /* reduced right-hand side: known neighbours moved to the right */
#pragma omp parallel for schedule(static)
        for (int yy = 0; yy < H; ++yy) {
            for (int xx = 0; xx < W; ++xx) {
                size_t i = (size_t)yy * W + xx;
                double acc = 0.0;
                if (!c[i]) {
                    if (xx > 0 && c[i - 1])     acc += fc[i - 1];
                    if (xx < W - 1 && c[i + 1]) acc += fc[i + 1];
                    if (yy > 0 && c[i - W])     acc += fc[i - W];
                    if (yy < H - 1 && c[i + W]) acc += fc[i + W];
                }
                b[i] = acc;
                x[i] = 0.0;
                r[i] = acc;
            }
        }
        double bnorm = sqrt(dot(b, b, n));
        int it = 0;
        double rn = bnorm;
        if (bnorm > 0.0) {
#pragma omp parallel for schedule(static)
            for (size_t i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
            double rz = dot(r, z, n);
            while (rn > rel_tol * bnorm && it < max_iter) {
                apply_reduced(c, W, H, p, q);
                double pq = dot(p, q, n);
                if (!(pq > 0.0)) break;
                double alpha = rz / pq;
#pragma omp parallel for schedule(static)
                for (size_t i = 0; i < n; ++i) {
                    x[i] += alpha * p[i];
                    r[i] -= alpha * q[i];
                    z[i] = dinv[i] * r[i];
                }
                double rz_new = dot(r, z, n);
                double beta = rz_new / rz;
                rz = rz_new;
#pragma omp parallel for schedule(static)
                for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
                rn = sqrt(dot(r, r, n));
                ++it;
            }
            /* report the true residual of the final iterate */
            apply_reduced(c, W, H, x, q);
            double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
            for (size_t i = 0; i < n; ++i) { double d = b[i] - q[i]; s += d * d; }
            rn = sqrt(s);
            if (rn > rel_tol * bnorm * 10.0) status = ORACLE_NOT_CONVERGED;
        }
        for (size_t i = 0; i < n; ++i) uc[i] = c[i] ? (double)fc[i] : x[i];
        if (iters) iters[ch] = it;
        if (relres) relres[ch] = bnorm > 0.0 ? rn / bnorm : 0.0;
    }
    free(b); free(x); free(r); free(z); free(p); free(q); free(dinv);
    return status;
}
