/*
 * Oracle: textbook Jacobi-preconditioned conjugate gradients on an explicit CSR matrix, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this file; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it (through oracle/poisson.py).
 *
 * The paper solves its pressure Poisson equation (Sec. 2 Eq. pois; Sec. 2.1 Eq. poisson1) with
 * "a preconditioned conjugate-gradient method" (Sec. 1) and names no preconditioner; the oracle
 * uses the diagonal (Jacobi) one.  The algorithm is the standard one:
 *     r = b - A x;  z = D^-1 r;  p = z;  rz = r.z
 *     repeat: q = A p;  alpha = rz / p.q;  x += alpha p;  r -= alpha q;
 *             stop when |r| <= rtol |b|;
 *             z = D^-1 r;  beta = r.z_new / rz;  p = z + beta p
 * and the residual b - A x is recomputed from scratch at the end.
 *
 * Reductions are summed over fixed 65536-element chunks in chunk order, so the result does not
 * depend on the number of OpenMP threads.
 *
 * A solve can also report when it first passed a looser tolerance (mark_rtol): the iteration and
 * the wall time since the start of the solve at which |r| <= mark_rtol |b| first held.  One solve
 * to a tight tolerance then also times the solve to the looser one, with the same iterates.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CHUNK 65536

static double wall_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void csr_matvec(int64_t n, const int64_t* ip, const int32_t* ix, const double* a,
                       const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = ip[i]; k < ip[i + 1]; ++k) s += a[k] * x[ix[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* x, const double* y, double* part) {
    int64_t nc = (n + CHUNK - 1) / CHUNK;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t lo = c * CHUNK, hi = lo + CHUNK < n ? lo + CHUNK : n;
        double s = 0.0;
        for (int64_t i = lo; i < hi; ++i) s += x[i] * y[i];
        part[c] = s;
    }
    double s = 0.0;
    for (int64_t c = 0; c < nc; ++c) s += part[c];
    return s;
}

int oracle_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

void oracle_csr_matvec(int64_t n, const int64_t* ip, const int32_t* ix, const double* a,
                       const double* x, double* y) {
    csr_matvec(n, ip, ix, a, x, y);
}

/* Returns 0 on convergence, 1 if maxit was reached, 2 on breakdown (p.q <= 0 or not finite),
 * 3 on a non-positive diagonal.  x holds the initial guess on entry and the iterate on exit.
 * alpha_hist / beta_hist (may be NULL) receive the CG coefficients of each iteration.
 * mark_iter / mark_seconds (may be NULL) receive the first iteration at which the updated
 * residual met mark_rtol and the seconds from entry to that point (-1 if it never did). */
int oracle_jacobi_pcg(int64_t n, const int64_t* ip, const int32_t* ix, const double* a,
                      const double* b, double* x, double rtol, int64_t maxit,
                      int64_t* iters_out, double* relres_out,
                      double* alpha_hist, double* beta_hist,
                      double mark_rtol, int64_t* mark_iter, double* mark_seconds) {
    const double t_start = wall_seconds();
    if (mark_iter) *mark_iter = -1;
    if (mark_seconds) *mark_seconds = -1.0;
    double* dinv = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* part = (double*)malloc(sizeof(double) * ((n + CHUNK - 1) / CHUNK + 1));
    int status = 1;
    int64_t it = 0;

    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = ip[i]; k < ip[i + 1]; ++k)
            if (ix[k] == i) d += a[k];
        if (!(d > 0.0)) { status = 3; goto done; }
        dinv[i] = 1.0 / d;
    }
    double bnorm = sqrt(dot(n, b, b, part));
    csr_matvec(n, ip, ix, a, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    double rz = dot(n, r, z, part);
    double rr0 = sqrt(dot(n, r, r, part));
    if (mark_iter && (bnorm == 0.0 || rr0 <= mark_rtol * bnorm)) {
        *mark_iter = 0;
        if (mark_seconds) *mark_seconds = wall_seconds() - t_start;
    }
    if (bnorm == 0.0 || rr0 <= rtol * bnorm) { status = 0; goto done; }
    for (it = 1; it <= maxit; ++it) {
        csr_matvec(n, ip, ix, a, p, q);
        double pq = dot(n, p, q, part);
        if (!(pq > 0.0) || !isfinite(pq)) { status = 2; break; }
        double alpha = rz / pq;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        double rr = dot(n, r, r, part);
        if (alpha_hist) alpha_hist[it - 1] = alpha;
        if (mark_iter && *mark_iter < 0 && sqrt(rr) <= mark_rtol * bnorm) {
            *mark_iter = it;
            if (mark_seconds) *mark_seconds = wall_seconds() - t_start;
        }
        if (sqrt(rr) <= rtol * bnorm) { status = 0; if (beta_hist) beta_hist[it - 1] = 0.0; break; }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz_new = dot(n, r, z, part);
        double beta = rz_new / rz;
        if (beta_hist) beta_hist[it - 1] = beta;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (it > maxit) it = maxit;
done:
    if (status != 3) {
        double bn = sqrt(dot(n, b, b, part));
        csr_matvec(n, ip, ix, a, x, q);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
        *relres_out = bn > 0.0 ? sqrt(dot(n, r, r, part)) / bn : 0.0;
    } else {
        *relres_out = NAN;
    }
    *iters_out = it;
    free(dinv); free(r); free(z); free(p); free(q); free(part);
    return status;
}
