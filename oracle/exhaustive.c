/*
 * Oracle: exhaustive Gaussian summation in FP64 with compensated accumulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA path.
 *
 * Computes the plain definition of the Gaussian sum (Section 1):
 *     G(x_q) = sum_{r=1..N} w_r * exp(-||x_q - x_r||^2 / (2 h^2))
 * for every query q and every bandwidth h_j, in double precision, summing the
 * N terms with Neumaier's improved Kahan-Babuska compensated summation so the
 * result is accurate to a few ulps whatever N is.  Queries are independent;
 * OpenMP splits them statically across the host cores.
 *
 * Layout: queries M x D and refs N x D row-major doubles, weights N doubles,
 * h nh doubles, out M x nh row-major doubles.  skip_self != 0 (only valid when
 * queries and refs are the same array) leaves out the r == q term; the LSCV
 * leave-one-out score needs that sum.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Neumaier: s accumulates, c carries the lost low-order parts. */
static inline void neumaier_add(double *s, double *c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *c += (*s - t) + v;
    else
        *c += (v - t) + *s;
    *s = t;
}

#define ORACLE_MAX_NH 256

/* Returns 0, or -1 when nh is outside [1, ORACLE_MAX_NH]. */
int oracle_gauss_sum(const double *queries, int64_t M, const double *refs, const double *w,
                     int64_t N, int D, const double *h, int nh, int skip_self, double *out) {
    if (nh < 1 || nh > ORACLE_MAX_NH) return -1;
    double inv2h2[ORACLE_MAX_NH];
    for (int j = 0; j < nh; ++j) inv2h2[j] = 1.0 / (2.0 * h[j] * h[j]);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < M; ++q) {
        const double *xq = queries + q * (int64_t)D;
        double s[ORACLE_MAX_NH], c[ORACLE_MAX_NH];
        for (int j = 0; j < nh; ++j) s[j] = c[j] = 0.0;
        for (int64_t r = 0; r < N; ++r) {
            if (skip_self && r == q) continue;
            const double *xr = refs + r * (int64_t)D;
            double d2 = 0.0;
            for (int d = 0; d < D; ++d) {
                double diff = xq[d] - xr[d];
                d2 += diff * diff;
            }
            for (int j = 0; j < nh; ++j) neumaier_add(&s[j], &c[j], w[r] * exp(-d2 * inv2h2[j]));
        }
        for (int j = 0; j < nh; ++j) out[q * (int64_t)nh + j] = s[j] + c[j];
    }
    return 0;
}
