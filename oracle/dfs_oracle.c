/*
 * Test oracle (test infrastructure only: tests, the smoke check and the CPU
 * baseline of the benchmark call it; the product path never does).
 *
 * Plain FP64 direct summation of the DFS series in complex exponential form
 * (Eq. 5.3, Sec. 5): for every point p,
 *
 *     v_p = sum_{n=-N2/2}^{N2/2-1} sum_{m=-N1/2}^{N1/2-1}
 *               c_{n,m} exp(i m phi_p) exp(i n theta_p)
 *
 * i.e. the type-II nonuniform DFT the paper evaluates at the departure
 * points (Sec. 5, the direct O((M_lon N_lat)^2) cost it quotes).  Nothing is
 * blocked, fused or reordered beyond the order written above; the inner sum
 * runs over m for each n and the outer over n.
 *
 * Numerics, chosen so that the oracle's own error sits far below 1e-11:
 *  - exp(i m phi) is taken from sin/cos of the exact product m*phi, formed
 *    as hi + lo with an FMA (two-product) and corrected to first order in lo;
 *  - both sums are Neumaier-compensated, real and imaginary parts apart;
 *  - no long double (software binary128 on aarch64).
 *
 * Layout: coef is (N2, N1) complex interleaved (re, im), row r <-> n = r - N2/2,
 * column q <-> m = q - N1/2, m fastest.  out is P complex interleaved.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double s, c; } acc_t;   /* Neumaier running sum and compensation */

static void acc_add(acc_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}

/* exp(i k t) for the exact product k*t. */
static void cis_of_product(double k, double t, double *re, double *im) {
    double hi = k * t;
    double lo = fma(k, t, -hi);
    double s = sin(hi), c = cos(hi);
    *re = c - lo * s;
    *im = s + lo * c;
}

int dfs_oracle_eval(int n1, int n2, const double *coef, int64_t npts,
                    const double *lon, const double *colat, double *out, int nthreads) {
    if (n1 <= 0 || n2 <= 0 || npts < 0 || !coef || (npts > 0 && (!lon || !colat || !out)))
        return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int bad = 0;
#pragma omp parallel
    {
        double *em = (double *)malloc(sizeof(double) * 2 * (size_t)n1);
        double *en = (double *)malloc(sizeof(double) * 2 * (size_t)n2);
        if (!em || !en) {
#pragma omp atomic write
            bad = 1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t p = 0; p < npts; ++p) {
                for (int q = 0; q < n1; ++q)
                    cis_of_product((double)(q - n1 / 2), lon[p], &em[2 * q], &em[2 * q + 1]);
                for (int r = 0; r < n2; ++r)
                    cis_of_product((double)(r - n2 / 2), colat[p], &en[2 * r], &en[2 * r + 1]);
                acc_t tr = {0, 0}, ti = {0, 0};
                for (int r = 0; r < n2; ++r) {
                    const double *row = coef + 2 * (size_t)r * (size_t)n1;
                    acc_t sr = {0, 0}, si = {0, 0};
                    for (int q = 0; q < n1; ++q) {
                        double cr = row[2 * q], ci = row[2 * q + 1];
                        double er = em[2 * q], ei = em[2 * q + 1];
                        acc_add(&sr, cr * er - ci * ei);
                        acc_add(&si, cr * ei + ci * er);
                    }
                    double ir = sr.s + sr.c, ii = si.s + si.c;
                    acc_add(&tr, ir * en[2 * r] - ii * en[2 * r + 1]);
                    acc_add(&ti, ir * en[2 * r + 1] + ii * en[2 * r]);
                }
                out[2 * p] = tr.s + tr.c;
                out[2 * p + 1] = ti.s + ti.c;
            }
        }
        free(em);
        free(en);
    }
    return bad ? 2 : 0;
}

int dfs_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
