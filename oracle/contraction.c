/*
 * Oracle (test infrastructure, not product code): the plain FP64 tensor
 * contraction of Section 1 ("Tensor Notation"),
 *
 *     C[f] = beta * C[f] + alpha * sum_{k in contracted} A[f_A, k] * B[f_B, k],
 *
 * written out as nested loops over the free indices of C with the contracted
 * indices innermost, every operand addressed through explicit element
 * strides (the Fortran-contiguous storage of Section 1 is the special case
 * stride[m] = prod_{m' < m} extent[m']).
 *
 * The caller classifies the indices: for each of the nf modes of C it passes
 * the extent and the stride of that index in C, A and B (0 when the operand
 * does not carry the index); for each of the nk contracted indices it passes
 * the extent and the strides in A and B.  Summation over the contracted
 * indices runs as an odometer whose first contracted index varies slowest.
 * beta == 0 means C is written without being read (BLAS convention).
 *
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark use
 * this file.  It shares no code with the CUDA library.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_MODES 16

static double sum_over_contracted(int nk, const int64_t *ext_k,
                                  const int64_t *sA_k, const int64_t *sB_k,
                                  const double *A, const double *B,
                                  int64_t offA, int64_t offB)
{
    int64_t idx[ORACLE_MAX_MODES];
    double s = 0.0;
    for (int m = 0; m < nk; ++m) idx[m] = 0;
    for (;;) {
        int64_t oa = offA, ob = offB;
        for (int m = 0; m < nk; ++m) {
            oa += idx[m] * sA_k[m];
            ob += idx[m] * sB_k[m];
        }
        s += A[oa] * B[ob];
        /* advance the odometer: last contracted index fastest */
        int m = nk - 1;
        while (m >= 0) {
            if (++idx[m] < ext_k[m]) break;
            idx[m] = 0;
            --m;
        }
        if (m < 0) break;
    }
    return s;
}

/*
 * Full contraction.  Only C elements whose last C mode lies in
 * [outer_lo, outer_hi) are computed (the whole tensor when outer_lo = 0 and
 * outer_hi = extent of that mode), so that a bounded slab can be timed.
 * nf >= 1 is required (a scalar C is passed as one mode of extent 1).
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_contract(int nf, const int64_t *ext_f, const int64_t *sC_f,
                    const int64_t *sA_f, const int64_t *sB_f,
                    int nk, const int64_t *ext_k, const int64_t *sA_k,
                    const int64_t *sB_k,
                    double alpha, const double *A, const double *B,
                    double beta, double *C,
                    int64_t outer_lo, int64_t outer_hi, int nthreads)
{
    if (nf < 1 || nf > ORACLE_MAX_MODES || nk < 0 || nk > ORACLE_MAX_MODES)
        return -1;
    if (outer_lo < 0 || outer_hi > ext_f[nf - 1] || outer_lo > outer_hi)
        return -1;
    int64_t inner = 1; /* number of C elements per value of the last C mode */
    for (int m = 0; m < nf - 1; ++m) inner *= ext_f[m];
    if (nthreads < 1) nthreads = 1;

    int64_t t;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (t = outer_lo; t < outer_hi; ++t) {
        int64_t idx[ORACLE_MAX_MODES];
        for (int64_t lin = 0; lin < inner; ++lin) {
            /* decode the free multi-index: first C mode fastest */
            int64_t r = lin;
            for (int m = 0; m < nf - 1; ++m) {
                idx[m] = r % ext_f[m];
                r /= ext_f[m];
            }
            idx[nf - 1] = t;
            int64_t oc = 0, oa = 0, ob = 0;
            for (int m = 0; m < nf; ++m) {
                oc += idx[m] * sC_f[m];
                oa += idx[m] * sA_f[m];
                ob += idx[m] * sB_f[m];
            }
            double s = (nk > 0)
                ? sum_over_contracted(nk, ext_k, sA_k, sB_k, A, B, oa, ob)
                : A[oa] * B[ob];
            C[oc] = (beta == 0.0) ? alpha * s : beta * C[oc] + alpha * s;
        }
    }
    return 0;
}

/*
 * The contraction sum (alpha = 1, beta = 0) at npts chosen points of C.
 * points holds npts rows of nf free-index values (C mode order).
 */
int oracle_contract_points(int nf, const int64_t *sA_f, const int64_t *sB_f,
                           int nk, const int64_t *ext_k, const int64_t *sA_k,
                           const int64_t *sB_k, const double *A, const double *B,
                           int64_t npts, const int64_t *points, double *out,
                           int nthreads)
{
    if (nf < 0 || nf > ORACLE_MAX_MODES || nk < 0 || nk > ORACLE_MAX_MODES)
        return -1;
    if (nthreads < 1) nthreads = 1;
    int64_t p;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (p = 0; p < npts; ++p) {
        int64_t oa = 0, ob = 0;
        for (int m = 0; m < nf; ++m) {
            oa += points[p * nf + m] * sA_f[m];
            ob += points[p * nf + m] * sB_f[m];
        }
        out[p] = (nk > 0)
            ? sum_over_contracted(nk, ext_k, sA_k, sB_k, A, B, oa, ob)
            : A[oa] * B[ob];
    }
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
