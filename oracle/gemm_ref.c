/*
 * CPU oracle, plain C part.  TEST INFRASTRUCTURE ONLY: nothing on the product
 * path links or calls this file; only the tests, the smoke check and the
 * bench's CPU-baseline leg do.
 *
 * Compiled with -O2 -ffp-contract=off so that every a*b + c below is a rounded
 * multiply followed by a rounded add (no fused multiply-add), in the order
 * written.
 */
#include <math.h>
#include <stdint.h>

/*
 * oracle_dgemm: C = A x B in binary64 by the plain triple loop.
 * Definition followed: Section II-A (SUMMA) and Section III -- after all n/b
 * steps every block c_ij equals sum_k a_ik x b_kj.  Each element is accumulated
 * over k in ascending order starting from +0.0:
 *     c_ij <- 0;  for k = 0..K-1:  c_ij <- c_ij + a_ik * b_kj
 * Row-major storage, leading dimensions lda >= K, ldb >= N, ldc >= N.
 * Rows are independent, so the i loop is split over nthreads OpenMP threads;
 * this does not change any element's arithmetic.
 */
void oracle_dgemm(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                  const double *B, int64_t ldb, double *C, int64_t ldc,
                  int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t i = 0; i < M; ++i) {
    double *c = C + i * ldc;
    for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      const double a = A[i * lda + k];
      const double *b = B + k * ldb;
      for (int64_t j = 0; j < N; ++j) c[j] = c[j] + a * b[j];
    }
  }
}

/* Error-free transformations (Ogita, Rump, Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005): TwoSum (Knuth) and TwoProduct
 * (via fma, exact when no underflow). */
static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/*
 * oracle_dot2_entries: for n listed entries (rows[t], cols[t]) compute
 *   c_out[t]     = Dot2(A[row, :], B[:, col])  (Algorithm Dot2 of the paper
 *                  above: as accurate as if computed in twice binary64 and then
 *                  rounded), the near-exact reference value of C_ij;
 *   absab_out[t] = sum_k |a_ik| |b_kj|  in plain binary64, the denominator
 *                  (|A||B|)_ij of the accuracy metric.
 */
void oracle_dot2_entries(int64_t M, int64_t N, int64_t K, const double *A,
                         int64_t lda, const double *B, int64_t ldb, int64_t n,
                         const int64_t *rows, const int64_t *cols,
                         double *c_out, double *absab_out, int nthreads) {
  (void)M;
  (void)N;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
  for (int64_t t = 0; t < n; ++t) {
    const double *a = A + rows[t] * lda;
    const int64_t j = cols[t];
    double p = 0.0, s = 0.0, absab = 0.0;
    if (K > 0) {
      two_prod(a[0], B[j], &p, &s);
      absab = fabs(a[0]) * fabs(B[j]);
    }
    for (int64_t k = 1; k < K; ++k) {
      double h, r, q;
      const double bk = B[k * ldb + j];
      two_prod(a[k], bk, &h, &r);
      two_sum(p, h, &p, &q);
      s = s + (q + r);
      absab = absab + fabs(a[k]) * fabs(bk);
    }
    c_out[t] = p + s;
    absab_out[t] = absab;
  }
}
