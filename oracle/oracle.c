/*
 * oracle.c -- plain, slow CPU oracle for double-precision GEMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA
 * library; it is checked against closed forms and exact arithmetic in
 * tests/test_oracle.py.
 *
 * Operation (paper Section 1.2, the BLAS dgemm statement):
 *     C := alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
 * C is m x n, op(A) is m x k, op(B) is k x n; k is the inner (third) dimension.
 * Storage (paper Section 2.1, column-major with leading dimension):
 *     element (i, j) of a matrix X with leading dimension ldx is X[j*ldx + i].
 * The element formula is the triple loop of Section 2.1,
 *     c_ij := sum_p a_ip b_pj  (+ c_ij),
 * here with the alpha/beta scaling of Section 1.2.
 *
 * Accumulation: each dot product is summed with the compensated "Dot2"
 * algorithm of Ogita, Rump and Oishi, "Accurate sum and dot product",
 * SIAM J. Sci. Comput. 26 (2005), Algorithm 5.3: an error-free product
 * (via fma) and an error-free sum (Knuth's TwoSum) per term, with the error
 * terms collected in a second accumulator.  The result is as accurate as if
 * computed in twice the working precision and rounded once.  The alpha/beta
 * epilogue is formed with the same error-free transformations.
 *
 * Quick returns follow the reference BLAS conventions (the paper is silent):
 *   m == 0 or n == 0            -> nothing is done;
 *   alpha == 0 or k == 0        -> C := beta*C, A and B are not read;
 *   beta == 0                   -> C0 is not read (NaN in C0 does not propagate).
 *
 * Must be compiled without value-changing floating-point optimisation
 * (-ffp-contract=off, no -ffast-math): the error-free transformations rely on
 * every operation being rounded exactly as written.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static int trans_code(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1; /* 'C' == 'T' for real data */
  return -1;
}

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

/* BLAS-style argument check; returns 0 or the 1-based index of the first bad argument. */
static int check_args(char transa, char transb, int64_t m, int64_t n, int64_t k,
                      int64_t lda, int64_t ldb, int64_t ldc) {
  int ta = trans_code(transa), tb = trans_code(transb);
  if (ta < 0) return 1;
  if (tb < 0) return 2;
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  if (lda < max64(1, ta ? k : m)) return 8;
  if (ldb < max64(1, tb ? n : k)) return 10;
  if (ldc < max64(1, m)) return 13;
  return 0;
}

/* element (i, p) of op(A) and (p, j) of op(B), column-major with leading dimension */
static inline double op_a(const double* A, int64_t lda, int ta, int64_t i, int64_t p) {
  return ta ? A[i * lda + p] : A[p * lda + i];
}
static inline double op_b(const double* B, int64_t ldb, int tb, int64_t p, int64_t j) {
  return tb ? B[p * ldb + j] : B[j * ldb + p];
}

/* error-free sum: x + y == a + b exactly, x = fl(a + b) (Knuth) */
static inline void two_sum(double a, double b, double* x, double* y) {
  double s = a + b;
  double z = s - a;
  *y = (a - (s - z)) + (b - z);
  *x = s;
}
/* error-free product: x + y == a * b exactly, x = fl(a * b) */
static inline void two_prod(double a, double b, double* x, double* y) {
  double p = a * b;
  *y = fma(a, b, -p);
  *x = p;
}

typedef struct {
  int ta, tb;
  int64_t m, n, k;
  double alpha, beta;
  const double *A, *B, *C0;
  int64_t lda, ldb, ldc;
  const int64_t* rows;
  int64_t nrows;
  double* out;
  int64_t ldo;
  int mode; /* 0: dgemm value, 1: |alpha||A||B| + |beta||C0| */
  int64_t j0, j1;
} job_t;

/* one element of C := alpha*op(A)*op(B) + beta*C0 with Dot2 accumulation */
static double dgemm_elem(const job_t* J, int64_t i, int64_t j) {
  double c0 = (J->beta != 0.0) ? J->C0[j * J->ldc + i] : 0.0;
  if (J->alpha == 0.0 || J->k == 0) return (J->beta == 0.0) ? 0.0 : J->beta * c0;
  double hi = 0.0, lo = 0.0, naive = 0.0;
  for (int64_t p = 0; p < J->k; ++p) {
    double a = op_a(J->A, J->lda, J->ta, i, p);
    double b = op_b(J->B, J->ldb, J->tb, p, j);
    double h, r, q;
    two_prod(a, b, &h, &r);
    two_sum(hi, h, &hi, &q);
    lo += q + r;
    naive += a * b;
  }
  if (!isfinite(hi) || !isfinite(lo)) {
    /* non-finite intermediates: fall back to plain IEEE propagation */
    double v = J->alpha * naive;
    return (J->beta == 0.0) ? v : v + J->beta * c0;
  }
  /* alpha*(hi + lo) + beta*c0 with error-free transformations, one final rounding chain */
  double h1, l1, h3 = 0.0, l3 = 0.0, h, e;
  two_prod(J->alpha, hi, &h1, &l1);
  l1 += J->alpha * lo;
  if (J->beta != 0.0) two_prod(J->beta, c0, &h3, &l3);
  two_sum(h1, h3, &h, &e);
  return h + (e + (l1 + l3));
}

/* one element of |alpha| * sum_p |a_ip||b_pj| + |beta| |c0|  (plain FP64 sums) */
static double absbound_elem(const job_t* J, int64_t i, int64_t j) {
  double s = 0.0;
  if (J->alpha != 0.0) {
    for (int64_t p = 0; p < J->k; ++p)
      s += fabs(op_a(J->A, J->lda, J->ta, i, p)) * fabs(op_b(J->B, J->ldb, J->tb, p, j));
    s *= fabs(J->alpha);
  }
  if (J->beta != 0.0) s += fabs(J->beta) * fabs(J->C0[j * J->ldc + i]);
  return s;
}

static void* run_job(void* arg) {
  const job_t* J = (const job_t*)arg;
  for (int64_t j = J->j0; j < J->j1; ++j) {
    for (int64_t r = 0; r < J->nrows; ++r) {
      int64_t i = J->rows ? J->rows[r] : r;
      double v = (J->mode == 0) ? dgemm_elem(J, i, j) : absbound_elem(J, i, j);
      J->out[j * J->ldo + r] = v;
    }
  }
  return NULL;
}

int oracle_num_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static int run_parallel(job_t* tmpl, int nthreads) {
  if (nthreads <= 0) nthreads = oracle_num_threads();
  if (nthreads > 256) nthreads = 256;
  if (tmpl->n < nthreads) nthreads = (int)(tmpl->n > 0 ? tmpl->n : 1);
  job_t jobs[256];
  pthread_t th[256];
  int started[256];
  int64_t per = (tmpl->n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = *tmpl;
    jobs[t].j0 = t * per < tmpl->n ? t * per : tmpl->n;
    jobs[t].j1 = (t + 1) * per < tmpl->n ? (t + 1) * per : tmpl->n;
    started[t] = 0;
  }
  for (int t = 1; t < nthreads; ++t)
    started[t] = (pthread_create(&th[t], NULL, run_job, &jobs[t]) == 0);
  run_job(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else run_job(&jobs[t]);
  }
  return 0;
}

static int run_rows(int mode, char transa, char transb, int64_t m, int64_t n, int64_t k,
                    double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                    double beta, const double* C0, int64_t ldc, const int64_t* rows,
                    int64_t nrows, double* out, int64_t ldo, int nthreads) {
  int bad = check_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (bad) return bad;
  if (!rows) nrows = m;
  if (ldo < max64(1, nrows)) return 17;
  if (rows)
    for (int64_t r = 0; r < nrows; ++r)
      if (rows[r] < 0 || rows[r] >= m) return 15;
  if (m == 0 || n == 0 || nrows == 0) return 0;
  job_t J;
  memset(&J, 0, sizeof(J));
  J.ta = trans_code(transa);
  J.tb = trans_code(transb);
  J.m = m; J.n = n; J.k = k;
  J.alpha = alpha; J.beta = beta;
  J.A = A; J.B = B; J.C0 = C0;
  J.lda = lda; J.ldb = ldb; J.ldc = ldc;
  J.rows = rows; J.nrows = nrows;
  J.out = out; J.ldo = ldo;
  J.mode = mode;
  return run_parallel(&J, nthreads);
}

/*
 * Rows `rows[0..nrows)` (all m rows when rows == NULL) of
 *     alpha * op(A) * op(B) + beta * C0
 * written to out (column-major, leading dimension ldo; row r of out is row
 * rows[r] of the result).  C0 is read only; out may alias C0 when rows == NULL
 * and ldo == ldc (each element reads its own c0 before writing it).
 * Returns 0, or the BLAS index of the first invalid argument
 * (1 transa, 2 transb, 3 m, 4 n, 5 k, 8 lda, 10 ldb, 13 ldc, 15 rows, 17 ldo).
 */
int oracle_dgemm_rows(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                      const double* C0, int64_t ldc, const int64_t* rows, int64_t nrows,
                      double* out, int64_t ldo, int nthreads) {
  return run_rows(0, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, rows, nrows,
                  out, ldo, nthreads);
}

/* In-place form with the exact dgemm argument list (C is overwritten). */
int oracle_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, int nthreads) {
  return run_rows(0, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, NULL, m, C,
                  ldc, nthreads);
}

/*
 * Rows of G = |alpha| |op(A)| |op(B)| + |beta| |C0| (the magnitude that scales the
 * componentwise error bound |C - C_exact| <= 2 k u G, u = 2^-53).  Same layout
 * and argument conventions as oracle_dgemm_rows.
 */
int oracle_abs_bound_rows(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                          const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                          const double* C0, int64_t ldc, const int64_t* rows, int64_t nrows,
                          double* out, int64_t ldo, int nthreads) {
  return run_rows(1, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C0, ldc, rows, nrows,
                  out, ldo, nthreads);
}
