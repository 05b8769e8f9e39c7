/*
 * level3.c -- plain CPU oracle for the GEMM-based level-3 BLAS operations DSYRK,
 * DTRMM and DTRSM, the extension the paper names for its GEMM kernel ("Poorman's
 * BLAS", Section 3.1: every level-3 operation can be cast in terms of matrix-matrix
 * products with submatrices, after Kagstrom, Ling and Van Loan, TOMS 24(3), 1998).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): nothing on the product path uses it.  It
 * shares no code with the CUDA library.
 *
 * Definitions (reference BLAS argument lists and conventions; column-major storage
 * with leading dimensions as in Section 2.1):
 *   DSYRK  C := alpha op(A) op(A)^T + beta C on the `uplo` triangle of C only, with
 *          op(A) = A (n x k) for trans = 'N' and A^T (A is k x n) for 'T'/'C'.
 *   DTRMM  B := alpha op(A) B (side 'L', A m x m) or alpha B op(A) (side 'R', A n x n),
 *          A triangular: only the `uplo` triangle is read; diag = 'U' means a unit
 *          diagonal that is not read.
 *   DTRSM  solves op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'); X
 *          overwrites B.
 * Each element is an inner product accumulated with Dot2 (Ogita, Rump and Oishi 2005:
 * error-free products and sums, one rounding at the end).  DTRSM is substitution in
 * the order the triangle fixes; each numerator alpha b - sum a x is a Dot2 sum, then
 * one division by the diagonal.
 * Quick returns follow reference BLAS: alpha = 0 gives beta C (DSYRK, triangle only)
 * or B := 0 (DTRMM, DTRSM) without reading A.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static inline void l3_two_sum(double a, double b, double* x, double* y) {
  double s = a + b;
  double z = s - a;
  *y = (a - (s - z)) + (b - z);
  *x = s;
}
static inline void l3_two_prod(double a, double b, double* x, double* y) {
  double p = a * b;
  *y = fma(a, b, -p);
  *x = p;
}

/* Dot2 accumulator */
typedef struct {
  double hi, lo, naive;
} acc2_t;
static inline void acc_add_prod(acc2_t* s, double a, double b) {
  double h, r, q;
  l3_two_prod(a, b, &h, &r);
  l3_two_sum(s->hi, h, &s->hi, &q);
  s->lo += q + r;
  s->naive += a * b;
}
static inline int acc_finite(const acc2_t* s) { return isfinite(s->hi) && isfinite(s->lo); }

static int l3_nthreads(int want, int64_t units) {
  if (want < 1) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    want = c > 0 ? (int)c : 1;
  }
  if (want > units) want = (int)units;
  return want < 1 ? 1 : want;
}

static int l3_upper(char u) { return (u == 'U' || u == 'u') ? 1 : (u == 'L' || u == 'l') ? 0 : -1; }
static int l3_trans(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}
static int l3_side(char s) { return (s == 'L' || s == 'l') ? 0 : (s == 'R' || s == 'r') ? 1 : -1; }
static int l3_diag(char d) { return (d == 'U' || d == 'u') ? 1 : (d == 'N' || d == 'n') ? 0 : -1; }
static int64_t l3_max(int64_t a, int64_t b) { return a > b ? a : b; }

/* alpha * (hi + lo) + beta * c0 with one final rounding chain (as the GEMM oracle) */
static double l3_finish(const acc2_t* s, double alpha, double beta, double c0) {
  if (!acc_finite(s)) {
    double v = alpha * s->naive;
    return beta == 0.0 ? v : v + beta * c0;
  }
  double h1, l1, h3 = 0.0, l3 = 0.0, h, e;
  l3_two_prod(alpha, s->hi, &h1, &l1);
  l1 += alpha * s->lo;
  if (beta != 0.0) l3_two_prod(beta, c0, &h3, &l3);
  l3_two_sum(h1, h3, &h, &e);
  return h + (e + (l1 + l3));
}

/* ------------------------------------------------------------------ DSYRK */
typedef struct {
  int up, tr;
  int64_t n, k;
  double alpha, beta;
  const double* A;
  int64_t lda;
  double* C;
  int64_t ldc;
  int64_t j0, j1;
} syrk_job_t;

static inline double syrk_opa(const syrk_job_t* J, int64_t i, int64_t p) {
  return J->tr ? J->A[i * J->lda + p] : J->A[p * J->lda + i];
}

static void* syrk_run(void* arg) {
  syrk_job_t* J = (syrk_job_t*)arg;
  for (int64_t j = J->j0; j < J->j1; ++j) {
    const int64_t i0 = J->up ? 0 : j, i1 = J->up ? j + 1 : J->n;
    for (int64_t i = i0; i < i1; ++i) {
      double* c = &J->C[j * J->ldc + i];
      const double c0 = J->beta != 0.0 ? *c : 0.0;
      if (J->alpha == 0.0 || J->k == 0) {
        *c = J->beta == 0.0 ? 0.0 : J->beta * c0;
        continue;
      }
      acc2_t s = {0.0, 0.0, 0.0};
      for (int64_t p = 0; p < J->k; ++p) acc_add_prod(&s, syrk_opa(J, i, p), syrk_opa(J, j, p));
      *c = l3_finish(&s, J->alpha, J->beta, c0);
    }
  }
  return NULL;
}

/* Returns 0 or the reference-BLAS index of the first invalid argument. */
int oracle_dsyrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                 double beta, double* C, int64_t ldc, int nthreads) {
  const int up = l3_upper(uplo), tr = l3_trans(trans);
  if (up < 0) return 1;
  if (tr < 0) return 2;
  if (n < 0) return 3;
  if (k < 0) return 4;
  if (lda < l3_max(1, tr ? k : n)) return 7;
  if (ldc < l3_max(1, n)) return 10;
  if (n == 0 || ((alpha == 0.0 || k == 0) && beta == 1.0)) return 0;
  const int nt = l3_nthreads(nthreads, n);
  syrk_job_t* jobs = (syrk_job_t*)calloc((size_t)nt, sizeof(syrk_job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -2;
  }
  for (int w = 0; w < nt; ++w) {
    syrk_job_t* J = &jobs[w];
    J->up = up; J->tr = tr; J->n = n; J->k = k; J->alpha = alpha; J->beta = beta;
    J->A = A; J->lda = lda; J->C = C; J->ldc = ldc;
    /* columns split so each thread gets about the same triangle area */
    const double f0 = (double)w / nt, f1 = (double)(w + 1) / nt;
    const double a0 = up ? sqrt(f0) : 1.0 - sqrt(1.0 - f0), a1 = up ? sqrt(f1) : 1.0 - sqrt(1.0 - f1);
    J->j0 = w == 0 ? 0 : (int64_t)(a0 * (double)n);
    J->j1 = w == nt - 1 ? n : (int64_t)(a1 * (double)n);
    if (pthread_create(&th[w], NULL, syrk_run, J) != 0) {
      syrk_run(J);
      th[w] = 0;
    }
  }
  for (int w = 0; w < nt; ++w)
    if (th[w]) pthread_join(th[w], NULL);
  free(jobs);
  free(th);
  return 0;
}

/* ------------------------------------------------------ DTRMM and DTRSM */
typedef struct {
  int side, up, tr, unit, solve;
  int64_t m, n;
  double alpha;
  const double* A;
  int64_t lda;
  double* B;
  int64_t ldb;
  int64_t u0, u1; /* columns (side L) or rows (side R) of B handled by this thread */
  int err;
} tri_job_t;

/* element (r, c) of op(A) with the triangle and the unit diagonal applied */
static inline double tri_op(const tri_job_t* J, int64_t r, int64_t c) {
  /* op(A)(r, c) = A(r, c) or A(c, r); stored triangle `up` refers to A itself */
  const int64_t ar = J->tr ? c : r, ac = J->tr ? r : c;
  if (ar == ac) return J->unit ? 1.0 : J->A[ac * J->lda + ar];
  const int in = J->up ? (ar < ac) : (ar > ac);
  return in ? J->A[ac * J->lda + ar] : 0.0;
}

static void* tri_run(void* arg) {
  tri_job_t* J = (tri_job_t*)arg;
  const int64_t len = J->side ? J->n : J->m;  /* order of op(A) */
  /* op(A) is lower triangular when (uplo = L) xor (transposed) */
  const int low = J->up ? J->tr : !J->tr;
  double* v = (double*)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
  double* x = (double*)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
  if (!v || !x) {
    free(v);
    free(x);
    J->err = -2;
    return NULL;
  }
  for (int64_t u = J->u0; u < J->u1; ++u) {
    /* the vector: column u of B (side L) or row u of B (side R) */
    for (int64_t q = 0; q < len; ++q) v[q] = J->side ? J->B[q * J->ldb + u] : J->B[u * J->ldb + q];
    if (!J->solve) {
      /* side L: x_r = alpha sum_c op(A)_rc v_c;  side R: x_c = alpha sum_r v_r op(A)_rc */
      for (int64_t q = 0; q < len; ++q) {
        /* the triangle's range: row q of a lower op(A) (side L) or column q of an upper
           one (side R) holds t <= q; the other two cases hold t >= q */
        const int head = J->side ? !low : low;
        const int64_t t0 = head ? 0 : q, t1 = head ? q + 1 : len;
        acc2_t s = {0.0, 0.0, 0.0};
        for (int64_t t = t0; t < t1; ++t) acc_add_prod(&s, J->side ? tri_op(J, t, q) : tri_op(J, q, t), v[t]);
        x[q] = l3_finish(&s, J->alpha, 0.0, 0.0);
      }
    } else {
      /* side L: op(A) x = alpha v, substitution down (lower) or up (upper) op(A);
         side R: x op(A) = alpha v, i.e. op(A)^T x = alpha v: the transpose is lower
         exactly when op(A) is upper */
      const int fwd = J->side ? !low : low;
      for (int64_t step = 0; step < len; ++step) {
        const int64_t q = fwd ? step : len - 1 - step;
        acc2_t s = {0.0, 0.0, 0.0};
        acc_add_prod(&s, J->alpha, v[q]);
        const int64_t t0 = fwd ? 0 : q + 1, t1 = fwd ? q : len;
        for (int64_t t = t0; t < t1; ++t) {
          const double a = J->side ? tri_op(J, t, q) : tri_op(J, q, t);
          acc_add_prod(&s, -a, x[t]);
        }
        const double num = acc_finite(&s) ? s.hi + s.lo : s.naive;
        x[q] = J->unit ? num : num / tri_op(J, q, q);
      }
    }
    for (int64_t q = 0; q < len; ++q) {
      if (J->side) J->B[q * J->ldb + u] = x[q];
      else J->B[u * J->ldb + q] = x[q];
    }
  }
  free(v);
  free(x);
  return NULL;
}

static int tri_common(int solve, char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha,
                      const double* A, int64_t lda, double* B, int64_t ldb, int nthreads) {
  const int sd = l3_side(side), up = l3_upper(uplo), tr = l3_trans(transa), un = l3_diag(diag);
  if (sd < 0) return 1;
  if (up < 0) return 2;
  if (tr < 0) return 3;
  if (un < 0) return 4;
  if (m < 0) return 5;
  if (n < 0) return 6;
  if (lda < l3_max(1, sd ? n : m)) return 9;
  if (ldb < l3_max(1, m)) return 11;
  if (m == 0 || n == 0) return 0;
  if (alpha == 0.0) {
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < m; ++i) B[j * ldb + i] = 0.0;
    return 0;
  }
  const int64_t units = sd ? m : n;  /* rows of B (side R) or columns (side L) */
  const int nt = l3_nthreads(nthreads, units);
  tri_job_t* jobs = (tri_job_t*)calloc((size_t)nt, sizeof(tri_job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -2;
  }
  int rc = 0;
  for (int w = 0; w < nt; ++w) {
    tri_job_t* J = &jobs[w];
    J->side = sd; J->up = up; J->tr = tr; J->unit = un; J->solve = solve;
    J->m = m; J->n = n; J->alpha = alpha; J->A = A; J->lda = lda; J->B = B; J->ldb = ldb;
    J->u0 = units * w / nt;
    J->u1 = units * (w + 1) / nt;
    if (pthread_create(&th[w], NULL, tri_run, J) != 0) {
      tri_run(J);
      th[w] = 0;
    }
  }
  for (int w = 0; w < nt; ++w) {
    if (th[w]) pthread_join(th[w], NULL);
    if (jobs[w].err) rc = jobs[w].err;
  }
  free(jobs);
  free(th);
  return rc;
}

/* B := alpha op(A) B or alpha B op(A); returns 0 or the reference-BLAS argument index */
int oracle_dtrmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha, const double* A,
                 int64_t lda, double* B, int64_t ldb, int nthreads) {
  return tri_common(0, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, nthreads);
}

/* B := X with op(A) X = alpha B or X op(A) = alpha B; returns 0 or the argument index */
int oracle_dtrsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha, const double* A,
                 int64_t lda, double* B, int64_t ldb, int nthreads) {
  return tri_common(1, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, nthreads);
}
