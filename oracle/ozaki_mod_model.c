/*
 * ozaki_mod_model.c -- plain CPU model of the modular (Ozaki scheme II) emulation of
 * double-precision GEMM, used to check the GPU emulation bit for bit.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): nothing on the product path uses it.  It
 * shares no code with the CUDA library.
 *
 * The operation is the dgemm of the paper (Section 1.2):
 *     C := alpha * op(A) * op(B) + beta * C.
 * The method is the integer modular emulation of Ozaki, Uchino and Imamura, "Ozaki
 * Scheme II: a GEMM-oriented emulation of floating-point matrix multiplication using
 * an integer modular technique" (2025).  Steps, for t integer bits:
 *
 *  1. Scaling.  sigma_i = max_p e(a_ip) over the non-zero finite entries of row i of
 *     op(A), x = f 2^e(x) with 0.5 <= |f| < 1 (frexp); tau_j likewise over column j
 *     of op(B).  A zero row/column gets exponent 0.
 *  2. Integers.  A'_ip = rint(a_ip 2^(t - sigma_i)) and B'_pj = rint(b_pj 2^(t - tau_j)),
 *     rounded to nearest with ties to even; |A'|, |B'| <= 2^t.
 *  3. Product.  C'_ij = sum_p A'_ip B'_pj, an exact integer.  The method obtains it from
 *     the products of the residues of A' and B' modulo pairwise coprime moduli and the
 *     Chinese remainder theorem; whenever the product M of the moduli exceeds
 *     2 max |C'_ij| the reconstruction is C' itself, so the model evaluates C' directly
 *     in 128-bit integers.
 *  4. Result.  W = beta*c0 (0 when beta == 0, c0 not read), then
 *         W = fma(alpha * 2^(tau_j - 2t), fl(C'_ij) * 2^sigma_i, W),
 *     where fl is the correctly rounded conversion to double (ties to even) and each
 *     power-of-two factor is applied with ldexp.
 *
 * With dA = A' 2^(sigma - t) - A (|dA_ip| <= 2^(sigma_i - t - 1)) and likewise dB, the
 * product error is at most 2^(sigma_i + tau_j - t - 1) (nu_j + mu_i + k 2^(-t-1)) with
 * mu_i = sum_p |a_ip| 2^-sigma_i and nu_j = sum_p |b_pj| 2^-tau_j, plus the roundings of
 * step 4.
 *
 * Readings where the method is silent: non-finite entries make the whole matching row
 * or column of the result NaN (as in the scheme I model); quick returns are those of the
 * plain oracle.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef __int128 i128;

static int om_trans(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}

static int om_exponent(double x) {
  int e = 0;
  if (x == 0.0) return 0;
  (void)frexp(x, &e);
  return e;
}

/* correctly rounded conversion of a 128-bit integer to double */
double oracle_ozmod_i128_to_double(int64_t hi, uint64_t lo) {
  const i128 v = (i128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
  return (double)v;
}

typedef struct {
  int ta, tb, t;
  int64_t m, n, k;
  double alpha, beta;
  const double *A, *B, *C0;
  int64_t lda, ldb, ldc;
  const int64_t* rows;
  int64_t nrows;
  const int64_t* ra;  /* [nrows][k] integers A' of the requested rows */
  const int* rsig;    /* [nrows] */
  const int* rbad;    /* [nrows] */
  double* out;
  int64_t ldo;
  int64_t j0, j1;
  int err;
} omjob_t;

static inline double om_b(const omjob_t* J, int64_t p, int64_t j) {
  return J->tb ? J->B[p * J->ldb + j] : J->B[j * J->ldb + p];
}

static void* om_run(void* arg) {
  omjob_t* J = (omjob_t*)arg;
  const int64_t k = J->k;
  int64_t* cb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
  if (!cb) { J->err = -2; return NULL; }
  for (int64_t j = J->j0; j < J->j1; ++j) {
    int tau = 0, cbad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = om_b(J, p, j);
      if (!isfinite(v)) { cbad = 1; continue; }
      if (v != 0.0) {
        const int e = om_exponent(v);
        if (!any || e > tau) tau = e;
        any = 1;
      }
    }
    for (int64_t p = 0; p < k; ++p) {
      const double v = om_b(J, p, j);
      cb[p] = isfinite(v) ? (int64_t)rint(ldexp(v, J->t - tau)) : 0;
    }
    for (int64_t r = 0; r < J->nrows; ++r) {
      const int64_t i = J->rows ? J->rows[r] : r;
      const double c0 = (J->beta != 0.0) ? J->C0[j * J->ldc + i] : 0.0;
      double W = (J->beta != 0.0) ? J->beta * c0 : 0.0;
      if (J->rbad[r] || cbad) {
        J->out[j * J->ldo + r] = NAN;
        continue;
      }
      const int64_t* a = J->ra + r * k;
      i128 s = 0;
      for (int64_t p = 0; p < k; ++p) s += (i128)a[p] * (i128)cb[p];
      const double x = (double)s;
      W = fma(ldexp(J->alpha, tau - 2 * J->t), ldexp(x, J->rsig[r]), W);
      J->out[j * J->ldo + r] = W;
    }
  }
  free(cb);
  return NULL;
}

/*
 * Rows `rows[0..nrows)` (all m rows when rows == NULL) of the modular emulation with t
 * integer bits, written to out (column-major, leading dimension ldo).  t in [1, 62]
 * (the exact sum of step 3 must fit 128 bits: k 2^(2t) < 2^127).
 * Returns 0, a BLAS argument index (1,2,3,4,5,8,10,13; 15 rows; 17 ldo; 18 t), or -2.
 */
int oracle_ozmod_dgemm_rows(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                            const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                            const double* C0, int64_t ldc, int t, const int64_t* rows, int64_t nrows,
                            double* out, int64_t ldo, int nthreads) {
  const int ta = om_trans(transa), tb = om_trans(transb);
  if (ta < 0) return 1;
  if (tb < 0) return 2;
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  if (lda < ((ta ? k : m) > 1 ? (ta ? k : m) : 1)) return 8;
  if (ldb < ((tb ? n : k) > 1 ? (tb ? n : k) : 1)) return 10;
  if (ldc < (m > 1 ? m : 1)) return 13;
  if (!rows) nrows = m;
  if (nrows < 0) return 15;
  if (ldo < (nrows > 1 ? nrows : 1)) return 17;
  if (t < 1 || t > 62) return 18;
  if (k > 0 && (double)k * ldexp(1.0, 2 * t) >= ldexp(1.0, 126)) return 18;
  for (int64_t r = 0; r < nrows; ++r)
    if (rows && (rows[r] < 0 || rows[r] >= m)) return 15;
  if (m == 0 || n == 0 || nrows == 0) return 0;
  if (alpha == 0.0 || k == 0) {  /* quick return: C := beta*C */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows ? rows[r] : r;
        out[j * ldo + r] = beta == 0.0 ? 0.0 : beta * C0[j * ldc + i];
      }
    return 0;
  }
  int64_t* ra = (int64_t*)malloc(sizeof(int64_t) * (size_t)nrows * (size_t)k);
  int* rsig = (int*)malloc(sizeof(int) * (size_t)nrows);
  int* rbad = (int*)malloc(sizeof(int) * (size_t)nrows);
  if (!ra || !rsig || !rbad) {
    free(ra); free(rsig); free(rbad);
    return -2;
  }
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows ? rows[r] : r;
    int sig = 0, bad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      if (!isfinite(v)) { bad = 1; continue; }
      if (v != 0.0) {
        const int e = om_exponent(v);
        if (!any || e > sig) sig = e;
        any = 1;
      }
    }
    rsig[r] = sig;
    rbad[r] = bad;
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      ra[r * k + p] = isfinite(v) ? (int64_t)rint(ldexp(v, t - sig)) : 0;
    }
  }
  if (nthreads < 1) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    nthreads = c > 0 ? (int)c : 1;
  }
  if (nthreads > n) nthreads = (int)n;
  if (nthreads < 1) nthreads = 1;
  omjob_t* jobs = (omjob_t*)calloc((size_t)nthreads, sizeof(omjob_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  int rc = 0;
  if (!jobs || !th) rc = -2;
  for (int w = 0; w < nthreads && !rc; ++w) {
    omjob_t* J = &jobs[w];
    J->ta = ta; J->tb = tb; J->t = t;
    J->m = m; J->n = n; J->k = k;
    J->alpha = alpha; J->beta = beta;
    J->A = A; J->B = B; J->C0 = C0;
    J->lda = lda; J->ldb = ldb; J->ldc = ldc;
    J->rows = rows; J->nrows = nrows;
    J->ra = ra; J->rsig = rsig; J->rbad = rbad;
    J->out = out; J->ldo = ldo;
    J->j0 = n * w / nthreads;
    J->j1 = n * (w + 1) / nthreads;
    if (pthread_create(&th[w], NULL, om_run, J) != 0) {
      om_run(J);
      th[w] = 0;
    }
  }
  for (int w = 0; w < nthreads && jobs && th; ++w) {
    if (th[w]) pthread_join(th[w], NULL);
    if (jobs[w].err) rc = jobs[w].err;
  }
  free(jobs); free(th); free(ra); free(rsig); free(rbad);
  return rc;
}
