/*
 * ozaki_model.c -- plain CPU model of the split (Ozaki-scheme) emulation of
 * double-precision GEMM, used to check the GPU emulation bit for bit.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): nothing on the product path uses it.
 * It shares no code with the CUDA library.  Where the CUDA library extracts
 * digits with integer bit operations, this model uses the textbook floating-
 * point recursion; both are exact, so they must agree bit for bit.
 *
 * The operation is the dgemm of the paper (Section 1.2):
 *     C := alpha * op(A) * op(B) + beta * C.
 * The method is the error-free splitting of Ozaki, Ogita, Oishi and Rump,
 * "Error-free transformations of matrix multiplication by using fast routines
 * of matrix multiplication and its applications", Numer. Algorithms 59 (2012),
 * in its fixed-point digit form (digits are small integers, as in the
 * integer-slice variants of Ootomo, Ozaki and Yokota, 2024).  Steps, for
 * digit width b bits and s slices:
 *
 *  1. Scaling.  sigma_i = max_p e(a_ip) over the non-zero entries of row i of
 *     op(A), where x = f * 2^e(x) with 0.5 <= |f| < 1 (frexp); tau_j likewise
 *     over column j of op(B).  A zero row/column gets exponent 0.
 *  2. Splitting.  r_0 = a_ip * 2^-sigma_i (so |r_0| < 1); for t = 1..s:
 *         d_t = trunc(2^b * r_{t-1}),   r_t = 2^b * r_{t-1} - d_t.
 *     Every step is exact in FP64; |d_t| <= 2^b - 1.  Same for op(B) with tau_j.
 *  3. Products.  For level g = 2..s+1 (pairs t + u = g, 1 <= t, u <= s) the
 *     exact integer level sum over a segment S of the inner dimension is
 *         P_{g,S}(i,j) = sum_{t=1}^{g-1} sum_{p in S} d_t(a_ip) d_{g-t}(b_pj).
 *     The segments are consecutive runs of kseg indices of k.
 *  4. Accumulation.  W = beta*c0 (0 when beta == 0, c0 not read).  Then for
 *     each segment S in order, the levels are taken from the smallest (g = s+1)
 *     down to g = 2 in groups of up to four consecutive levels; a group whose
 *     smallest level is h sums its levels exactly as one integer,
 *         Y = sum_{g in group} P_{g,S} 2^(b (h - g)),
 *     and adds it with one rounding,
 *         W = fma(alpha * 2^(tau_j - h*b), Y * 2^sigma_i, W),
 *     the power of two split between the two factors as written (each factor is
 *     formed with ldexp, so the result stays a single rounding of the exact value
 *     while both factors are normal numbers, and results near the underflow range
 *     do not lose bits to an intermediate underflow of 2^(sigma_i + tau_j - h*b)).
 *     The result is W.  |P_{g,S}| <= 9 * kseg * (2^b - 1)^2 < 2^30.2 for the
 *     kseg = 8192, b = 7 of the GPU path, so |Y| < 2^51.2 and Y is exact in FP64.
 *
 * Pairs with t + u > s + 1 are dropped; the truncation and the dropped pairs
 * bound the error by |alpha| 2^(sigma_i + tau_j - s*b) (mu_i + nu_j + (s-1)(1+2^-b) N)
 * plus the FP64 rounding of step 4, where mu_i = sum_p |a_ip| 2^-sigma_i,
 * nu_j = sum_p |b_pj| 2^-tau_j and N = k.
 *
 * Readings where the method is silent: non-finite entries cannot be split, so a
 * row of op(A) or column of op(B) that holds Inf/NaN makes the whole matching
 * row/column of the result NaN; quick returns are those of the plain oracle.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static int oz_trans(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}

/* frexp exponent of x (x = f 2^e, 0.5 <= |f| < 1); 0 for x == 0 */
int oracle_ozaki_exponent(double x) {
  int e = 0;
  if (x == 0.0) return 0;
  (void)frexp(x, &e);
  return e;
}

/* digits d_1..d_s of x scaled by 2^-sigma (step 2); |x| must be < 2^sigma */
void oracle_ozaki_split(double x, int sigma, int s, int bits, int32_t* digits) {
  double r = ldexp(x, -sigma);
  for (int t = 0; t < s; ++t) {
    double y = ldexp(r, bits);
    double d = trunc(y);
    digits[t] = (int32_t)d;
    r = y - d;
  }
}

typedef struct {
  int ta, tb, s, bits;
  int64_t m, n, k, kseg;
  double alpha, beta;
  const double *A, *B, *C0;
  int64_t lda, ldb, ldc;
  const int64_t* rows;
  int64_t nrows;
  const int16_t* rdig; /* [nrows][s][k] digits of the requested rows of op(A) */
  const int* rsig;     /* [nrows] sigma */
  const int* rbad;     /* [nrows] non-finite flag */
  double* out;
  int64_t ldo;
  int64_t j0, j1;
  int err;
} ozjob_t;

static inline double oz_b(const ozjob_t* J, int64_t p, int64_t j) {
  return J->tb ? J->B[p * J->ldb + j] : J->B[j * J->ldb + p];
}
static inline double oz_a(const ozjob_t* J, int64_t i, int64_t p) {
  return J->ta ? J->A[i * J->lda + p] : J->A[p * J->lda + i];
}

static void* oz_run(void* arg) {
  ozjob_t* J = (ozjob_t*)arg;
  const int s = J->s, b = J->bits;
  const int64_t k = J->k;
  int16_t* cdig = (int16_t*)malloc(sizeof(int16_t) * (size_t)(s > 0 ? s : 1) * (size_t)(k > 0 ? k : 1));
  int32_t dg[16];
  if (!cdig) { J->err = -2; return NULL; }
  for (int64_t j = J->j0; j < J->j1; ++j) {
    /* step 1 and 2 for column j of op(B) */
    int tau = 0, cbad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      double v = oz_b(J, p, j);
      if (!isfinite(v)) { cbad = 1; continue; }
      if (v != 0.0) {
        int e = oracle_ozaki_exponent(v);
        if (!any || e > tau) tau = e;
        any = 1;
      }
    }
    for (int64_t p = 0; p < k; ++p) {
      double v = oz_b(J, p, j);
      if (!isfinite(v)) v = 0.0;
      oracle_ozaki_split(v, tau, s, b, dg);
      for (int t = 0; t < s; ++t) cdig[(size_t)t * k + p] = (int16_t)dg[t];
    }
    for (int64_t r = 0; r < J->nrows; ++r) {
      int64_t i = J->rows ? J->rows[r] : r;
      double c0 = (J->beta != 0.0) ? J->C0[j * J->ldc + i] : 0.0;
      double W = (J->beta != 0.0) ? J->beta * c0 : 0.0;
      if (J->rbad[r] || cbad) {
        J->out[j * J->ldo + r] = NAN;
        continue;
      }
      const int16_t* rd = J->rdig + (size_t)r * s * k;
      for (int64_t p0 = 0; p0 < k; p0 += J->kseg) {
        const int64_t p1 = p0 + J->kseg < k ? p0 + J->kseg : k;
        for (int h = s + 1; h >= 2; h -= 4) {  /* level groups {h, h-1, h-2, h-3} */
          int64_t Y = 0;
          for (int g = h; g >= 2 && g > h - 4; --g) {
            int64_t P = 0;
            for (int t = 1; t <= g - 1; ++t) {
              const int16_t* dt = rd + (size_t)(t - 1) * k;
              const int16_t* eu = cdig + (size_t)(g - t - 1) * k;
              for (int64_t p = p0; p < p1; ++p) P += (int64_t)dt[p] * (int64_t)eu[p];
            }
            Y += P * ((int64_t)1 << (b * (h - g)));
          }
          W = fma(ldexp(J->alpha, tau - h * b), ldexp((double)Y, J->rsig[r]), W);
        }
      }
      J->out[j * J->ldo + r] = W;
    }
  }
  free(cdig);
  return NULL;
}

/*
 * Rows `rows[0..nrows)` (all m rows when rows == NULL) of the split emulation
 * described above, written to out (column-major, leading dimension ldo).
 * slices in [1, 9], bits in [1, 8] with slices*bits <= 63, kseg >= 1.
 * Returns 0, a BLAS argument index (1,2,3,4,5,8,10,13; 15 rows; 17 ldo;
 * 18 slices/bits; 19 kseg), or -2 when memory runs out.
 */
int oracle_ozaki_dgemm_rows(char transa, char transb, int64_t m, int64_t n, int64_t k,
                            double alpha, const double* A, int64_t lda, const double* B,
                            int64_t ldb, double beta, const double* C0, int64_t ldc, int slices,
                            int bits, int64_t kseg, const int64_t* rows, int64_t nrows,
                            double* out, int64_t ldo, int nthreads) {
  int ta = oz_trans(transa), tb = oz_trans(transb);
  if (ta < 0) return 1;
  if (tb < 0) return 2;
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  if (lda < ((ta ? k : m) > 1 ? (ta ? k : m) : 1)) return 8;
  if (ldb < ((tb ? n : k) > 1 ? (tb ? n : k) : 1)) return 10;
  if (ldc < (m > 1 ? m : 1)) return 13;
  if (!rows) nrows = m;
  if (rows)
    for (int64_t r = 0; r < nrows; ++r)
      if (rows[r] < 0 || rows[r] >= m) return 15;
  if (ldo < (nrows > 1 ? nrows : 1)) return 17;
  if (slices < 1 || slices > 9 || bits < 1 || bits > 8 || slices * bits > 63) return 18;
  if (kseg < 1) return 19;
  if (m == 0 || n == 0 || nrows == 0) return 0;

  if (alpha == 0.0 || k == 0) { /* quick return: C := beta*C */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        out[j * ldo + r] = (beta == 0.0) ? 0.0 : beta * C0[j * ldc + i];
      }
    return 0;
  }

  const int s = slices;
  int16_t* rdig = (int16_t*)malloc(sizeof(int16_t) * (size_t)nrows * s * (size_t)k);
  int* rsig = (int*)malloc(sizeof(int) * (size_t)nrows);
  int* rbad = (int*)malloc(sizeof(int) * (size_t)nrows);
  if (!rdig || !rsig || !rbad) {
    free(rdig); free(rsig); free(rbad);
    return -2;
  }
  ozjob_t T;
  memset(&T, 0, sizeof(T));
  T.ta = ta; T.tb = tb; T.s = s; T.bits = bits;
  T.m = m; T.n = n; T.k = k; T.kseg = kseg;
  T.alpha = alpha; T.beta = beta;
  T.A = A; T.B = B; T.C0 = C0;
  T.lda = lda; T.ldb = ldb; T.ldc = ldc;
  T.rows = rows; T.nrows = nrows;
  T.out = out; T.ldo = ldo;

  /* steps 1 and 2 for the requested rows of op(A) */
  int32_t dg[16];
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows ? rows[r] : r;
    int sig = 0, bad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      double v = oz_a(&T, i, p);
      if (!isfinite(v)) { bad = 1; continue; }
      if (v != 0.0) {
        int e = oracle_ozaki_exponent(v);
        if (!any || e > sig) sig = e;
        any = 1;
      }
    }
    rsig[r] = sig;
    rbad[r] = bad;
    for (int64_t p = 0; p < k; ++p) {
      double v = oz_a(&T, i, p);
      if (!isfinite(v)) v = 0.0;
      oracle_ozaki_split(v, sig, s, bits, dg);
      for (int t = 0; t < s; ++t) rdig[((size_t)r * s + t) * k + p] = (int16_t)dg[t];
    }
  }
  T.rdig = rdig; T.rsig = rsig; T.rbad = rbad;

  /* steps 3 and 4, threaded over columns */
  if (nthreads <= 0) {
    long nc = sysconf(_SC_NPROCESSORS_ONLN);
    nthreads = nc > 0 ? (int)nc : 1;
  }
  if (nthreads > 256) nthreads = 256;
  if (n < nthreads) nthreads = (int)n;
  ozjob_t jobs[256];
  pthread_t th[256];
  int started[256];
  int64_t per = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = T;
    jobs[t].j0 = t * per < n ? t * per : n;
    jobs[t].j1 = (t + 1) * per < n ? (t + 1) * per : n;
    started[t] = 0;
  }
  for (int t = 1; t < nthreads; ++t) started[t] = (pthread_create(&th[t], NULL, oz_run, &jobs[t]) == 0);
  oz_run(&jobs[0]);
  int err = jobs[0].err;
  for (int t = 1; t < nthreads; ++t) {
    if (started[t]) pthread_join(th[t], NULL);
    else oz_run(&jobs[t]);
    if (jobs[t].err) err = jobs[t].err;
  }
  free(rdig); free(rsig); free(rbad);
  return err;
}
