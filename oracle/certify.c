/*
 * certify.c -- plain CPU statement of the certified precision choice of the two emulations
 * of double-precision GEMM (the split one of Ozaki, Ogita, Oishi and Rump, and the modular
 * "Ozaki scheme II" of Ozaki, Uchino and Imamura), for C := alpha op(A) op(B) + beta C
 * (Section 1.2 of the paper).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): nothing on the product path uses it, and it
 * shares no code with the CUDA library.
 *
 * Both emulations scale row i of op(A) by 2^-sigma_i and column j of op(B) by 2^-tau_j
 * (frexp exponents, as in ozaki_model.c / ozaki_mod_model.c), so every scaled entry
 * a^_ip = a_ip 2^-sigma_i, b^_pj = b_pj 2^-tau_j has magnitude below 1.  With
 * mu_i = sum_p |a^_ip|, nu_j = sum_p |b^_pj| and G^_ij = sum_p |a^_ip||b^_pj|, the truncation
 * error of element (i, j), in units of 2^(sigma_i + tau_j), is at most
 *
 *     split, s digit slices of 7 bits:  2^-7s (mu_i + nu_j + (s - 1)(1 + 2^-7) k)
 *     modular, t integer bits:          2^(-t-1) (mu_i + nu_j + k 2^(-t-1))
 *
 * (the rounding of every scaled entry is at most 2^(-t-1), the truncated digit tail below
 * 2^-7s, and the dropped digit pairs are those of levels above s + 1).  Every one of these
 * errors vanishes with its entry, and an entry of magnitude at least theta_i (the smallest
 * non-zero |a^_ip| of row i; phi_j likewise for column j of op(B)) is at least theta_i/|a^_ip|
 * times smaller than its own term of G^: so the sums over p may be replaced by
 *     nu_j -> min(nu_j, G^_ij / theta_i),   mu_i -> min(mu_i, G^_ij / phi_j),
 *     k    -> min(k, G^_ij / (theta_i phi_j))       (the count of p with both entries non-zero),
 * which is what makes triangular, sparse and block operands certifiable.  The FP64 target is
 * the componentwise bound tol (|alpha| |A||B| + |beta||C0|); the beta term only loosens it,
 * so it is met when the truncation error stays below (tol - r u) G_ij, where r u (u = 2^-53)
 * is set aside for the final roundings: r = 3 for the modular emulation (the conversion of
 * the exact integer, the product with beta C0 and the fused update) and r = 3 g + 3 for the
 * split one, g = ceil(k / 8192) segments of at most three fused group updates.
 *
 * The certified choice is the smallest s (t) for which that holds on every element with
 * G_ij > 0 whose row and column are finite.  An element with G_ij = 0 has no error: each
 * of its terms has a zero factor, which both emulations represent exactly.  Independently,
 * when every scaled entry of op(A) is an integer multiple of 2^-tA and every one of op(B) of
 * 2^-tB, the integers of the modular emulation are exact for t >= max(tA, tB), and the digits
 * of the split one are exact with ceil(tA/7) and ceil(tB/7) digits, whose products all lie on
 * levels up to ceil(tA/7) + ceil(tB/7); then only the final roundings remain, which the
 * target must still cover (2 u for the modular emulation, (g ceil(s/4) + 1) u for the split).
 * The choice takes the smaller of the two.  The modular emulation also needs the fewest
 * leading moduli of {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199,
 * 197, 193} whose product exceeds twice a bound of every |(A'B')_ij|, A'_ip = rn(a^_ip 2^t) and
 * B'_pj = rn(b^_pj 2^t) the rounded integers, so that each element is the representative of its
 * residues in (-M/2, M/2]; more than 16, or t above 62, is infeasible.  The bound is the smaller
 * of k 2^(2t) (every |A'_ip|, |B'_pj| <= 2^t) and, by Cauchy-Schwarz and |A'_ip - a^_ip 2^t| <= 1/2,
 *     (2^t alpha + sqrt(k)/2) (2^t beta + sqrt(k)/2),
 * alpha^2 = max_i sum_p a^_ip^2 over every row of op(A), beta^2 = max_j sum_p b^_pj^2 over every
 * column of op(B) (finite entries).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
  int t_cert;   /* modular: smallest t in 1..62 whose bound holds on every element; 63: none */
  int t_exact;  /* smallest t making every scaled entry an integer; 0: both operands zero; 63: above 62 */
  int t;        /* the choice (63: infeasible) */
  int moduli;   /* moduli for t at k (0: infeasible) */
  int s_cert;   /* split: smallest s in 1..9 whose bound holds on every element; 10: none */
  int s_exact;  /* s with exact digits and every product kept; 10: above 9 */
  int s;        /* the choice (10: infeasible) */
  int pad;
  double rho;   /* max over the elements of (min(mu_i, G^/phi_j) + min(nu_j, G^/theta_i)) / G^_ij */
  double gamma; /* max over the elements of min(k, G^/(theta_i phi_j)) / (k G^_ij) */
  double alpha2; /* max over all rows of op(A) of sum_p a^_ip^2 */
  double beta2;  /* max over all columns of op(B) of sum_p b^_pj^2 */
} oracle_cert_t;

static const int oc_moduli[16] = {256, 255, 253, 251, 247, 241, 239, 233,
                                  229, 227, 223, 217, 211, 199, 197, 193};

static int oc_trans(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}

static int oc_exponent(double x) {
  int e = 0;
  (void)frexp(x, &e);
  return e;
}

/* exponent of the lowest set bit of a finite non-zero x: x = odd * 2^lambda */
static int oc_lowbit(double x) {
  int e = 0;
  const double f = frexp(fabs(x), &e); /* |x| = f 2^e, f in [0.5, 1) with at most 53 bits */
  int64_t F = (int64_t)ldexp(f, 53);   /* exact integer */
  int lam = e - 53;
  while ((F & 1) == 0) {
    F >>= 1;
    ++lam;
  }
  return lam;
}

/* fewest leading moduli whose product exceeds 2 k 2^(2t); 0 when none of the 16 does */
int oracle_cert_moduli(int t, int64_t k) {
  if (t < 1 || t > 62 || k < 1) return 0;
  /* compare logarithms with a margin, then decide exactly with 128-bit integers */
  unsigned __int128 M = 1;
  int kb = 0;
  while (((int64_t)1 << kb) < k) ++kb;
  if (2 * t + kb + 1 >= 127) return 0;
  const unsigned __int128 need = ((unsigned __int128)2 * (unsigned __int128)k) << (2 * t);
  for (int l = 0; l < 16; ++l) {
    M *= (unsigned __int128)oc_moduli[l];
    if (M > need) return l + 1;
  }
  return 0;
}

/* fewest leading moduli whose product exceeds 2 min(k 2^(2t), (2^t alpha + sqrt(k)/2)(2^t beta + sqrt(k)/2));
   0 when none of the 16 does */
int oracle_cert_moduli_cs(int t, int64_t k, double alpha2, double beta2) {
  const int nk = oracle_cert_moduli(t, k);
  if (t < 1 || t > 62 || k < 1 || !(alpha2 >= 0.0) || !(beta2 >= 0.0)) return nk;
  const long double h = sqrtl((long double)k) / 2.0L;
  const long double bound = (ldexpl(sqrtl((long double)alpha2), t) + h) * (ldexpl(sqrtl((long double)beta2), t) + h);
  if (!(bound < ldexpl((long double)k, 2 * t))) return nk;
  unsigned __int128 M = 1;
  for (int l = 0; l < 16; ++l) {
    M *= (unsigned __int128)oc_moduli[l];
    const long double Ml = (long double)(uint64_t)(M >> 64) * 18446744073709551616.0L + (long double)(uint64_t)M;
    if (Ml > 2.0L * bound) return (nk == 0 || l + 1 < nk) ? l + 1 : nk;
  }
  return nk;
}

/* Two-sum / two-product compensated sum of non-negative terms (Ogita, Rump, Oishi). */
typedef struct {
  double hi, lo;
} oc_acc;
static inline void oc_add(oc_acc* a, double x) {
  const double s = a->hi + x;
  const double bp = s - a->hi;
  a->lo += (a->hi - (s - bp)) + (x - bp);
  a->hi = s;
}
static inline void oc_add_prod(oc_acc* a, double x, double y) {
  const double p = x * y;
  const double e = fma(x, y, -p);
  oc_add(a, p);
  a->lo += e;
}

typedef struct {
  int ta, tb;
  int64_t m, n, k;
  const double *A, *B;
  int64_t lda, ldb;
  const int64_t* rows;
  int64_t nrows;
  const double* ra; /* [nrows][k] |a^| of the requested rows */
  const double* rmu;
  const double* rth; /* [nrows] theta_i: the smallest non-zero |a^_ip| (0 for a zero row) */
  const int* rbad;
  double tau_mod, tau_split;
  int64_t j0, j1;
  /* results of this worker */
  int t_cert, s_cert;
  double rho, gamma;
  int err;
} ocjob_t;

static inline double oc_b(const ocjob_t* J, int64_t p, int64_t j) {
  return J->tb ? J->B[p * J->ldb + j] : J->B[j * J->ldb + p];
}

static void* oc_run(void* arg) {
  ocjob_t* J = (ocjob_t*)arg;
  const int64_t k = J->k;
  double* cb = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  if (!cb) {
    J->err = -2;
    return NULL;
  }
  const double kd = (double)k;
  for (int64_t j = J->j0; j < J->j1; ++j) {
    int tau = 0, cbad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = oc_b(J, p, j);
      if (!isfinite(v)) { cbad = 1; continue; }
      if (v != 0.0) {
        const int e = oc_exponent(v);
        if (!any || e > tau) tau = e;
        any = 1;
      }
    }
    if (cbad) continue; /* the column's results are NaN: no bound applies */
    oc_acc nu = {0.0, 0.0};
    for (int64_t p = 0; p < k; ++p) {
      const double v = oc_b(J, p, j);
      cb[p] = ldexp(fabs(v), -tau);
      oc_add(&nu, cb[p]);
    }
    const double nuj = nu.hi + nu.lo;
    double phj = 0.0; /* phi_j: the smallest non-zero |b^_pj| */
    for (int64_t p = 0; p < k; ++p)
      if (cb[p] > 0.0 && (phj == 0.0 || cb[p] < phj)) phj = cb[p];
    for (int64_t r = 0; r < J->nrows; ++r) {
      if (J->rbad[r]) continue;
      const double* a = J->ra + r * k;
      oc_acc g = {0.0, 0.0};
      for (int64_t p = 0; p < k; ++p) oc_add_prod(&g, a[p], cb[p]);
      const double G = g.hi + g.lo;
      if (!(G > 0.0)) continue; /* every term has a zero factor: no error */
      const double th = J->rth[r];
      /* the error sums over p, each term vanishing with its entry (zero-aware) */
      const double s1 = fmin(nuj, G / th), s2 = fmin(J->rmu[r], G / phj), s3 = fmin(kd, G / (th * phj));
      const double mn = s1 + s2;
      const double rho = mn / G, gam = s3 / (kd * G);
      if (rho > J->rho) J->rho = rho;
      if (gam > J->gamma) J->gamma = gam;
      int t = 1;
      while (t <= 62 && !(ldexp(1.0, -t - 1) * (mn + s3 * ldexp(1.0, -t - 1)) <= J->tau_mod * G)) ++t;
      if (t > J->t_cert) J->t_cert = t;
      int s = 1;
      while (s <= 9 && !(ldexp(1.0, -7 * s) * (mn + (s - 1) * (1.0 + ldexp(1.0, -7)) * s3) <= J->tau_split * G)) ++s;
      if (s > J->s_cert) J->s_cert = s;
    }
  }
  free(cb);
  return NULL;
}

/*
 * The certified choice for rows rows[0..nrows) of op(A) (all m rows when rows == NULL)
 * against every column of op(B), for the target tol (tol <= 0: 2 k 2^-53).  The exactness
 * widths tA, tB cover all of op(A) and op(B).  Returns 0, a BLAS argument index (1, 2, 3,
 * 4, 5, 8, 10; 13 rows), or -2 (no memory).
 */
int oracle_certify(char transa, char transb, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                   const double* B, int64_t ldb, double tol, const int64_t* rows, int64_t nrows, int nthreads,
                   oracle_cert_t* out) {
  const int ta = oc_trans(transa), tb = oc_trans(transb);
  if (ta < 0) return 1;
  if (tb < 0) return 2;
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  if (lda < ((ta ? k : m) > 1 ? (ta ? k : m) : 1)) return 8;
  if (ldb < ((tb ? n : k) > 1 ? (tb ? n : k) : 1)) return 10;
  if (!rows) nrows = m;
  if (nrows < 0) return 13;
  for (int64_t r = 0; r < nrows; ++r)
    if (rows && (rows[r] < 0 || rows[r] >= m)) return 13;
  memset(out, 0, sizeof(*out));
  const double u = ldexp(1.0, -53);
  const double kd = (double)(k > 0 ? k : 1);
  if (!(tol > 0.0)) tol = 2.0 * kd * u;
  const int64_t segs = (k + 8191) / 8192;

  /* exactness widths and largest scaled square sums over all of op(A) (rows) and op(B) (columns) */
  int tA = 0, tB = 0;
  double alpha2 = 0.0, beta2 = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    int sig = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      if (isfinite(v) && v != 0.0) {
        const int e = oc_exponent(v);
        if (!any || e > sig) sig = e;
        any = 1;
      }
    }
    oc_acc sq = {0.0, 0.0};
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      if (isfinite(v) && v != 0.0) {
        const int w = sig - oc_lowbit(v);
        if (w > tA) tA = w;
        const double x = ldexp(fabs(v), -sig);
        oc_add_prod(&sq, x, x);
      }
    }
    if (sq.hi + sq.lo > alpha2) alpha2 = sq.hi + sq.lo;
  }
  for (int64_t j = 0; j < n; ++j) {
    int tau = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = tb ? B[p * ldb + j] : B[j * ldb + p];
      if (isfinite(v) && v != 0.0) {
        const int e = oc_exponent(v);
        if (!any || e > tau) tau = e;
        any = 1;
      }
    }
    oc_acc sq = {0.0, 0.0};
    for (int64_t p = 0; p < k; ++p) {
      const double v = tb ? B[p * ldb + j] : B[j * ldb + p];
      if (isfinite(v) && v != 0.0) {
        const int w = tau - oc_lowbit(v);
        if (w > tB) tB = w;
        const double x = ldexp(fabs(v), -tau);
        oc_add_prod(&sq, x, x);
      }
    }
    if (sq.hi + sq.lo > beta2) beta2 = sq.hi + sq.lo;
  }

  /* the scaled magnitudes of the requested rows */
  double* ra = (double*)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1) * (size_t)(k > 0 ? k : 1));
  double* rmu = (double*)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1));
  double* rth = (double*)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1));
  int* rbad = (int*)malloc(sizeof(int) * (size_t)(nrows > 0 ? nrows : 1));
  if (!ra || !rmu || !rth || !rbad) {
    free(ra); free(rmu); free(rth); free(rbad);
    return -2;
  }
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows ? rows[r] : r;
    int sig = 0, bad = 0, any = 0;
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      if (!isfinite(v)) { bad = 1; continue; }
      if (v != 0.0) {
        const int e = oc_exponent(v);
        if (!any || e > sig) sig = e;
        any = 1;
      }
    }
    oc_acc mu = {0.0, 0.0};
    for (int64_t p = 0; p < k; ++p) {
      const double v = ta ? A[i * lda + p] : A[p * lda + i];
      ra[r * k + p] = isfinite(v) ? ldexp(fabs(v), -sig) : 0.0;
      oc_add(&mu, ra[r * k + p]);
    }
    rmu[r] = mu.hi + mu.lo;
    rbad[r] = bad;
    double th = 0.0;
    for (int64_t p = 0; p < k; ++p)
      if (ra[r * k + p] > 0.0 && (th == 0.0 || ra[r * k + p] < th)) th = ra[r * k + p];
    rth[r] = th;
  }

  int t_cert = 1, s_cert = 1;
  double rho = 0.0, gamma = 0.0;
  int rc = 0;
  if (m > 0 && n > 0 && k > 0 && nrows > 0) {
    if (nthreads < 1) {
      long c = sysconf(_SC_NPROCESSORS_ONLN);
      nthreads = c > 0 ? (int)c : 1;
    }
    if (nthreads > n) nthreads = (int)n;
    ocjob_t* jobs = (ocjob_t*)calloc((size_t)nthreads, sizeof(ocjob_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) rc = -2;
    for (int w = 0; w < nthreads && !rc; ++w) {
      ocjob_t* J = &jobs[w];
      J->ta = ta; J->tb = tb;
      J->m = m; J->n = n; J->k = k;
      J->A = A; J->B = B; J->lda = lda; J->ldb = ldb;
      J->rows = rows; J->nrows = nrows;
      J->ra = ra; J->rmu = rmu; J->rth = rth; J->rbad = rbad;
      J->tau_mod = tol - 3.0 * u;
      J->tau_split = tol - (3.0 * (double)segs + 3.0) * u;
      J->j0 = n * w / nthreads;
      J->j1 = n * (w + 1) / nthreads;
      J->t_cert = 1;
      J->s_cert = 1;
      if (pthread_create(&th[w], NULL, oc_run, J) != 0) {
        oc_run(J);
        th[w] = 0;
      }
    }
    for (int w = 0; w < nthreads && jobs && th; ++w) {
      if (th[w]) pthread_join(th[w], NULL);
      if (jobs[w].err) rc = jobs[w].err;
      if (jobs[w].t_cert > t_cert) t_cert = jobs[w].t_cert;
      if (jobs[w].s_cert > s_cert) s_cert = jobs[w].s_cert;
      if (jobs[w].rho > rho) rho = jobs[w].rho;
      if (jobs[w].gamma > gamma) gamma = jobs[w].gamma;
    }
    free(jobs);
    free(th);
  }
  free(ra); free(rmu); free(rth); free(rbad);
  if (rc) return rc;

  const int tx = tA > tB ? tA : tB;
  out->t_cert = t_cert;
  out->t_exact = tx > 62 ? 63 : tx;
  int t = t_cert;
  if (tx <= 62 && tol >= 2.0 * u) {
    const int te = tx < 1 ? 1 : tx;
    if (te < t) t = te;
  }
  out->moduli = t <= 62 ? oracle_cert_moduli_cs(t, k > 0 ? k : 1, alpha2, beta2) : 0;
  out->t = out->moduli ? t : 63;

  const int dA = (tA + 6) / 7, dB = (tB + 6) / 7;
  int sx = dA + dB - 1;
  if (sx < 1) sx = 1;
  out->s_cert = s_cert;
  out->s_exact = sx > 9 ? 10 : sx;
  int s = s_cert;
  if (sx <= 9 && tol >= ((double)segs * (double)((sx + 3) / 4) + 1.0) * u && sx < s) s = sx;
  out->s = s;
  out->rho = rho;
  out->gamma = gamma;
  out->alpha2 = alpha2;
  out->beta2 = beta2;
  return 0;
}
