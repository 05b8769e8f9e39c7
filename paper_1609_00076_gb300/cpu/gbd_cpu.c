/* gbd_cpu.c -- host DGEMM by the GotoBLAS algorithm as refactored in BLIS (Section 3.1, the
 * five loops of figure "blis_gemm"), parallelised with OpenMP (Section 4).  The GPU library
 * does not use it: it is the paper's own method on the host cores, measured beside the GPU
 * paths as context.
 *
 * Blocking (the parameters the paper derives from the caches):
 *   nr x kc micro-panel of op(B) (12 KiB) stays in the L1 cache across the micro-panels of A;
 *   mc x kc block of op(A) (256 KiB) stays in a core's L2 cache across loop 2;
 *   kc x nc block of op(B) (6 MiB) stays in the shared last-level cache across loop 3;
 *   mr x nr = 8 x 6 block of C lives in registers during loop 0 (24 two-wide or 12 four-wide
 *   vector accumulators; the compiler vectorises the mr direction).
 * Packing (the arrows of the paper's figure): op(A) into mr-tall micro-panels with each
 * column of mr contiguous, op(B) into nr-wide micro-panels with each row of nr contiguous,
 * both zero-padded past the matrix, so the micro-kernel always runs a full mr x nr block and
 * only its write-back is masked.
 * Threads: each (jc, pc) step packs op(B) with the micro-panels shared out among the
 * threads, then shares out loop 3; every thread packs its own block of op(A).
 * Summation order: every element of C is summed over k in increasing order, in blocks of kc
 * (loop 4 runs in order, outside the parallel loop), so the result does not depend on the
 * thread count.
 */
#include "gbdcpu.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { MR = 8, NR = 6, MC = 128, KC = 256, NC = 3072 };

static int trans_code(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}

static int64_t max1(int64_t x) { return x > 1 ? x : 1; }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

/* rows [i0, i0 + mc) and columns [p0, p0 + kc) of op(A) into ceil(mc / MR) micro-panels;
 * element (i, p) of panel q at Ap[q * MR * kc + p * MR + i] */
static void pack_a(int ta, const double* A, int64_t lda, int64_t i0, int64_t p0, int mc, int kc, double* Ap) {
  for (int ir = 0; ir < mc; ir += MR) {
    double* dst = Ap + (int64_t)ir * kc;
    const int rows = mc - ir < MR ? mc - ir : MR;
    if (!ta) {  /* op(A) = A: (i, p) at A[i + p lda], i contiguous */
      for (int p = 0; p < kc; ++p) {
        const double* src = A + (i0 + ir) + (p0 + p) * lda;
        for (int i = 0; i < rows; ++i) dst[p * MR + i] = src[i];
        for (int i = rows; i < MR; ++i) dst[p * MR + i] = 0.0;
      }
    } else {  /* op(A) = A^T: (i, p) at A[p + i lda], p contiguous */
      for (int i = 0; i < rows; ++i) {
        const double* src = A + p0 + (i0 + ir + i) * lda;
        for (int p = 0; p < kc; ++p) dst[p * MR + i] = src[p];
      }
      for (int i = rows; i < MR; ++i)
        for (int p = 0; p < kc; ++p) dst[p * MR + i] = 0.0;
    }
  }
}

/* micro-panel q of the kc x nc block of op(B) at (p0, j0): columns j0 + q NR + [0, NR);
 * element (p, j) at Bq[p * NR + j] */
static void pack_b_panel(int tb, const double* B, int64_t ldb, int64_t p0, int64_t j0, int nc, int kc, int q,
                         double* Bq) {
  const int jr = q * NR;
  const int cols = nc - jr < NR ? nc - jr : NR;
  if (!tb) {  /* op(B) = B: (p, j) at B[p + j ldb], p contiguous */
    for (int j = 0; j < cols; ++j) {
      const double* src = B + p0 + (j0 + jr + j) * ldb;
      for (int p = 0; p < kc; ++p) Bq[p * NR + j] = src[p];
    }
    for (int j = cols; j < NR; ++j)
      for (int p = 0; p < kc; ++p) Bq[p * NR + j] = 0.0;
  } else {  /* op(B) = B^T: (p, j) at B[j + p ldb], j contiguous */
    for (int p = 0; p < kc; ++p) {
      const double* src = B + (j0 + jr) + (p0 + p) * ldb;
      for (int j = 0; j < cols; ++j) Bq[p * NR + j] = src[j];
      for (int j = cols; j < NR; ++j) Bq[p * NR + j] = 0.0;
    }
  }
}

/* Loop 0: the MR x NR block acc = sum over p of the rank-1 updates a(:, p) b(p, :), then the
 * rows < mr and columns < nr of it into C: C := alpha acc + beta C0 on the first k block
 * (C0 not read when beta == 0), C := alpha acc + C on the later ones. */
static void micro_kernel(int kc, const double* restrict a, const double* restrict b, double alpha, double beta,
                         int first, double* restrict c, int64_t ldc, int mr, int nr) {
  double acc[NR][MR];
  for (int j = 0; j < NR; ++j)
    for (int i = 0; i < MR; ++i) acc[j][i] = 0.0;
  for (int p = 0; p < kc; ++p) {
    const double* ap = a + p * MR;
    const double* bp = b + p * NR;
#pragma GCC unroll 6
    for (int j = 0; j < NR; ++j) {
      const double bj = bp[j];
#pragma GCC unroll 8
      for (int i = 0; i < MR; ++i) acc[j][i] += ap[i] * bj;
    }
  }
  for (int j = 0; j < nr; ++j) {
    double* cj = c + j * ldc;
    for (int i = 0; i < mr; ++i) {
      const double v = alpha * acc[j][i];
      if (!first) cj[i] = v + cj[i];
      else cj[i] = beta == 0.0 ? v : v + beta * cj[i];
    }
  }
}

static void* alloc_aligned(size_t bytes) {
  const size_t a = 64;
  return aligned_alloc(a, (bytes + a - 1) / a * a);
}

int gbd_cpu_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void gbd_cpu_dgemm_blocking(int* mc, int* kc, int* nc, int* mr, int* nr) {
  if (mc) *mc = MC;
  if (kc) *kc = KC;
  if (nc) *nc = NC;
  if (mr) *mr = MR;
  if (nr) *nr = NR;
}

int gbd_cpu_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                  int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int threads) {
  const int ta = trans_code(transa), tb = trans_code(transb);
  if (ta < 0) return 1;
  if (tb < 0) return 2;
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  if (lda < max1(ta ? k : m)) return 8;
  if (ldb < max1(tb ? n : k)) return 10;
  if (ldc < max1(m)) return 13;
  if (m == 0 || n == 0 || ((alpha == 0.0 || k == 0) && beta == 1.0)) return 0;
  if (alpha == 0.0 || k == 0) {  /* C := beta C, A and B not read */
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < m; ++i) C[i + j * ldc] = beta == 0.0 ? 0.0 : beta * C[i + j * ldc];
    return 0;
  }
  const int nt = threads > 0 ? threads : gbd_cpu_max_threads();
  const int nc_max = (int)min64(NC, (n + NR - 1) / NR * NR);
  const int kc_max = (int)min64(KC, k);
  const int mc_max = (int)min64(MC, (m + MR - 1) / MR * MR);
  double* Bp = (double*)alloc_aligned(sizeof(double) * (size_t)kc_max * (size_t)((nc_max + NR - 1) / NR * NR));
  double* Apool = (double*)alloc_aligned(sizeof(double) * (size_t)mc_max * (size_t)kc_max * (size_t)nt);
  if (!Bp || !Apool) {
    free(Bp);
    free(Apool);
    return -1;
  }
  const int64_t mblocks = (m + MC - 1) / MC;
  for (int64_t jc = 0; jc < n; jc += NC) {              /* loop 5 */
    const int nc = (int)min64(NC, n - jc);
    const int npanels = (nc + NR - 1) / NR;
    for (int64_t pc = 0; pc < k; pc += KC) {            /* loop 4 */
      const int kc = (int)min64(KC, k - pc);
      const int first = pc == 0;
#pragma omp parallel num_threads(nt)
      {
#ifdef _OPENMP
        double* Ap = Apool + (size_t)omp_get_thread_num() * (size_t)mc_max * (size_t)kc_max;
#else
        double* Ap = Apool;
#endif
#pragma omp for schedule(static)
        for (int q = 0; q < npanels; ++q)  /* pack op(B)(pc:pc+kc, jc:jc+nc) */
          pack_b_panel(tb, B, ldb, pc, jc, nc, kc, q, Bp + (size_t)q * NR * kc);
        /* the implied barrier: every panel of op(B) is packed */
#pragma omp for schedule(dynamic)
        for (int64_t ib = 0; ib < mblocks; ++ib) {     /* loop 3 */
          const int64_t ic = ib * MC;
          const int mc = (int)min64(MC, m - ic);
          pack_a(ta, A, lda, ic, pc, mc, kc, Ap);
          for (int jr = 0; jr < nc; jr += NR)           /* loop 2 */
            for (int ir = 0; ir < mc; ir += MR)         /* loop 1 */
              micro_kernel(kc, Ap + (size_t)ir * kc, Bp + (size_t)jr * kc, alpha, beta, first,
                           C + (ic + ir) + (jc + jr) * ldc, ldc, mc - ir < MR ? mc - ir : MR,
                           nc - jr < NR ? nc - jr : NR);
        }
      }
    }
  }
  free(Bp);
  free(Apool);
  return 0;
}
