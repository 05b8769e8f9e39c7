/* gbdcpu.h -- the paper's own CPU method as a host-side DGEMM: the GotoBLAS algorithm as
 * refactored in BLIS (five loops around a micro-kernel, with packing), parallelised with
 * OpenMP.  It is a context baseline for the GPU library (include/gbdgemm.h) on the host
 * cores, not part of the GPU path.
 *
 * Operation (Section 1.2): C := alpha * op(A) * op(B) + beta * C, op(X) = X or X^T, with
 * the BLAS argument list; column-major storage with leading dimensions (Section 2.1).
 * Algorithm (Section 3.1, figure "blis_gemm"): loop 5 over n in steps of nc, loop 4 over k
 * in steps of kc (the kc x nc block of op(B) packed into nr-wide micro-panels), loop 3
 * over m in steps of mc (the mc x kc block of op(A) packed into mr-tall micro-panels),
 * loops 2 and 1 over the nr- and mr-wide micro-panels, loop 0 the micro-kernel's rank-1
 * updates of an mr x nr block of C held in registers.  Parallelisation (Section 4): the
 * packing of op(B) and loop 3 are shared among the threads.
 */
#ifndef GBDCPU_H
#define GBDCPU_H

#include <stdint.h>

#if defined(__GNUC__)
#define GBDCPU_API __attribute__((visibility("default")))
#else
#define GBDCPU_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* C := alpha op(A) op(B) + beta C on the host cores.
 *
 * transa, transb: 'N'/'n' (op(X) = X) or 'T'/'t'/'C'/'c' (op(X) = X^T; real data).
 * m, n, k: op(A) is m x k, op(B) is k x n, C is m x n.
 * A, B, C: HOST pointers, column-major; element (i, j) of X is X[i + j * ldx].  The caller
 *   owns them; A and B are only read, C is read (unless beta == 0) and written.
 * lda >= max(1, rows of A as stored), ldb likewise, ldc >= max(1, m).
 * threads: the OpenMP threads to use (<= 0: OpenMP's default).  The result does not depend
 *   on it: every element of C is summed in the same order whatever the thread count.
 *
 * Quick returns (reference BLAS): m == 0 or n == 0, or (alpha == 0 or k == 0) with
 * beta == 1, return at once; alpha == 0 or k == 0 gives C := beta C with A and B not read;
 * beta == 0 means C is not read (NaN in C does not propagate).
 *
 * Rounding: each element is the sum over k in increasing order, in blocks of kc: a block's
 * products summed in a register, then C := alpha * block + beta * C0 (first block) or
 * C := alpha * block + C.  The error is within (k + 2) u (|alpha| |op(A)| |op(B)| +
 * |beta| |C0|), u = 2^-53 (fused multiply-adds where the compiler forms them only lower it).
 *
 * Returns 0, the reference-BLAS index of the first invalid argument (1 transa, 2 transb,
 * 3 m, 4 n, 5 k, 8 lda, 10 ldb, 13 ldc), or -1 when the packing buffers cannot be
 * allocated (C untouched).
 */
GBDCPU_API int gbd_cpu_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                             const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                             int64_t ldc, int threads);

/* The blocking parameters of gbd_cpu_dgemm: mc, kc, nc (cache blocks) and mr, nr (the
 * micro-kernel's register block).  Any pointer may be NULL. */
GBDCPU_API void gbd_cpu_dgemm_blocking(int* mc, int* kc, int* nc, int* mr, int* nr);

/* The threads gbd_cpu_dgemm uses for threads <= 0 (1 when built without OpenMP). */
GBDCPU_API int gbd_cpu_max_threads(void);

#ifdef __cplusplus
}
#endif

#endif /* GBDCPU_H */
