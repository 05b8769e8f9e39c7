/*
 * gbdgemm.h -- C ABI of the GB300 (sm_103a) double-precision GEMM library.
 *
 * The operation is the BLAS dgemm of the BLISlab paper (Huang and van de Geijn,
 * FLAME Working Note #80, Section 1.2):
 *
 *     C := alpha * op(A) * op(B) + beta * C,     op(X) = X  or  X^T,
 *
 * with C m x n, op(A) m x k and op(B) k x n.  All matrices are column-major with
 * a leading dimension (Section 2.1): element (i, j) of X is X[i + j*ldx], and the
 * matrix may sit inside a larger array (an interior pointer with ldx larger than
 * its row count is legal).  A is stored m x k when transa is 'N' and k x m when
 * it is 'T'; B is stored k x n for 'N' and n x k for 'T'.
 *
 * Conventions shared by every entry point:
 *  - All matrix pointers are DEVICE pointers owned by the caller; the library
 *    never allocates, frees or retains them.  A and B must not overlap C.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream) unless stated otherwise.
 *  - transa/transb accept 'N','n','T','t','C','c'; 'C' means 'T' for real data.
 *  - Quick returns follow the reference BLAS: nothing is done when m == 0 or
 *    n == 0, or when (alpha == 0 or k == 0) and beta == 1.  When alpha == 0 or
 *    k == 0, C := beta*C and A, B are not read.  When beta == 0, C is not read
 *    on input (NaN/Inf already in C do not propagate).
 *  - Return value: 0 on success; a positive value is the 1-based position of
 *    the first invalid argument in the dgemm argument list (reference-BLAS
 *    xerbla numbering: 1 transa, 2 transb, 3 m, 4 n, 5 k, 8 lda, 10 ldb,
 *    13 ldc); a negative value is one of the GBD_ERR_* codes below.  No
 *    exception ever crosses this boundary.
 *  - Results are deterministic: the same call on the same inputs gives the
 *    same bits, independent of other work on the device.
 */
#ifndef GBDGEMM_H
#define GBDGEMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GBD_API __attribute__((visibility("default")))
#else
#define GBD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define GBD_OK 0
#define GBD_ERR_CUDA (-1)        /* a CUDA runtime/driver call failed (see gbd_last_error) */
#define GBD_ERR_WORKSPACE (-2)   /* workspace missing, too small or misaligned */
#define GBD_ERR_TIMEOUT (-3)     /* a bounded device-side wait gave up (watchdog) */
#define GBD_ERR_DEVICE (-4)      /* the current device is not an sm_103 GPU */
#define GBD_ERR_LIMIT (-5)       /* a size is outside what the kernel supports */
#define GBD_ERR_ARG (-6)         /* an argument outside the dgemm list is invalid */

/* Library version, major*10000 + minor*100 + patch. */
GBD_API int gbd_version(void);

/* Human-readable text for the last error raised by the calling thread (never NULL). */
GBD_API const char* gbd_last_error(void);

/*
 * Native double-precision GEMM on the FP64 tensor-core MMA (mma.sync f64).
 *
 * Computes C := alpha*op(A)*op(B) + beta*C (Section 1.2) with FP64 products and
 * FP64 accumulation in a fixed order; the epilogue forms fma(alpha, acc, beta*c)
 * (alpha*acc when beta == 0).  Tiles are staged in shared memory by the Tensor
 * Memory Accelerator when A and B start on 16-byte boundaries and lda, ldb are
 * even, and by per-element asynchronous copies otherwise (odd leading
 * dimensions and interior pointers such as the paper's lda = 3 example).
 * Arguments are those of the BLAS call; A, B, C are device pointers; lda >=
 * max(1, rows of A as stored), ldb likewise, ldc >= max(1, m).
 * Returns 0, a BLAS argument index, or GBD_ERR_*.  Asynchronous on stream.
 */
GBD_API int gbd_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                      double* C, int64_t ldc, void* stream);

/* Which path computed an emulated call (gbd_emu_info.path). */
#define GBD_PATH_NONE 0     /* a quick return: nothing was multiplied */
#define GBD_PATH_SPLIT 1    /* digit slices (gbd_dgemm_emu) */
#define GBD_PATH_MODULAR 2  /* residues (gbd_dgemm_emu_mod) */
#define GBD_PATH_NATIVE 3   /* gbd_dgemm_emu found the target out of its reach and ran gbd_dgemm */

/*
 * Report of one emulated call (filled when the `info` argument is not NULL).
 *
 * In automatic mode the precision is certified, not estimated: with sigma_i, tau_j the
 * row and column exponents, mu_i = sum_p |a_ip| 2^-sigma_i, nu_j = sum_p |b_pj| 2^-tau_j and
 * L_ij a guaranteed lower bound of (|op(A)||op(B)|)_ij 2^-(sigma_i + tau_j) computed on the
 * tensor cores, every element's a-priori truncation bound is at most `bound` times
 * (|op(A)||op(B)|)_ij, and `bound` plus the allowance for the final roundings stays within
 * the target.  Elements whose |A||B| terms all have a zero factor carry no error.
 */
typedef struct gbd_emu_info {
  int record_phases; /* input: non-zero to time the phases with CUDA events on `stream`
                        (the call then waits for its own completion before returning) */
  int slices;       /* split: digit slices per operand; modular: moduli; 0 for the native path */
  int digit_bits;   /* split: bits per digit (7); modular: integer bits t */
  int products;     /* tensor-core products: slices*(slices+1)/2 (split), the moduli (modular) */
  int path;         /* GBD_PATH_* */
  int exact;        /* automatic mode: 1 when every scaled entry is an integer at the chosen
                       precision, so the products are exact (integer inputs, for instance) */
  double rho;       /* automatic mode: max over elements of (mu_i + nu_j) / L_ij */
  double gamma;     /* automatic mode: max over elements of 1 / L_ij */
  double bound;     /* automatic mode: the certified componentwise relative bound of the truncation
                       error at the chosen precision (0 when exact) */
  double prep_ms;   /* record_phases: device time of the preparation and certification kernels */
  double gemm_ms;   /* record_phases: device time of the product kernels */
  double recon_ms;  /* record_phases, modular path: device time of the reconstruction of C from
                       the parked residues (after the products); 0 for the other paths */
} gbd_emu_info;

/*
 * Bytes of device workspace that gbd_dgemm_emu needs for an m x n x k problem
 * with `slices` digit slices per operand (0 = automatic: sized for the maximum,
 * 9).  Returns 0 for negative sizes.  Host-only; needs no GPU.
 */
GBD_API size_t gbd_dgemm_emu_workspace_size(int64_t m, int64_t n, int64_t k, int slices);

/*
 * Double-precision GEMM emulated on the BF16 tensor cores (tcgen05) with the
 * error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59,
 * 2012), in fixed-point digit form; the operation and the argument list are
 * those of gbd_dgemm (Section 1.2 of the paper).
 *
 * Steps: per-row exponents sigma_i of op(A) and per-column exponents tau_j of
 * op(B); `slices` digits of 7 bits per entry (truncation of a_ip 2^-sigma_i);
 * for each level g = 2..slices+1 the exact integer sum P_g of the digit
 * products with t + u = g, on tcgen05.mma with FP32 accumulation over chunks of
 * 1024 that is exact by construction; then C := beta*C and, for each segment of
 * 8192 of the inner dimension, the levels from the smallest in groups of up to
 * four: Y = sum_g P_g 2^(7(h-g)) exactly in 64-bit integers (h the group's
 * smallest level) and C := fma(alpha 2^(sigma_i + tau_j - 7h), Y, C) in FP64.
 *
 * slices: 1..9, or 0 for the certified automatic choice: the smallest count whose
 *   a-priori truncation bound, plus the final roundings, stays within `tol` times
 *   |alpha||op(A)||op(B)| on every element (tol <= 0 means the FP64 bound 2 k 2^-53), with
 *   (|op(A)||op(B)|)_ij bounded from below by a BF16 product of magnitude planes on the
 *   tensor cores (see gbd_emu_info); or the count at which the digits are exact.  When no
 *   count up to 9 can be certified the call computes C with gbd_dgemm instead (info->path =
 *   GBD_PATH_NATIVE), so the result always meets the target.  Automatic mode reads 16 bytes
 *   back from the device and therefore synchronises `stream`; with slices > 0 the call is
 *   fully asynchronous and the caller answers for the accuracy.
 * workspace: device memory of at least gbd_dgemm_emu_workspace_size(m, n, k,
 *   slices) bytes, 256-byte aligned, owned by the caller; its contents on entry
 *   do not matter and it must not be reused until the call has completed on
 *   `stream`.
 * info: optional report (may be NULL); its record_phases field is read on entry.
 * Rows of op(A) or columns of op(B) holding Inf or NaN give NaN in the matching
 * rows/columns of C.  Supported sizes: m, n < 4194240, k < 2^31.
 * Returns 0, a BLAS argument index, or GBD_ERR_* (GBD_ERR_WORKSPACE when the
 * workspace is missing, small or misaligned; GBD_ERR_ARG for a bad `slices`).
 */
GBD_API int gbd_dgemm_emu(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                          const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                          double* C, int64_t ldc, int slices, double tol, void* workspace,
                          size_t workspace_bytes, gbd_emu_info* info, void* stream);

/*
 * A guaranteed lower bound of |op(A)||op(B)|, the magnitude that scales the componentwise
 * error bound of every GEMM (Section 1.2's operation; the paper states no error analysis):
 * L_ij <= sum_p |op(A)_ip| |op(B)_pj|, computed on the tensor cores exactly as the automatic
 * modes of the emulations do to certify their precision.  Per row of op(A) and column of op(B)
 * the entries are scaled by the power of two of their largest magnitude and rounded toward
 * zero to BF16 (with a floor of 2^-63 relative to that largest magnitude, so that L_ij = 0
 * exactly when every term has a zero factor), multiplied with FP32 accumulation, and the
 * accumulation's possible overshoot and the floors are subtracted with downward rounding.
 * fp8: 0 for BF16 planes (8 significant bits, within about 2 % of |A||B| on well-scaled data),
 *   1 for FP8 E5M2 planes (3 significant bits, the emulations' choice: the products run at the
 *   FP8 tensor-core rate; within about 25 %).
 * L (device, m x n, column-major, leading dimension ldl >= max(1, m)) receives L_ij, NaN in
 * rows of op(A) and columns of op(B) that hold Inf or NaN.  The workspace (256-byte aligned)
 * holds at least gbd_abs_product_lower_bound_workspace_size(m, n, k) bytes.
 * Returns 0, a BLAS argument index (1 transa, 2 transb, 3 m, 4 n, 5 k, 8 lda, 10 ldb, 11 ldl,
 * 12 fp8) or GBD_ERR_*.  Asynchronous on stream.
 */
GBD_API size_t gbd_abs_product_lower_bound_workspace_size(int64_t m, int64_t n, int64_t k);
GBD_API int gbd_abs_product_lower_bound(char transa, char transb, int64_t m, int64_t n, int64_t k, const double* A,
                                        int64_t lda, const double* B, int64_t ldb, double* L, int64_t ldl, int fp8,
                                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * gbd_dgemm_emu for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment convenience of this library.
 *
 * Some callers must not call cudaMalloc (or any allocator) while they run: code
 * in a latency-critical loop where an allocation can block or fail at an
 * arbitrary moment, plug-ins whose host application owns all device memory, or
 * code that runs while an allocator lock is held.  This entry point takes the
 * same arguments as gbd_dgemm_emu except the workspace and computes the same
 * result (the same bits for the same slice count), using a scratch area built
 * into the library instead: a 64 MiB device array that every GPU loading the
 * library keeps until the process exits.  It allocates nothing.
 *
 * Limit: problems whose gbd_dgemm_emu_workspace_size(m, n, k, slices) exceeds
 * 64 MiB (67108864 bytes) are rejected with GBD_ERR_LIMIT; with automatic slices every
 * square problem up to 768 fits (769 needs 79 MiB).  The BLAS quick returns (m, n or k
 * zero, alpha zero) need no scratch and are never rejected.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  Under lazy module loading, the
 * CUDA default, that look-up also loads the library's module holding the array, which
 * commits its 64 MiB of device memory: the first call on a device can therefore block
 * or fail with GBD_ERR_CUDA like an allocation.  Make one small call on every device at
 * set-up time, before the loop that must not allocate and before any stream capture.
 * Automatic slices (slices = 0) read the certification back from the device, so such a
 * call synchronises `stream` and cannot be captured; pass an explicit slice count to
 * avoid both.  When no slice count can be certified the call runs gbd_dgemm, which
 * needs no scratch either.
 * Sharing: all calls on a device use the same array, which keeps the previous
 * call's contents; the parts that must start at zero are cleared by every call.
 * Calls whose work overlaps on the GPU (other streams, other host threads) race
 * on the array and corrupt each other's results: serialise them.
 * info: optional; its record_phases field is ignored (timing would allocate events).
 * Returns 0, a BLAS argument index, or GBD_ERR_* (GBD_ERR_LIMIT for a problem
 * above the scratch size).
 */
GBD_API int gbd_dgemm_emu_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k,
                                  double alpha, const double* A, int64_t lda, const double* B,
                                  int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                                  double tol, gbd_emu_info* info, void* stream);

/*
 * Double-precision GEMM emulated with the integer modular technique of Ozaki, Uchino
 * and Imamura ("Ozaki Scheme II", 2025); the operation and the argument list are those
 * of gbd_dgemm (Section 1.2 of the paper).
 *
 * Steps: the exponents sigma_i, tau_j of gbd_dgemm_emu; the integers
 * A' = rint(a_ip 2^(t - sigma_i)) and B' = rint(b_pj 2^(t - tau_j)) (ties to even,
 * |.| <= 2^t); their residues modulo the first n of the pairwise coprime moduli
 * 256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, with
 * n the fewest whose product M exceeds 2 k 2^(2t); one BF16 tcgen05 product per modulus
 * (exact FP32 chunks, int32 sums); the Chinese remainder reconstruction of the exact
 * integer C' = A'B'; and C := fma(alpha 2^(tau_j - 2t), fl(C') 2^sigma_i, beta C) with fl
 * correctly rounded.  The products number n (13 at 44 bits and k = 8192) where the split
 * emulation needs s(s+1)/2.
 *
 * bits: t in 1..62, or automatic: the certified choice (the smallest t whose a-priori
 *   truncation bound, plus the final roundings, stays within `tol` times
 *   |alpha||op(A)||op(B)| on every element, tol <= 0 meaning 2 k 2^-53, as for gbd_dgemm_emu;
 *   or the width at which every scaled entry is an integer), made on the device from a
 *   tensor-core product of magnitude planes, the same way in both automatic forms:
 *     0: the choice is read back (the call synchronises `stream` once); when it needs more
 *        than 16 moduli at this k the call returns GBD_ERR_LIMIT before touching C
 *        (gbd_dgemm_emu covers any target);
 *    -1: nothing is read back and the call never synchronises; an unreachable target fills
 *        C with NaN and sets the device error word, which gbd_check_device_error reports
 *        as GBD_ERR_LIMIT.
 *   Given t that needs more than 16 moduli returns GBD_ERR_LIMIT.
 * workspace: at least gbd_dgemm_emu_mod_workspace_size(m, n, k, bits) bytes, 256-byte
 *   aligned (bits <= 0 sizes it for 16 moduli); as for gbd_dgemm_emu.
 * info: optional; slices and products report n, digit_bits reports t, rho, gamma, bound and
 *   exact the certification (automatic modes); with bits = -1 a non-NULL info is filled by
 *   reading the choice back, which synchronises `stream`.  record_phases times the
 *   preparation with the certification (prep_ms) and the products with the reconstruction
 *   (gemm_ms).
 * Kernels: the preparation, the certification (magnitude planes and their product) and the
 *   plan, then the residues and the products: (256 x 256 tile, modulus) work units on
 *   SM pairs, modulus by modulus, or 128 x 128 tiles on single SMs (with each tile's moduli
 *   spread over several SMs when there are few tiles), by a wave-quantised estimate of their
 *   times.  The environment variables GBD_EMU_KERNEL (pair, single or split) and
 *   GBD_EMU_GROUP_M (rows of 256 x 256 tiles per raster group of the pair form) override
 *   the choice (tests and tuning); the result is the same bits either way.
 * Returns 0, a BLAS argument index, or GBD_ERR_*.
 */
GBD_API size_t gbd_dgemm_emu_mod_workspace_size(int64_t m, int64_t n, int64_t k, int bits);
/*
 * The moduli gbd_dgemm_emu_mod uses for t = bits integer bits at inner dimension k (host
 * only): writes them to moduli[0..n) when moduli is not NULL (room for 16) and returns n,
 * or 0 when 16 moduli are not enough (or bits < 1, k < 1).
 */
GBD_API int gbd_dgemm_emu_mod_moduli(int bits, int64_t k, int* moduli);
GBD_API int gbd_dgemm_emu_mod(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                              const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                              double* C, int64_t ldc, int bits, double tol, void* workspace,
                              size_t workspace_bytes, gbd_emu_info* info, void* stream);

/*
 * gbd_dgemm_emu with A, B and C in HOST memory.  The paper's dgemm works on
 * operands in the caller's memory (Section 1.2); this entry point gives that
 * interface to a caller whose matrices are on the host, with the GPU transfers
 * inside the call.  On `stream`, in order: op(A)'s storage (rows x cols with
 * leading dimension lda, rows = m or k as for gbd_dgemm) and B's are copied into
 * `device_buffer` (packed, leading dimension = rows), and C too when beta != 0;
 * gbd_dgemm_emu runs on the copies; the m x n result is copied back into C
 * (leading dimension ldc).  Elements of A, B, C outside the matrices (the
 * leading-dimension padding) are neither read nor written.
 *
 * Host memory: page-locked (cudaHostAlloc / cudaHostRegister) for asynchronous
 *   transfers; pageable memory works, but then the copies synchronise the host.
 *   The host buffers must stay valid, and C unread, until `stream` has reached
 *   the end of the call.
 * device_buffer: device memory of at least gbd_dgemm_emu_host_buffer_size(...)
 *   bytes, 256-byte aligned, owned by the caller, not reused until the call has
 *   completed on `stream`.  Two buffers used on two streams let consecutive
 *   calls overlap one call's transfers with the other's computation.
 * slices, tol, info and the automatic-mode synchronisation: as gbd_dgemm_emu.
 * Returns 0, a BLAS argument index, or GBD_ERR_* (GBD_ERR_WORKSPACE when the
 * buffer is missing, small or misaligned).
 */
GBD_API size_t gbd_dgemm_emu_host_buffer_size(char transa, char transb, int64_t m, int64_t n, int64_t k,
                                              int slices);
GBD_API int gbd_dgemm_emu_host(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                               double* C, int64_t ldc, int slices, double tol, void* device_buffer,
                               size_t buffer_bytes, gbd_emu_info* info, void* stream);
/*
 * The same with the modular emulation (gbd_dgemm_emu_mod) on the device copies: `bits`,
 * `tol`, `info` and the automatic-mode synchronisation as gbd_dgemm_emu_mod; the buffer
 * as above, sized by gbd_dgemm_emu_mod_host_buffer_size.
 */
GBD_API size_t gbd_dgemm_emu_mod_host_buffer_size(char transa, char transb, int64_t m, int64_t n,
                                                  int64_t k, int bits);
GBD_API int gbd_dgemm_emu_mod_host(char transa, char transb, int64_t m, int64_t n, int64_t k,
                                   double alpha, const double* A, int64_t lda, const double* B,
                                   int64_t ldb, double beta, double* C, int64_t ldc, int bits,
                                   double tol, void* device_buffer, size_t buffer_bytes,
                                   gbd_emu_info* info, void* stream);

/* ------------------------------------------------------------------------- */
/* Grouped calls: many independent problems per launch                       */
/* ------------------------------------------------------------------------- */
#define GBD_MODE_NATIVE 0    /* FP64 mma.sync, as gbd_dgemm */
#define GBD_MODE_EMULATED 1  /* split digits on tcgen05, as gbd_dgemm_emu */
#define GBD_MODE_MODULAR 2   /* residues on tcgen05, as gbd_dgemm_emu_mod, planned on the device */

/* One problem of a grouped call: the dgemm argument list of Section 1.2 plus how
 * to compute it.  Pointers are device pointers owned by the caller; problems must
 * not write overlapping parts of C. */
typedef struct gbd_problem {
  char transa, transb;
  uint8_t ksplit;  /* native: parts of the inner dimension per output tile, 2..16 (each part a
                      separate work item, the parts' sums added in part order by the last one to
                      finish: the same bits whatever order they run in), or 0/1 = none; capped at
                      the problem's 16-deep k-blocks */
  uint8_t reserved;  /* zero */
  int32_t mode;    /* GBD_MODE_NATIVE, GBD_MODE_EMULATED or GBD_MODE_MODULAR */
  int32_t slices;  /* emulated: 1..9, or 0 = certified automatically when the plan is created;
                      modular: integer bits 1..62, or 0 = certified on the device by every run */
  int32_t tile;    /* native: CTA tile edge 32 or 64; emulated: 128 (one-SM kernel) or 256 (two-SM
                      kernel); modular: 128 (one-SM kernel), or 0: 256 x 256 tiles on CTA pairs
                      when m, n and k are all at least 256, else the one-SM kernel; 0 = library
                      default (the autotuner's hook) */
  int64_t m, n, k;
  double alpha, beta;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  double tol;      /* emulated and modular, automatic precision: target relative error (<= 0: 2 k 2^-53) */
} gbd_problem;

/* Opaque host-side plan of a grouped call (problem tables live in the workspace). */
typedef struct gbd_plan gbd_plan;

/*
 * Bytes of device workspace for a grouped call over `probs` (host-only; needs no
 * GPU).  Emulated problems with slices == 0 are sized for 9 slices, modular ones with
 * bits == 0 for 16 moduli.
 */
GBD_API size_t gbd_dgemm_grouped_workspace_size(const gbd_problem* probs, int count);

/*
 * Builds a plan: validates every problem, lays out `workspace` (caller-owned,
 * 256-byte aligned, at least gbd_dgemm_grouped_workspace_size bytes) and copies the
 * problem tables to the device through page-locked staging owned by the plan
 * (stream-ordered copies on `stream`).  Emulated problems with automatic slices are
 * certified now, from the data present now (the only case that synchronises `stream`);
 * a problem that no slice count up to 9 certifies joins the FP64 problems.  Modular
 * problems are certified and planned on the device by every run instead, so a plan
 * of modular and native problems is made without any synchronisation and its runs
 * re-certify whatever data the buffers hold.  Native problems are ordered longest tile
 * first for the atomic tile counter; emulated ones by decreasing tile cost; modular ones
 * by decreasing k.
 * slices_used: optional array of `count` ints, receives each emulated problem's
 * slice count (-1 when it was sent to the FP64 path; 0 for native and modular problems
 * and quick returns).
 * Returns 0, GBD_ERR_ARG (gbd_last_error names the problem and the BLAS argument
 * index), GBD_ERR_WORKSPACE, GBD_ERR_LIMIT or GBD_ERR_CUDA.
 */
GBD_API int gbd_grouped_plan_create(const gbd_problem* probs, int count, void* workspace,
                                    size_t workspace_bytes, int* slices_used, void* stream,
                                    gbd_plan** plan);

/*
 * Runs a plan on `stream`: for emulated problems their exponent and split kernels
 * and one persistent slice-product launch per slice count over all their tiles; for
 * modular problems their batched preparation, the certification product (FP8), one
 * plan per problem, the residues, the modular products in two persistent launches (the
 * problems with m, n, k >= 256 as (256 x 256 tile, modulus) units on CTA pairs, the
 * others' 128 x 128 tiles on single SMs) and the reconstruction of C; then one
 * persistent FP64-MMA launch for native problems,
 * every quick return, and each modular problem whose plan found the target out of the
 * reach of 16 moduli (its tiles in that launch test the plan on the device).  Only
 * kernel launches and memsets are issued, so the call may be captured in a CUDA graph
 * and replayed while the plan, the workspace and the problems' buffers stay alive; each
 * run reads A, B, C afresh.  A problem's result is bit-identical to the single-problem
 * call with the same arguments (emulated: the same slice count; modular: gbd_dgemm_emu_mod
 * with bits = -1, or gbd_dgemm when its plan was infeasible).  Asynchronous.
 */
GBD_API int gbd_grouped_plan_run(gbd_plan* plan, void* stream);

/* Frees the host side of a plan (never the workspace). */
GBD_API void gbd_grouped_plan_destroy(gbd_plan* plan);

/* Create, run and destroy a plan in one call. */
GBD_API int gbd_dgemm_grouped(const gbd_problem* probs, int count, void* workspace,
                              size_t workspace_bytes, int* slices_used, void* stream);

/*
 * Measures the FP64 tensor-core rate of the current device (the native path's roofline):
 * 4 x (SMs) blocks of 256 threads, each warp issuing iters x 8 independent
 * mma.sync.m16n8k16.f64 (4096 flops each) on register operands; one warm-up launch, then
 * one launch timed with CUDA events on `stream` (synchronised).  *tflops receives the rate.
 */
GBD_API int gbd_fp64_mma_probe(int64_t iters, double* tflops, void* stream);

/*
 * Exercises the watchdog: launches one thread that waits on a barrier nothing
 * completes, gives up after `limit_ms` milliseconds (1..10000), sets the device
 * error word exactly as a kernel whose wait ran out would, and ends normally (no
 * fault, no hang; the context stays usable).  A following gbd_check_device_error
 * returns GBD_ERR_TIMEOUT.  Asynchronous on `stream`.
 */
GBD_API int gbd_watchdog_selftest(int limit_ms, void* stream);

/*
 * Reads and clears the device error word of the current device that the
 * kernels set when a bounded wait gives up (or when a gbd_dgemm_emu_mod call in
 * device-side automatic mode, bits = -1, met an unreachable target).  Synchronises
 * `stream` first.  Returns 0 when nothing was recorded since the last call,
 * GBD_ERR_LIMIT when only such a modular call was, GBD_ERR_TIMEOUT when a wait gave
 * up, or GBD_ERR_CUDA.
 */
GBD_API int gbd_check_device_error(void* stream);

/* ------------------------------------------------------------------------- */
/* Context: a device and a pool of library-owned workspaces                   */
/* ------------------------------------------------------------------------- */
/*
 * The calls above take a caller-owned workspace.  A context owns them instead: it is bound
 * to one device, keeps one workspace per stream that it grows with stream-ordered
 * allocations (cudaMallocAsync / cudaFreeAsync on that stream, so no call waits for
 * another and a block is reused only by later calls on the same stream), and makes its
 * device current for the duration of each call.  Tensor maps and grouped plans are not
 * cached: both depend on the operands' addresses, and automatic precision on their data.
 * A context may be used from several host threads; calls that share a stream must be
 * issued in the order the stream should run them.
 */
typedef struct gbd_ctx gbd_ctx;

#define GBD_METHOD_NATIVE 0   /* gbd_dgemm (FP64 tensor-core MMA) */
#define GBD_METHOD_SPLIT 1    /* gbd_dgemm_emu with the certified slice count */
#define GBD_METHOD_MODULAR 2  /* gbd_dgemm_emu_mod with the certified bit count (bits = 0) */
#define GBD_METHOD_AUTO 3     /* modular, or split when 16 moduli cannot certify the target
                                 (which computes natively when 9 slices cannot either) */

/* Creates a context on `device` (an sm_103 GPU).  Returns 0, GBD_ERR_DEVICE, GBD_ERR_CUDA. */
GBD_API int gbd_create(gbd_ctx** ctx, int device);
/* Releases the context and its workspaces (each freed in its stream's order). */
GBD_API void gbd_destroy(gbd_ctx* ctx);
/* Bytes of workspace that `method` takes for an m x n x k problem (automatic precision);
 * host-only: ctx may be NULL.  Returns 0, 3/4/5 for a negative m/n/k, or GBD_ERR_ARG. */
GBD_API int gbd_workspace_size(const gbd_ctx* ctx, int method, int64_t m, int64_t n, int64_t k, size_t* bytes);
/*
 * C := alpha op(A) op(B) + beta C (Section 1.2) by `method`, with the workspace from the
 * context's pool for `stream`; tol as gbd_dgemm_emu (<= 0: the FP64 bound 2 k 2^-53).  The
 * emulated methods choose their precision automatically and synchronise `stream` once to
 * read the choice.  info (optional) reports the path taken.  Returns 0, a BLAS argument
 * index, or GBD_ERR_* (GBD_ERR_LIMIT from GBD_METHOD_MODULAR when 16 moduli cannot certify
 * the target; GBD_ERR_WORKSPACE when the pool cannot grow).
 */
GBD_API int gbd_ctx_dgemm(gbd_ctx* ctx, int method, char transa, char transb, int64_t m, int64_t n, int64_t k,
                          double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                          double* C, int64_t ldc, double tol, gbd_emu_info* info, void* stream);
/* gbd_dgemm_grouped with the workspace from the context's pool for `stream`. */
GBD_API int gbd_ctx_dgemm_grouped(gbd_ctx* ctx, const gbd_problem* probs, int count, int* slices_used,
                                  void* stream);
/* gbd_check_device_error on the context's device: synchronises `stream`, then reads and
 * clears the device error word (0, GBD_ERR_TIMEOUT, GBD_ERR_LIMIT or GBD_ERR_CUDA). */
GBD_API int gbd_sync_error(gbd_ctx* ctx, void* stream);
/* Bytes the context's pool holds now (all streams). */
GBD_API size_t gbd_ctx_pool_bytes(gbd_ctx* ctx);

/* ------------------------------------------------------------------------- */
/* GEMM-based level-3 BLAS (the paper's "Poorman's BLAS", Section 3.1)        */
/* ------------------------------------------------------------------------- */
/*
 * DSYRK, DTRMM and DTRSM cast in terms of this library's GEMM, after Kagstrom, Ling and
 * Van Loan (TOMS 24(3), 1998), the work the paper cites for building every level-3
 * operation from matrix-matrix products of submatrices.  Argument lists, meanings and
 * return codes are those of reference BLAS; column-major storage with leading dimensions
 * (Section 2.1); device pointers owned by the caller; asynchronous on `stream`.
 *
 * mode: GBD_MODE_NATIVE (products by gbd_dgemm) or GBD_MODE_EMULATED: each product by the
 *   fastest path that meets `tol` (tol <= 0: each product's FP64 bound): gbd_dgemm below
 *   1e8 flops; gbd_dgemm_emu_mod for at least 2.5e6 outputs, or gbd_dgemm_emu when 16
 *   moduli cannot reach `tol`; gbd_dgemm_emu otherwise.  Each emulated product synchronises
 *   `stream` once.  Any other mode: GBD_ERR_ARG.  The environment variables
 *   GBD_L3_NATIVE_FLOPS and GBD_L3_MODULAR_OUTPUTS override the two thresholds (read at
 *   every call; for tests and tuning).
 * workspace: at least the matching *_workspace_size bytes, 256-byte aligned (may be NULL
 *   when that size is 0).  Its contents are scratch.
 *
 * gbd_dsyrk: C := alpha op(A) op(A)^T + beta C on the `uplo` ('U'/'L') triangle of the
 *   n x n matrix C; op(A) = A (n x k) for trans 'N', A^T (A is k x n) for 'T'/'C'.  The
 *   other triangle is neither read for the result nor written.  beta = 0: C is not read.
 *   In emulated mode, when the whole triangle meets the modular threshold (n^2 / 2
 *   outputs), it is one modular product whose tiles are those that meet the triangle;
 *   when 16 moduli cannot reach `tol` there, the call recurses on halves instead.
 *   Codes: 1 uplo, 2 trans, 3 n, 4 k, 7 lda, 10 ldc.
 * gbd_dtrmm: B := alpha op(A) B (side 'L', A m x m) or alpha B op(A) (side 'R', A n x n),
 *   A triangular: only its `uplo` triangle is read; diag 'U' means a unit diagonal, not
 *   read.  alpha = 0: B := 0 without reading A.
 * gbd_dtrsm: B := X solving op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'),
 *   same conventions.  No test for singularity is made (as in BLAS).
 *   Codes (both): 1 side, 2 uplo, 3 transa, 4 diag, 5 m, 6 n, 9 lda, 11 ldb.
 */
GBD_API size_t gbd_dsyrk_workspace_size(int64_t n, int64_t k, int mode);
GBD_API size_t gbd_dtrmm_workspace_size(char side, int64_t m, int64_t n, int mode);
GBD_API size_t gbd_dtrsm_workspace_size(char side, int64_t m, int64_t n, int mode);
GBD_API int gbd_dsyrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double* A,
                      int64_t lda, double beta, double* C, int64_t ldc, int mode, double tol,
                      void* workspace, size_t workspace_bytes, void* stream);
GBD_API int gbd_dtrmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                      double alpha, const double* A, int64_t lda, double* B, int64_t ldb, int mode,
                      double tol, void* workspace, size_t workspace_bytes, void* stream);
GBD_API int gbd_dtrsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                      double alpha, const double* A, int64_t lda, double* B, int64_t ldb, int mode,
                      double tol, void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBDGEMM_H */
