// level3.cu -- GEMM-based level-3 BLAS: DSYRK, DTRMM and DTRSM cast in terms of the
// library's GEMM (native FP64 or emulated), after the paper's "Poorman's BLAS" (Section
// 3.1, citing Kagstrom, Ling and Van Loan, TOMS 24(3), 1998): only the matrix-matrix
// product is tuned; every other level-3 operation is blocked so that nearly all of its
// flops are products of submatrices.
//
// Each operation recurses on halves of its triangle (split points on multiples of 64):
//   DSYRK  C11 := syrk(A1); C21 (or C12) := GEMM; C22 := syrk(A2).  A diagonal block of at
//          most 512 is one GEMM into scratch followed by a copy of its triangle.  In emulated
//          mode, when the whole triangle would go to the modular emulation, it is instead one
//          modular product whose tiles cover only the triangle (the recursion's products are
//          smaller, and each pays the emulation's fixed costs).
//   DTRMM  one half through the recursion, the coupling block as one GEMM with beta = 1,
//          ordered so every GEMM reads only blocks not yet overwritten.  A diagonal block of
//          at most 512: its strictly triangular part packed with zeros, one GEMM into scratch,
//          and the diagonal applied in the update B := fma(alpha d, B, T).  Apart from the
//          diagonal, the rows of the packed triangle keep their own scale: a large diagonal
//          (a diagonally dominant triangle) would otherwise set the scale of its row, and the
//          emulations could not certify the products of the row's small entries.
//   DTRSM  the leading half solved, the trailing right-hand sides updated by one GEMM
//          (beta = alpha folds the scaling in), the trailing half solved with alpha = 1.  The
//          diagonal blocks of at most 64 are inverted together in one launch before the
//          recursion (k_trsm_invert, substitution on the identity); each is then applied as a
//          dense triangular product, one thread per two rows of a solution (k_trsm_apply).
//          On GB300's narrow FP64 pipe this beats substitution on the right-hand sides, which
//          leaves the pipe idle (one thread per right-hand side) or wastes it (one warp).
// All work is stream-ordered on the caller's stream.  In emulated mode each product takes the
// fastest path that meets `tol`: products under 1e8 flops run natively (a native call is then
// faster than the emulation's fixed cost, and at least as accurate); products with at least
// 2.5e6 outputs (enough 128 x 128 tiles for every SM) use the modular emulation, and the split
// emulation when 16 moduli cannot reach `tol`; the rest use the split emulation, whose
// split inner dimension serves few output tiles.  Each emulated product synchronises the
// stream once (automatic mode).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gbd {
namespace {

constexpr int64_t kSyrkBase = 512;  // diagonal blocks of DSYRK
constexpr int64_t kTrmmBase = 512;  // diagonal blocks of DTRMM
constexpr int64_t kTrsmBase = 64;   // diagonal blocks of DTRSM (substitution kernel)
constexpr int kTrsmVecs = 16;       // right-hand sides per CTA of the diagonal-block product
constexpr double kNativeFlops = 1e8;    // emulated mode: smaller products run natively
constexpr double kModularOutputs = 2.5e6;  // emulated mode: larger outputs use the modular emulation

// the two thresholds, overridable by GBD_L3_NATIVE_FLOPS and GBD_L3_MODULAR_OUTPUTS (tests, tuning)
double threshold(const char* env, double dflt) {
  const char* v = getenv(env);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  const double x = strtod(v, &end);
  return end && end != v ? x : dflt;
}

int64_t split_point(int64_t r0, int64_t r1) {
  const int64_t half = (r1 - r0) / 2;
  const int64_t h = r0 + (half + 63) / 64 * 64;
  return h < r1 ? h : r0 + half;
}

int upper_code(char u) { return (u == 'U' || u == 'u') ? 1 : (u == 'L' || u == 'l') ? 0 : -1; }
int side_code(char s) { return (s == 'L' || s == 'l') ? 0 : (s == 'R' || s == 'r') ? 1 : -1; }
int diag_code(char d) { return (d == 'U' || d == 'u') ? 1 : (d == 'N' || d == 'n') ? 0 : -1; }
int64_t max1(int64_t a) { return a > 1 ? a : 1; }

// ---------------------------------------------------------------------------- kernels
// C[i, j] := W[i, j] on the triangle of a b x b block (lower: i >= j; upper: i <= j)
__global__ void __launch_bounds__(256) k_tri_copy(const double* __restrict__ W, int64_t ldw, double* __restrict__ C,
                                                  int64_t ldc, int64_t b, int upper) {
  const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t j = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= b || j >= b) return;
  if (upper ? i <= j : i >= j) C[j * ldc + i] = W[j * ldw + i];
}

// C := beta C on the triangle of an n x n matrix (beta == 0: zeros, C not read)
__global__ void __launch_bounds__(256) k_tri_scale(double* __restrict__ C, int64_t ldc, int64_t n, int upper,
                                                   double beta) {
  const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t j = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= n || j >= n) return;
  if (upper ? i <= j : i >= j) C[j * ldc + i] = beta == 0.0 ? 0.0 : beta * C[j * ldc + i];
}

// D := the strictly triangular part of the b x b block of A at `a` (zeros on the diagonal and
// off the triangle; the diagonal is not read)
__global__ void __launch_bounds__(256) k_tri_pack(const double* __restrict__ a, int64_t lda, double* __restrict__ D,
                                                  int64_t ldd, int64_t b, int upper) {
  const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t j = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= b || j >= b) return;
  D[j * ldd + i] = (upper ? i < j : i > j) ? a[j * lda + i] : 0.0;
}

// X[i, j] := fma(alpha d_q, X[i, j], T[i, j]) over a rows x cols block, q = i (by_row) or j, with
// d_q = 1 for a unit diagonal and otherwise the diagonal element q of the block of A at `a`
// (columns in a grid-stride loop)
__global__ void __launch_bounds__(256) k_diag_update(const double* __restrict__ a, int64_t lda, int unit,
                                                     double alpha, const double* __restrict__ T, int64_t ldt,
                                                     double* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                                                     int by_row) {
  const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  if (i >= rows) return;
  for (int64_t j = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5); j < cols; j += (int64_t)gridDim.y * 8) {
    const int64_t q = by_row ? i : j;
    const double d = unit ? 1.0 : a[q * lda + q];
    X[j * ldx + i] = fma(alpha * d, X[j * ldx + i], T[j * ldt + i]);
  }
}

// The diagonal blocks of the solve, inverted once per call: block q covers rows
// [r0[q], r0[q] + b[q]) (b <= 64) of the stored A; E is that block's stored triangle (unit
// diagonal if `unit`) or its transpose (teff), and Dinv[q] = E^-1, row-major 64 x 64.  Thread c
// solves E y = e_c by substitution (E^-1 is triangular like E) with E in shared memory.
struct TrsmBlock {
  int64_t r0;
  int b;
  int pad;
};

constexpr int kTrsmInvSmem = 2 * 64 * 64 * 8;
__global__ void __launch_bounds__(64) k_trsm_invert(const double* __restrict__ A, int64_t lda,
                                                    const TrsmBlock* __restrict__ blocks, int upper, int unit,
                                                    int teff, double* __restrict__ Dinv) {
  extern __shared__ double sm[];
  double (*E)[64] = reinterpret_cast<double (*)[64]>(sm);            // E[s][t] (a row read by all threads)
  double (*Y)[64] = reinterpret_cast<double (*)[64]>(sm + 64 * 64);  // Y[s][c]: column c of E^-1
  const TrsmBlock blk = blocks[blockIdx.x];
  const int b = blk.b;
  const double* a = A + blk.r0 * lda + blk.r0;
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int i = idx % b, j = idx / b;  // stored element (i, j), i fastest (contiguous)
    double v = 0.0;
    if (i == j) v = unit ? 1.0 : a[(int64_t)j * lda + i];
    else if (upper ? i < j : i > j) v = a[(int64_t)j * lda + i];
    if (teff) E[j][i] = v;
    else E[i][j] = v;
  }
  __syncthreads();
  const int c = threadIdx.x;
  const bool lower = (upper == 0) != (teff != 0);
  if (c < b) {
    for (int step = 0; step < b; ++step) {
      const int s = lower ? step : b - 1 - step;
      double y = 0.0;
      if (lower ? s >= c : s <= c) {
        double acc = s == c ? 1.0 : 0.0;
        const int t0 = lower ? c : s + 1, t1 = lower ? s : c + 1;
        for (int t = t0; t < t1; ++t) acc = fma(-E[s][t], Y[t][c], acc);
        y = unit ? acc : acc / E[s][s];
      }
      Y[s][c] = y;
    }
  }
  __syncthreads();
  double* out = Dinv + (int64_t)blockIdx.x * 64 * 64;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) {
    const int s = idx / 64, t = idx % 64;
    out[idx] = (s < b && t < b) ? Y[s][t] : 0.0;
  }
}

// X := E^-1 (alpha V) for nvec right-hand sides of the b x b diagonal block whose inverse is
// Dinv (row-major 64 x 64); element q of right-hand side u lives at B[q * sq + u * su].  A CTA
// takes 16 right-hand sides: the inverse and the scaled right-hand sides are staged in shared
// memory, then thread (h, v) forms rows h and b - 1 - h of solution v.  Row s of a triangular
// E^-1 has s + 1 (lower) or b - s (upper) terms, so each thread's pair has b + 1 and the
// warp's lanes, which the FP64 pipe charges for whether busy or masked, all work alike.
__device__ __forceinline__ double tri_row(const double (*Di)[65], const double (*R)[kTrsmVecs + 1], int s, int v, int b,
                                          bool lower) {
  const int t0 = lower ? 0 : s, t1 = lower ? s + 1 : b;
  double x = 0.0, x1 = 0.0;
  int t = t0;
  for (; t + 1 < t1; t += 2) {
    x = fma(Di[s][t], R[t][v], x);
    x1 = fma(Di[s][t + 1], R[t + 1][v], x1);
  }
  if (t < t1) x = fma(Di[s][t], R[t][v], x);
  return x + x1;
}

__global__ void __launch_bounds__(32 * kTrsmVecs) k_trsm_apply(const double* __restrict__ Dinv, int b, int lower,
                                                               double* __restrict__ B, int64_t sq, int64_t su,
                                                               int64_t nvec, double alpha) {
  __shared__ double Di[64][65];
  __shared__ double R[64][kTrsmVecs + 1];  // R[t][v]; the pad spreads the row-fast staging over banks
  const int64_t u0 = (int64_t)blockIdx.x * kTrsmVecs;
  const int nv = (int)min((int64_t)kTrsmVecs, nvec - u0);
  for (int idx = threadIdx.x; idx < 64 * 64; idx += blockDim.x) Di[idx / 64][idx % 64] = Dinv[idx];
  const bool q_fast = sq == 1;
  for (int idx = threadIdx.x; idx < b * nv; idx += blockDim.x) {
    const int q = q_fast ? idx % b : idx / nv, v = q_fast ? idx / b : idx % nv;
    R[q][v] = alpha * B[(int64_t)q * sq + (u0 + v) * su];
  }
  __syncthreads();
  const int h = threadIdx.x % 32, v = threadIdx.x / 32;
  const int s1 = b - 1 - h;  // the partner row (h itself for the middle row of an odd b)
  const bool act = v < nv && h <= s1;
  double x0 = 0.0, x1 = 0.0;
  if (act) {
    x0 = tri_row(Di, R, h, v, b, lower != 0);
    if (s1 != h) x1 = tri_row(Di, R, s1, v, b, lower != 0);
  }
  __syncthreads();
  if (act) {
    R[h][v] = x0;
    if (s1 != h) R[s1][v] = x1;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < b * nv; idx += blockDim.x) {
    const int q = q_fast ? idx % b : idx / nv, vv = q_fast ? idx / b : idx % nv;
    B[(int64_t)q * sq + (u0 + vv) * su] = R[q][vv];
  }
}

dim3 grid2(int64_t rows, int64_t cols) { return dim3((unsigned)((rows + 31) / 32), (unsigned)((cols + 7) / 8)); }
// the same with the column blocks capped (kernels that loop over columns)
dim3 grid2_capped(int64_t rows, int64_t cols) {
  const int64_t gy = (cols + 7) / 8;
  return dim3((unsigned)((rows + 31) / 32), (unsigned)(gy < 65535 ? (gy > 0 ? gy : 1) : 65535));
}

// ---------------------------------------------------------------------------- driver
// One call's context: the GEMM dispatch and scratch.  In `dry` mode nothing is launched and
// `need` collects the largest emulated-GEMM workspace the recursion asks for.
struct Ctx {
  int mode;
  double tol;
  cudaStream_t s;
  void* gws;
  size_t gwsb;
  double* scr;  // level-3 scratch (W, D, T)
  bool dry;
  size_t need;
  std::vector<TrsmBlock>* blocks = nullptr;  // DTRSM: the diagonal blocks (sorted by first row for use)
  double* dinv = nullptr;                    // DTRSM: their inverses, 64 x 64 each, in that order
  // the inverse of the diagonal block starting at row r0
  const double* inverse_at(int64_t r0) const {
    size_t lo = 0, hi = blocks->size();
    while (hi - lo > 1) {
      const size_t mid = (lo + hi) / 2;
      if ((*blocks)[mid].r0 <= r0) lo = mid;
      else hi = mid;
    }
    return dinv + (int64_t)lo * 64 * 64;
  }
  double native_flops = kNativeFlops, modular_outputs = kModularOutputs;
  void thresholds() {
    native_flops = threshold("GBD_L3_NATIVE_FLOPS", kNativeFlops);
    modular_outputs = threshold("GBD_L3_MODULAR_OUTPUTS", kModularOutputs);
  }
  // DSYRK in emulated mode: the whole n x n triangle as one modular product
  bool syrk_modular(int64_t n, int64_t k) const {
    return mode != GBD_MODE_NATIVE && (double)n * (double)n * (double)k > native_flops &&
           0.5 * (double)n * (double)n >= modular_outputs;
  }

  int gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
           const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    if (m == 0 || n == 0) return GBD_OK;
    const bool native = mode == GBD_MODE_NATIVE || 2.0 * (double)m * (double)n * (double)k <= native_flops;
    const bool modular = !native && (double)m * (double)n >= modular_outputs;
    if (dry) {
      if (!native) {
        size_t w = gbd_dgemm_emu_workspace_size(m, n, k, 0);
        if (modular) {
          const size_t wm = gbd_dgemm_emu_mod_workspace_size(m, n, k, 0);
          if (wm > w) w = wm;
        }
        if (w > need) need = w;
      }
      return GBD_OK;
    }
    if (native) return gbd_dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    if (modular) {
      const int rc = gbd_dgemm_emu_mod(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, gws, gwsb,
                                       nullptr, s);
      if (rc != GBD_ERR_LIMIT) return rc;  // GBD_ERR_LIMIT: the target needs more than 16 moduli; C untouched
    }
    return gbd_dgemm_emu(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, gws, gwsb, nullptr, s);
  }
  int check(const char* what) {
    if (dry) return GBD_OK;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, what);
  }
  int copy2d(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols) {
    if (dry || rows == 0 || cols == 0) return GBD_OK;
    const cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)ldd * 8, src, (size_t)lds * 8, (size_t)rows * 8,
                                            (size_t)cols, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "level-3 block copy");
  }
};

// ---- DSYRK ----
struct Syrk {
  Ctx* c;
  int upper, tr;
  int64_t k;
  double alpha, beta;
  const double* A;
  int64_t lda;
  double* C;
  int64_t ldc;
  // rows [r0, r1) of op(A) as a GEMM operand: (pointer, its transpose flag)
  const double* rows(int64_t r0) const { return tr ? A + r0 * lda : A + r0; }

  int run(int64_t r0, int64_t r1) {
    const int64_t b = r1 - r0;
    const char ta = tr ? 'T' : 'N', tb = tr ? 'N' : 'T';
    int rc;
    if (b <= kSyrkBase) {
      // W := alpha op(A)_b op(A)_b^T + beta C_bb (the whole block), then its triangle into C
      double* W = c->scr;
      double* Cb = C + r0 * ldc + r0;
      if (beta != 0.0 && (rc = c->copy2d(W, b, Cb, ldc, b, b))) return rc;
      if ((rc = c->gemm(ta, tb, b, b, k, alpha, rows(r0), lda, rows(r0), lda, beta, W, b))) return rc;
      if (!c->dry) k_tri_copy<<<grid2(b, b), 256, 0, c->s>>>(W, b, Cb, ldc, b, upper);
      return c->check("triangle copy launch");
    }
    const int64_t h = split_point(r0, r1);
    if ((rc = run(r0, h))) return rc;
    if (upper) {  // C[r0:h, h:r1] := alpha op(A)[r0:h] op(A)[h:r1]^T + beta C
      rc = c->gemm(ta, tb, h - r0, r1 - h, k, alpha, rows(r0), lda, rows(h), lda, beta, C + h * ldc + r0, ldc);
    } else {  // C[h:r1, r0:h] := alpha op(A)[h:r1] op(A)[r0:h]^T + beta C
      rc = c->gemm(ta, tb, r1 - h, h - r0, k, alpha, rows(h), lda, rows(r0), lda, beta, C + r0 * ldc + h, ldc);
    }
    if (rc) return rc;
    return run(h, r1);
  }
};

// ---- DTRMM and DTRSM ----
struct Tri {
  Ctx* c;
  int side, upper, tr, unit;
  int64_t m, n;
  const double* A;
  int64_t lda;
  double* B;
  int64_t ldb;
  char ta() const { return tr ? 'T' : 'N'; }
  // op(A) is lower triangular when (uplo = L) xor transposed
  bool eff_lower() const { return (upper == 0) != (tr != 0); }
  // op(A)[r, c] as the top-left element of a GEMM operand in A's storage
  const double* opA(int64_t r, int64_t col) const { return tr ? A + col + r * lda : A + r + col * lda; }
  double* Brow(int64_t r) const { return B + r; }          // rows from r (side L)
  double* Bcol(int64_t col) const { return B + col * ldb; }  // columns from col (side R)

  // DTRMM on the diagonal block [r0, r1) of op(A)
  int trmm(int64_t r0, int64_t r1, double alpha) {
    const int64_t b = r1 - r0;
    int rc;
    if (b <= kTrmmBase) {
      double* D = c->scr;
      double* T = c->scr + kTrmmBase * kTrmmBase;
      const double* Ab = A + r0 * lda + r0;
      if (!c->dry) k_tri_pack<<<grid2(b, b), 256, 0, c->s>>>(Ab, lda, D, b, b, upper);
      if ((rc = c->check("triangle pack launch"))) return rc;
      if (side == 0) {  // T := alpha op(D) B[r0:r1, :] (D strictly triangular); B := alpha diag B + T
        if ((rc = c->gemm(ta(), 'N', b, n, b, alpha, D, b, Brow(r0), ldb, 0.0, T, b))) return rc;
        if (!c->dry) k_diag_update<<<grid2_capped(b, n), 256, 0, c->s>>>(Ab, lda, unit, alpha, T, b, Brow(r0), ldb, b, n, 1);
        return c->check("diagonal update launch");
      }
      // T := alpha B[:, r0:r1] op(D); B := alpha B diag + T
      if ((rc = c->gemm('N', ta(), m, b, b, alpha, Bcol(r0), ldb, D, b, 0.0, T, m))) return rc;
      if (!c->dry) k_diag_update<<<grid2_capped(m, b), 256, 0, c->s>>>(Ab, lda, unit, alpha, T, m, Bcol(r0), ldb, m, b, 0);
      return c->check("diagonal update launch");
    }
    const int64_t h = split_point(r0, r1);
    const bool lo = eff_lower();
    if (side == 0) {
      if (lo) {  // B2 := a A22 B2; B2 += a A21 B1; B1 := a A11 B1
        if ((rc = trmm(h, r1, alpha))) return rc;
        if ((rc = c->gemm(ta(), 'N', r1 - h, n, h - r0, alpha, opA(h, r0), lda, Brow(r0), ldb, 1.0, Brow(h), ldb)))
          return rc;
        return trmm(r0, h, alpha);
      }
      // B1 := a A11 B1; B1 += a A12 B2; B2 := a A22 B2
      if ((rc = trmm(r0, h, alpha))) return rc;
      if ((rc = c->gemm(ta(), 'N', h - r0, n, r1 - h, alpha, opA(r0, h), lda, Brow(h), ldb, 1.0, Brow(r0), ldb)))
        return rc;
      return trmm(h, r1, alpha);
    }
    if (lo) {  // B1 := a B1 A11; B1 += a B2 A21; B2 := a B2 A22
      if ((rc = trmm(r0, h, alpha))) return rc;
      if ((rc = c->gemm('N', ta(), m, h - r0, r1 - h, alpha, Bcol(h), ldb, opA(h, r0), lda, 1.0, Bcol(r0), ldb)))
        return rc;
      return trmm(h, r1, alpha);
    }
    // B2 := a B2 A22; B2 += a B1 A12; B1 := a B1 A11
    if ((rc = trmm(h, r1, alpha))) return rc;
    if ((rc = c->gemm('N', ta(), m, r1 - h, h - r0, alpha, Bcol(r0), ldb, opA(r0, h), lda, 1.0, Bcol(h), ldb)))
      return rc;
    return trmm(r0, h, alpha);
  }

  // DTRSM on the diagonal block [r0, r1) of op(A): X := solution for alpha B there
  int trsm(int64_t r0, int64_t r1, double alpha) {
    const int64_t b = r1 - r0;
    int rc;
    if (b <= kTrsmBase) {
      if (c->dry) {
        if (c->blocks) c->blocks->push_back(TrsmBlock{r0, (int)b, 0});
        return GBD_OK;
      }
      // side L: E = op(D), right-hand sides are the columns of B[r0:r1, :];
      // side R: X op(D) = alpha B  <=>  op(D)^T X^T = alpha B^T, right-hand sides are rows
      const int teff = side == 0 ? tr : !tr;
      const int lowerE = (upper == 0) != (teff != 0);
      const int64_t nvec = side == 0 ? n : m;
      double* base = side == 0 ? Brow(r0) : Bcol(r0);
      const int64_t sq = side == 0 ? 1 : ldb, su = side == 0 ? ldb : 1;
      k_trsm_apply<<<(unsigned)((nvec + kTrsmVecs - 1) / kTrsmVecs), 32 * kTrsmVecs, 0, c->s>>>(
          c->inverse_at(r0), (int)b, lowerE, base, sq, su, nvec, alpha);
      return c->check("triangular solve launch");
    }
    const int64_t h = split_point(r0, r1);
    const bool lo = eff_lower();
    if (side == 0) {
      if (lo) {  // X1; B2 := alpha B2 - A21 X1; X2
        if ((rc = trsm(r0, h, alpha))) return rc;
        if ((rc = c->gemm(ta(), 'N', r1 - h, n, h - r0, -1.0, opA(h, r0), lda, Brow(r0), ldb, alpha, Brow(h), ldb)))
          return rc;
        return trsm(h, r1, 1.0);
      }
      // X2; B1 := alpha B1 - A12 X2; X1
      if ((rc = trsm(h, r1, alpha))) return rc;
      if ((rc = c->gemm(ta(), 'N', h - r0, n, r1 - h, -1.0, opA(r0, h), lda, Brow(h), ldb, alpha, Brow(r0), ldb)))
        return rc;
      return trsm(r0, h, 1.0);
    }
    if (lo) {  // X op(A) with op(A) lower: X2 first; B1 := alpha B1 - X2 A21; X1
      if ((rc = trsm(h, r1, alpha))) return rc;
      if ((rc = c->gemm('N', ta(), m, h - r0, r1 - h, -1.0, Bcol(h), ldb, opA(h, r0), lda, alpha, Bcol(r0), ldb)))
        return rc;
      return trsm(r0, h, 1.0);
    }
    // upper: X1 first; B2 := alpha B2 - X1 A12; X2
    if ((rc = trsm(r0, h, alpha))) return rc;
    if ((rc = c->gemm('N', ta(), m, r1 - h, h - r0, -1.0, Bcol(r0), ldb, opA(r0, h), lda, alpha, Bcol(h), ldb)))
      return rc;
    return trsm(h, r1, 1.0);
  }
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t syrk_scratch(int64_t n) {
  const int64_t b = n < kSyrkBase ? n : kSyrkBase;
  return up256(sizeof(double) * (size_t)(b * b));
}
size_t trmm_scratch(int side, int64_t m, int64_t n) {
  const int64_t order = side == 0 ? m : n;
  const int64_t b = order < kTrmmBase ? order : kTrmmBase;
  // D at a fixed offset of kTrmmBase^2, then T (b x n or m x b)
  return up256(sizeof(double) * (size_t)(kTrmmBase * kTrmmBase + (side == 0 ? b * n : m * b)));
}

int check_tri_args(char side, char uplo, char transa, char diag, int64_t m, int64_t n, int64_t lda, int64_t ldb) {
  const int sd = side_code(side);
  if (sd < 0) return 1;
  if (upper_code(uplo) < 0) return 2;
  if (trans_code(transa) < 0) return 3;
  if (diag_code(diag) < 0) return 4;
  if (m < 0) return 5;
  if (n < 0) return 6;
  if (lda < max1(sd == 0 ? m : n)) return 9;
  if (ldb < max1(m)) return 11;
  return 0;
}

// DTRSM scratch: the diagonal blocks' list and their 64 x 64 inverses
size_t trsm_scratch(size_t nblocks) {
  return up256(sizeof(TrsmBlock) * nblocks) + up256(sizeof(double) * 64 * 64 * nblocks);
}

// workspace of one DTRMM/DTRSM call: level-3 scratch, then the emulated GEMM workspace; for
// DTRSM `blocks` (if given) receives the diagonal blocks in the order the recursion visits them
size_t tri_workspace(bool solve, int side, int64_t m, int64_t n, int mode, std::vector<TrsmBlock>* blocks = nullptr) {
  if (m <= 0 || n <= 0) return 0;
  std::vector<TrsmBlock> local;
  if (!blocks) blocks = &local;
  blocks->clear();
  Ctx c;
  memset(&c, 0, sizeof(c));
  c.mode = mode;
  c.thresholds();
  c.dry = true;
  Tri t;
  memset(&t, 0, sizeof(t));
  t.c = &c;
  t.side = side;
  t.m = m;
  t.n = n;
  t.lda = side == 0 ? m : n;
  t.ldb = m;
  const int64_t order = side == 0 ? m : n;
  // the two triangle orientations issue transposed GEMM shapes: size for both (the diagonal
  // blocks are the same for both; they are listed once)
  for (int up = 0; up < 2; ++up) {
    t.upper = up;
    c.blocks = up == 0 ? blocks : nullptr;
    if (solve) t.trsm(0, order, 1.0);
    else t.trmm(0, order, 1.0);
  }
  const size_t scr = solve ? trsm_scratch(blocks->size()) : trmm_scratch(side, m, n);
  return scr + up256(c.need);
}

int tri_call(bool solve, char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha,
             const double* A, int64_t lda, double* B, int64_t ldb, int mode, double tol, void* workspace,
             size_t workspace_bytes, void* stream) {
  int rc = check_tri_args(side, uplo, transa, diag, m, n, lda, ldb);
  if (rc) return rc;
  if (mode != GBD_MODE_NATIVE && mode != GBD_MODE_EMULATED)
    return set_error(GBD_ERR_ARG, "level-3: mode must be GBD_MODE_NATIVE or GBD_MODE_EMULATED");
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = current_device(nullptr, nullptr))) return rc;
  if (alpha == 0.0) {  // B := 0, A not read
    const cudaError_t e = cudaMemset2DAsync(B, (size_t)ldb * 8, 0, (size_t)m * 8, (size_t)n, s);
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "level-3: zeroing B");
  }
  const int sd = side_code(side);
  std::vector<TrsmBlock> blocks;
  const size_t need = tri_workspace(solve, sd, m, n, mode, &blocks);
  if (need > 0 && (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)))
    return set_error(GBD_ERR_WORKSPACE, "%s: workspace must be 256-byte aligned and hold %zu bytes",
                     solve ? "dtrsm" : "dtrmm", need);
  const size_t scr = solve ? trsm_scratch(blocks.size()) : trmm_scratch(sd, m, n);
  Ctx c;
  c.mode = mode;
  c.thresholds();
  c.tol = tol;
  c.s = s;
  c.scr = static_cast<double*>(workspace);
  c.gws = static_cast<char*>(workspace) + scr;
  c.gwsb = workspace_bytes > scr ? workspace_bytes - scr : 0;
  c.dry = false;
  c.need = 0;
  Tri t;
  t.c = &c;
  t.side = sd;
  t.upper = upper_code(uplo);
  t.tr = trans_code(transa);
  t.unit = diag_code(diag);
  t.m = m;
  t.n = n;
  t.A = A;
  t.lda = lda;
  t.B = B;
  t.ldb = ldb;
  const int64_t order = sd == 0 ? m : n;
  if (solve) {  // invert every diagonal block first, all in one launch
    // the dry pass lists them in its recursion's order, which depends on the side: sort by row
    std::sort(blocks.begin(), blocks.end(), [](const TrsmBlock& x, const TrsmBlock& y) { return x.r0 < y.r0; });
    const size_t nb = blocks.size();
    TrsmBlock* dblocks = static_cast<TrsmBlock*>(workspace);
    c.dinv = reinterpret_cast<double*>(static_cast<char*>(workspace) + up256(sizeof(TrsmBlock) * nb));
    c.blocks = &blocks;
    cudaError_t e = cudaMemcpyAsync(dblocks, blocks.data(), sizeof(TrsmBlock) * nb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "dtrsm: the diagonal blocks' list");
    const int teff = sd == 0 ? t.tr : !t.tr;
    e = cudaFuncSetAttribute(k_trsm_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmInvSmem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(diagonal inversion)");
    k_trsm_invert<<<(unsigned)nb, 64, kTrsmInvSmem, s>>>(A, lda, dblocks, t.upper, t.unit, teff, c.dinv);
    if ((rc = c.check("diagonal inversion launch"))) return rc;
  }
  return solve ? t.trsm(0, order, alpha) : t.trmm(0, order, alpha);
}

}  // namespace
}  // namespace gbd

extern "C" {

size_t gbd_dsyrk_workspace_size(int64_t n, int64_t k, int mode) {
  using namespace gbd;
  if (n <= 0 || k < 0) return 0;
  Ctx c;
  memset(&c, 0, sizeof(c));
  c.mode = mode;
  c.thresholds();
  c.dry = true;
  Syrk y;
  memset(&y, 0, sizeof(y));
  y.c = &c;
  y.k = k;
  y.lda = n;
  y.ldc = n;
  y.beta = 1.0;
  for (int up = 0; up < 2; ++up) {  // the two triangles issue transposed GEMM shapes
    y.upper = up;
    y.run(0, n);
  }
  if (c.syrk_modular(n, k)) {
    const size_t w = gbd_dgemm_emu_mod_workspace_size(n, n, k, 0);
    if (w > c.need) c.need = w;
  }
  return syrk_scratch(n) + up256(c.need);
}

size_t gbd_dtrmm_workspace_size(char side, int64_t m, int64_t n, int mode) {
  const int sd = gbd::side_code(side);
  return sd < 0 ? 0 : gbd::tri_workspace(false, sd, m, n, mode);
}

size_t gbd_dtrsm_workspace_size(char side, int64_t m, int64_t n, int mode) {
  const int sd = gbd::side_code(side);
  return sd < 0 ? 0 : gbd::tri_workspace(true, sd, m, n, mode);
}

int gbd_dsyrk(char uplo, char trans, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, double beta,
              double* C, int64_t ldc, int mode, double tol, void* workspace, size_t workspace_bytes, void* stream) {
  using namespace gbd;
  const int up = upper_code(uplo), tr = trans_code(trans);
  if (up < 0) return 1;
  if (tr < 0) return 2;
  if (n < 0) return 3;
  if (k < 0) return 4;
  if (lda < max1(tr ? k : n)) return 7;
  if (ldc < max1(n)) return 10;
  if (mode != GBD_MODE_NATIVE && mode != GBD_MODE_EMULATED)
    return set_error(GBD_ERR_ARG, "dsyrk: mode must be GBD_MODE_NATIVE or GBD_MODE_EMULATED");
  if (n == 0 || ((alpha == 0.0 || k == 0) && beta == 1.0)) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  if ((rc = current_device(nullptr, nullptr))) return rc;
  if ((n + 7) / 8 > 65535) return set_error(GBD_ERR_LIMIT, "dsyrk: n above 524280 is not supported");
  if (alpha == 0.0 || k == 0) {
    k_tri_scale<<<grid2(n, n), 256, 0, s>>>(C, ldc, n, up, beta);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBD_OK : cuda_fail(e, "dsyrk: scaling launch");
  }
  const size_t need = gbd_dsyrk_workspace_size(n, k, mode);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return set_error(GBD_ERR_WORKSPACE, "dsyrk: workspace must be 256-byte aligned and hold %zu bytes", need);
  const size_t scr = syrk_scratch(n);
  Ctx c;
  c.mode = mode;
  c.thresholds();
  c.tol = tol;
  c.s = s;
  c.scr = static_cast<double*>(workspace);
  c.gws = static_cast<char*>(workspace) + scr;
  c.gwsb = workspace_bytes - scr;
  c.dry = false;
  c.need = 0;
  Syrk y;
  y.c = &c;
  y.upper = up;
  y.tr = tr;
  y.k = k;
  y.alpha = alpha;
  y.beta = beta;
  y.A = A;
  y.lda = lda;
  y.C = C;
  y.ldc = ldc;
  if (c.syrk_modular(n, k)) {  // one product over the triangle; the recursion when 16 moduli fall short
    rc = dgemm_emu_mod_tri(tr ? 'T' : 'N', tr ? 'N' : 'T', n, k, alpha, A, lda, A, lda, beta, C, ldc, up, tol, c.gws,
                           c.gwsb, s);
    if (rc != GBD_ERR_LIMIT) return rc;
  }
  return y.run(0, n);
}

int gbd_dtrmm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha, const double* A,
              int64_t lda, double* B, int64_t ldb, int mode, double tol, void* workspace, size_t workspace_bytes,
              void* stream) {
  return gbd::tri_call(false, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, mode, tol, workspace,
                       workspace_bytes, stream);
}

int gbd_dtrsm(char side, char uplo, char transa, char diag, int64_t m, int64_t n, double alpha, const double* A,
              int64_t lda, double* B, int64_t ldb, int mode, double tol, void* workspace, size_t workspace_bytes,
              void* stream) {
  return gbd::tri_call(true, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, mode, tol, workspace,
                       workspace_bytes, stream);
}

}  // extern "C"
