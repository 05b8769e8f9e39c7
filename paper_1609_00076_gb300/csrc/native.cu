// native.cu -- native double-precision GEMM on the FP64 warp MMA (sm_103a).
//
// C := alpha*op(A)*op(B) + beta*C  (BLAS dgemm, paper Section 1.2), column-major
// with leading dimensions (Section 2.1).
//
// Design (GB300): FP64 arithmetic runs on a low-rate unit (about 1.05 TFLOP/s per
// GPU for both mma.sync f64 and DFMA), so this kernel is bound by the FP64 pipe,
// not by memory: the job of the tiling is to keep that pipe busy on every SM.
//  * CTA tile BM x BN (64x64 for large problems, 32x32 when 64x64 tiles would not
//    fill the 152 SMs), BK = 16, 4 warps in a 2x2 grid, each warp an
//    (BM/2) x (BN/2) block of m16n8k16 f64 MMAs with register accumulators.
//    This replaces the paper's register-blocked micro-kernel (Section 3.1).
//  * Tiles of op(A) and op(B) are staged in a STAGES-deep shared-memory ring.
//    With 16-byte aligned bases and even leading dimensions the Tensor Memory
//    Accelerator copies each tile (one elected thread, mbarrier completion,
//    out-of-range elements zero-filled); otherwise each element is copied with an
//    8-byte cp.async (zero-filled when out of range).  The shared-memory tile
//    takes the orientation of the stored matrix, so transposes cost nothing.
//    This replaces the packing of A_c and B_c (Section 3.1).
//  * Fused epilogue: the accumulator tile goes through shared memory and is
//    written down the columns of C (the paper's column walk, Section 2.2) with
//    16-byte vector stores when C and ldc allow: c = fma(alpha, acc, beta*c0),
//    or alpha*acc when beta == 0 (C0 not read).
#include <cstdint>
#include <cstring>

#include "native_tile.cuh"

namespace gbd {
namespace {

template <bool TA, bool TB, int BM, int BN, bool USE_TMA>
__global__ void __launch_bounds__(kNativeThreads) k_native_dgemm(const NativeArgs p,
                                                           const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  native_tile<TA, TB, BM, BN, USE_TMA>(p, &tmA, &tmB, (int64_t)blockIdx.x * BM, (int64_t)blockIdx.y * BN, smem_raw);
}

template <bool TA, bool TB, int BM, int BN, bool USE_TMA>
int launch_native(const NativeArgs& a, cudaStream_t stream) {
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  if (USE_TMA) {
    int rc;
    // A stored m x k ('N') or k x m ('T'); B stored k x n ('N') or n x k ('T')
    if (!TA) rc = encode_tmap_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.A, a.m, a.k, a.lda * 8, BM, kNativeBK, CU_TENSOR_MAP_SWIZZLE_NONE);
    else rc = encode_tmap_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.A, a.k, a.m, a.lda * 8, kNativeBK, BM, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
    if (!TB) rc = encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.B, a.k, a.n, a.ldb * 8, kNativeBK, BN, CU_TENSOR_MAP_SWIZZLE_NONE);
    else rc = encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.B, a.n, a.k, a.ldb * 8, BN, kNativeBK, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  constexpr size_t smem = native_smem_bytes<BM, BN>();
  static_assert(smem >= (size_t)BN * (BM + 2) * sizeof(double), "epilogue tile must fit the ring");
  auto kern = k_native_dgemm<TA, TB, BM, BN, USE_TMA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(native)");
  dim3 grid((unsigned)((a.m + BM - 1) / BM), (unsigned)((a.n + BN - 1) / BN));
  kern<<<grid, kNativeThreads, smem, stream>>>(a, tmA, tmB);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "native dgemm launch");
}

template <int BM, int BN, bool USE_TMA>
int dispatch_trans(int ta, int tb, const NativeArgs& a, cudaStream_t s) {
  if (!ta && !tb) return launch_native<false, false, BM, BN, USE_TMA>(a, s);
  if (ta && !tb) return launch_native<true, false, BM, BN, USE_TMA>(a, s);
  if (!ta && tb) return launch_native<false, true, BM, BN, USE_TMA>(a, s);
  return launch_native<true, true, BM, BN, USE_TMA>(a, s);
}

}  // namespace

// Tile choice: 64x64 unless that leaves SMs idle, then 32x32 (both FP64-pipe bound).
int native_dgemm(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                 int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 cudaStream_t stream) {
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  NativeArgs a;
  a.m = m; a.n = n; a.k = k;
  a.alpha = alpha; a.beta = beta;
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
  a.err = device_error_word();
  a.vec_c = ((reinterpret_cast<uintptr_t>(C) & 15u) == 0 && (ldc & 1) == 0) ? 1 : 0;
  const bool tma_ok = (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
                      (reinterpret_cast<uintptr_t>(B) & 15u) == 0 && (lda & 1) == 0 &&
                      (ldb & 1) == 0 && lda < ((int64_t)1 << 36) && ldb < ((int64_t)1 << 36);
  const bool use_tma = tma_ok;
  const int64_t tiles64 = ((m + 63) / 64) * ((n + 63) / 64);
  const bool big = tiles64 >= (int64_t)sms;
  if (big) return use_tma ? dispatch_trans<64, 64, true>(ta, tb, a, stream) : dispatch_trans<64, 64, false>(ta, tb, a, stream);
  return use_tma ? dispatch_trans<32, 32, true>(ta, tb, a, stream) : dispatch_trans<32, 32, false>(ta, tb, a, stream);
}

}  // namespace gbd

extern "C" {

int gbd_dgemm(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
              const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
              int64_t ldc, void* stream) {
  int rc = gbd::check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (alpha == 0.0 || k == 0) return gbd::scale_c(m, n, beta, C, ldc, s);
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim)
    return gbd::set_error(GBD_ERR_LIMIT, "dgemm: m, n and k must each be below 2^31");
  return gbd::native_dgemm(gbd::trans_code(transa), gbd::trans_code(transb), m, n, k, alpha, A, lda,
                           B, ldb, beta, C, ldc, s);
}

}  // extern "C"
