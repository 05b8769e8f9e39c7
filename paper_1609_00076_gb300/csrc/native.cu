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

#include "common.cuh"

namespace gbd {
namespace {

struct NativeArgs {
  int64_t m, n, k;
  double alpha, beta;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  unsigned int* err;
  int vec_c;  // C and ldc allow 16-byte stores at even rows
};

constexpr int kThreads = 128;
constexpr int kBK = 16;
constexpr int kStages = 4;

template <int BM, int BN>
constexpr size_t native_smem_bytes() {
  return (size_t)kStages * (BM * kBK + kBK * BN) * sizeof(double) + kStages * sizeof(uint64_t);
}

template <bool TA, bool TB, int BM, int BN, bool USE_TMA>
__global__ void __launch_bounds__(kThreads) k_native_dgemm(const NativeArgs p,
                                                           const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB) {
  constexpr int A_EL = BM * kBK, B_EL = kBK * BN;
  constexpr int WM = BM / 2, WN = BN / 2, MI = WM / 16, NI = WN / 8;
  static_assert(MI >= 1 && NI >= 1, "warp tile too small");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* sA = reinterpret_cast<double*>(smem_raw);  // [kStages][A_EL]
  double* sB = sA + kStages * A_EL;                  // [kStages][B_EL]
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * B_EL);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int nkb = (int)((p.k + kBK - 1) / kBK);
  const int wm0 = (warp >> 1) * WM, wn0 = (warp & 1) * WN;

  if (USE_TMA && tid == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // stage kb of the k loop into ring slot kb % kStages
  auto issue = [&](int kb) {
    const int s = kb % kStages;
    const int64_t k0 = (int64_t)kb * kBK;
    if (USE_TMA) {
      if (tid == 0 && kb < nkb) {
        mbar_arrive_expect_tx(&full[s], (uint32_t)((A_EL + B_EL) * sizeof(double)));
        if (!TA) tma_load_2d(sA + s * A_EL, &tmA, &full[s], (int)m0, (int)k0);
        else tma_load_2d(sA + s * A_EL, &tmA, &full[s], (int)k0, (int)m0);
        if (!TB) tma_load_2d(sB + s * B_EL, &tmB, &full[s], (int)k0, (int)n0);
        else tma_load_2d(sB + s * B_EL, &tmB, &full[s], (int)n0, (int)k0);
      }
    } else {
      if (kb < nkb) {
        double* a_s = sA + s * A_EL;
        double* b_s = sB + s * B_EL;
        for (int idx = tid; idx < A_EL; idx += kThreads) {
          int i, pk;
          if (!TA) { i = idx % BM; pk = idx / BM; }  // smem [BK][BM]
          else { pk = idx % kBK; i = idx / kBK; }    // smem [BM][BK]
          const int64_t gi = m0 + i, gp = k0 + pk;
          const bool ok = gi < p.m && gp < p.k;
          const double* src = ok ? (TA ? p.A + gi * p.lda + gp : p.A + gp * p.lda + gi) : p.A;
          cp_async_8(a_s + idx, src, ok);
        }
        for (int idx = tid; idx < B_EL; idx += kThreads) {
          int j, pk;
          if (!TB) { pk = idx % kBK; j = idx / kBK; }  // smem [BN][BK]
          else { j = idx % BN; pk = idx / BN; }        // smem [BK][BN]
          const int64_t gj = n0 + j, gp = k0 + pk;
          const bool ok = gj < p.n && gp < p.k;
          const double* src = ok ? (TB ? p.B + gp * p.ldb + gj : p.B + gj * p.ldb + gp) : p.B;
          cp_async_8(b_s + idx, src, ok);
        }
      }
      cp_async_commit();  // one group per stage, empty past the end, keeps the count uniform
    }
  };

  double acc[MI][NI][4];
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;

  for (int kb = 0; kb < kStages - 1; ++kb) issue(kb);

  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb % kStages;
    if (USE_TMA) mbar_wait(&full[s], (uint32_t)((kb / kStages) & 1), p.err, kErrWaitTma);
    else cp_async_wait<kStages - 2>();
    __syncthreads();  // tile kb visible to all; slot (kb-1) % kStages no longer read
    issue(kb + kStages - 1);

    const double* a_s = sA + s * A_EL;
    const double* b_s = sB + s * B_EL;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      double af[MI][8], bf[NI][4];
#pragma unroll
      for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = wm0 + mi * 16 + g + 8 * (q & 1);
          const int pk = kk + t + 4 * (q >> 1);
          af[mi][q] = TA ? a_s[i * kBK + pk] : a_s[pk * BM + i];
        }
#pragma unroll
      for (int ni = 0; ni < NI; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = wn0 + ni * 8 + g;
          const int pk = kk + t + 4 * q;
          bf[ni][q] = TB ? b_s[pk * BN + j] : b_s[j * kBK + pk];
        }
#pragma unroll
      for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni) dmma_16x8x16(acc[mi][ni], af[mi], bf[ni]);
    }
  }

  // ---- fused epilogue through shared memory, column by column ----
  __syncthreads();  // every load was consumed; the ring is free
  constexpr int LDS = BM + 2;
  double* sC = reinterpret_cast<double*>(smem_raw);  // [BN][LDS], column-major tile
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni) {
      const int r = wm0 + mi * 16 + g, c = wn0 + ni * 8 + 2 * t;
      sC[c * LDS + r] = acc[mi][ni][0];
      sC[(c + 1) * LDS + r] = acc[mi][ni][1];
      sC[c * LDS + r + 8] = acc[mi][ni][2];
      sC[(c + 1) * LDS + r + 8] = acc[mi][ni][3];
    }
  __syncthreads();
  const double alpha = p.alpha, beta = p.beta;
  for (int jj = warp; jj < BN; jj += kThreads / 32) {
    const int64_t j = n0 + jj;
    if (j >= p.n) break;
    double* ccol = p.C + j * p.ldc;
    for (int ii = 2 * lane; ii < BM; ii += 64) {
      const int64_t i = m0 + ii;
      if (i >= p.m) break;
      const double v0 = sC[jj * LDS + ii], v1 = sC[jj * LDS + ii + 1];
      if (p.vec_c && i + 1 < p.m) {
        double2* dst = reinterpret_cast<double2*>(ccol + i);
        double2 out;
        if (beta == 0.0) {
          out.x = alpha * v0;
          out.y = alpha * v1;
        } else {
          const double2 c0 = *dst;
          out.x = fma(alpha, v0, beta * c0.x);
          out.y = fma(alpha, v1, beta * c0.y);
        }
        *dst = out;
      } else {
        ccol[i] = (beta == 0.0) ? alpha * v0 : fma(alpha, v0, beta * ccol[i]);
        if (i + 1 < p.m) ccol[i + 1] = (beta == 0.0) ? alpha * v1 : fma(alpha, v1, beta * ccol[i + 1]);
      }
    }
  }
}

template <bool TA, bool TB, int BM, int BN, bool USE_TMA>
int launch_native(const NativeArgs& a, cudaStream_t stream) {
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  if (USE_TMA) {
    int rc;
    // A stored m x k ('N') or k x m ('T'); B stored k x n ('N') or n x k ('T')
    if (!TA) rc = encode_tmap_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.A, a.m, a.k, a.lda * 8, BM, kBK, CU_TENSOR_MAP_SWIZZLE_NONE);
    else rc = encode_tmap_2d(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.A, a.k, a.m, a.lda * 8, kBK, BM, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
    if (!TB) rc = encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.B, a.k, a.n, a.ldb * 8, kBK, BN, CU_TENSOR_MAP_SWIZZLE_NONE);
    else rc = encode_tmap_2d(&tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, a.B, a.n, a.k, a.ldb * 8, BN, kBK, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  constexpr size_t smem = native_smem_bytes<BM, BN>();
  static_assert(smem >= (size_t)BN * (BM + 2) * sizeof(double), "epilogue tile must fit the ring");
  auto kern = k_native_dgemm<TA, TB, BM, BN, USE_TMA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(native)");
  dim3 grid((unsigned)((a.m + BM - 1) / BM), (unsigned)((a.n + BN - 1) / BN));
  kern<<<grid, kThreads, smem, stream>>>(a, tmA, tmB);
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
