// common.cuh -- shared host/device helpers of the GB300 DGEMM library.
//
// Device side: inline-PTX wrappers for mbarriers, the Tensor Memory Accelerator
// (cp.async.bulk.tensor), per-element cp.async, and the FP64 warp MMA.
// Host side: argument checking with reference-BLAS error numbering, the
// per-thread error text, the per-device error word that bounded device waits
// set, and tensor-map encoding through the driver entry point.
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (types only; the driver is reached via cudaGetDriverEntryPointByVersion)
#include <cuda_runtime.h>

#include <cstdint>

#include "gbdgemm.h"

namespace gbd {

// ----------------------------------------------------------------------------
// host side (runtime.cu)
// ----------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
// 0 for 'N'/'n', 1 for 'T'/'t'/'C'/'c', -1 otherwise
int trans_code(char t);
// reference-BLAS argument check of the dgemm list; 0 or the index of the first bad argument
int check_dgemm_args(char transa, char transb, int64_t m, int64_t n, int64_t k, int64_t lda,
                     int64_t ldb, int64_t ldc);
// checks that the current device is sm_103 and returns its SM count
int current_device(int* device, int* num_sms);
// device pointer of the current device's error word (set by bounded waits)
unsigned int* device_error_word();
// 2-D tiled tensor map: dim0 (contiguous) = inner, dim1 = outer with row pitch in bytes
int encode_tmap_2d(CUtensorMap* out, CUtensorMapDataType dtype, const void* base, uint64_t inner,
                   uint64_t outer, uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer,
                   CUtensorMapSwizzle swizzle);
// tiled tensor map of any rank (dims[0] contiguous; pitches_bytes[i] = stride of dim i+1)
int encode_tmap(CUtensorMap* out, CUtensorMapDataType dtype, int rank, const void* base,
                const uint64_t* dims, const uint64_t* pitches_bytes, const uint32_t* box,
                CUtensorMapSwizzle swizzle);
// Page-locked staging blocks for host-to-device copies that must not synchronise: a block of at
// least `bytes` on the current device (reused once the copies recorded by its last staging_put
// have run; allocated the first time none is free), and its release after the copies from it
// were issued on `stream`.
int staging_get(size_t bytes, int* handle, void** ptr);
int staging_put(int handle, cudaStream_t stream);
// launches the C := beta*C quick path (alpha == 0 or k == 0)
int scale_c(int64_t m, int64_t n, double beta, double* C, int64_t ldc, cudaStream_t stream);
// (emu_mod.cu) C := alpha op(A) op(B) + beta C on the lower (upper != 0: upper) triangle of the
// n x n C only, by the modular emulation in automatic mode (bits chosen on the host, which
// synchronises `stream`): tiles off the triangle are skipped, elements off it neither read nor
// written.  alpha != 0, k > 0.  GBD_ERR_LIMIT (C untouched) when 16 moduli cannot reach `tol`.
int dgemm_emu_mod_tri(char transa, char transb, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int upper, double tol,
                      void* workspace, size_t workspace_bytes, cudaStream_t stream);

// error-word bits
constexpr unsigned int kErrWaitTma = 1u;     // a wait for a TMA tile gave up
constexpr unsigned int kErrWaitMma = 2u;     // a wait for MMA completion gave up
constexpr unsigned int kErrWaitEpi = 4u;     // a wait for the epilogue gave up
constexpr unsigned int kErrWaitSlot = 8u;    // a producer wait for a free stage gave up
constexpr unsigned int kErrTmemAlloc = 16u;  // TMEM allocation was not granted
constexpr unsigned int kErrModRange = 32u;   // a device-side automatic modular call needed more than 16 moduli

// time limit of every device-side wait, in nanoseconds of %globaltimer
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

// ----------------------------------------------------------------------------
// device side
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier; gives up after kWaitLimitNs, sets `code`
// in the error word and returns false.  Never spins forever.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned int* err,
                                          unsigned int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && global_ns() - t0 > kWaitLimitNs) {
      if (err) atomicOr(err, code);
      return false;
    }
  }
}

// TMA: 2-D tile load into shared memory, completion counted on `bar` (bytes)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// 8-byte asynchronous copy global -> shared; zero-fills when !pred (nothing is read)
__device__ __forceinline__ void cp_async_8(void* dst, const void* src, bool pred) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(pred ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// FP64 warp MMA, D(16x8) += A(16x16, row) * B(16x8, col).
// Fragment layout (lane = 4*g + t):  a[q] = A(g + 8*(q&1), t + 4*(q>>1)),
// b[q] = B(t + 4*q, g),  d[0..1] = D(g, 2t..2t+1), d[2..3] = D(g+8, 2t..2t+1).
__device__ __forceinline__ void dmma_16x8x16(double* d, const double* a, const double* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
        "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

}  // namespace gbd
