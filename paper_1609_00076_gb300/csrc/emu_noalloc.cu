// emu_noalloc.cu -- the split-emulation DGEMM for callers that must not allocate
// device memory.
//
// gbd_dgemm_emu needs a workspace (digit slices, exponents, running sums) that the
// caller normally allocates.  Some callers cannot do that: code running inside a
// real-time or safety-critical loop where an allocation may block or fail at an
// unpredictable moment, plug-ins whose host application owns every allocator, or
// code paths that run while an allocator lock is held.  For them this file keeps
// a fixed scratch area in the library itself: a file-scope __device__ array that
// every GPU using the library holds until process exit.  The entry point below
// calls no cudaMalloc, cudaFree or any other allocating routine.  Under lazy module
// loading (the CUDA default) the array is committed when this file's module first
// loads on a device, which the first call's address look-up triggers: that first
// call is the one that may wait for, or fail for lack of, the array's memory.
#include <mutex>

#include "emu.cuh"

namespace {

// Largest workspace the variant can use (see gbd_dgemm_emu_noalloc in the header).
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code cannot use
// the array's name as a device address (in host code it names a host-side stand-in),
// so the address is looked up once per device, with that device current.
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gbd::cuda_fail(e, "dgemm_emu_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return gbd::set_error(GBD_ERR_DEVICE, "dgemm_emu_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return gbd::cuda_fail(e, "dgemm_emu_noalloc: cudaGetSymbolAddress of the scratch array");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GBD_OK;
}

}  // namespace

extern "C" {

int gbd_dgemm_emu_noalloc(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                          const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                          int64_t ldc, int slices, double tol, gbd_emu_info* info, void* stream) {
  int rc = gbd::check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (slices < 0 || slices > gbd::emu::kMaxSlices)
    return gbd::set_error(GBD_ERR_ARG, "dgemm_emu_noalloc: slices must be 0 (automatic) or 1..%d",
                          gbd::emu::kMaxSlices);
  // the BLAS quick returns need no scratch at all: C := beta C (or nothing) without the array
  if (m == 0 || n == 0 || alpha == 0.0 || k == 0)
    return gbd_dgemm_emu(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, nullptr, 0, info,
                         stream);
  const size_t need = gbd_dgemm_emu_workspace_size(m, n, k, slices);
  if (need > kNoAllocScratchBytes)
    return gbd::set_error(GBD_ERR_LIMIT,
                          "dgemm_emu_noalloc: this problem needs %zu bytes of scratch; the built-in scratch holds "
                          "%zu bytes (use gbd_dgemm_emu with a caller workspace)",
                          need, kNoAllocScratchBytes);
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  // Phase timing would create CUDA events, which allocate: it is never done here.
  if (info) info->record_phases = 0;
  // gbd_dgemm_emu clears every part of the workspace that must start at zero
  // (exponents, flags, magnitude sums) before using it; the rest is overwritten.
  return gbd_dgemm_emu(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, scratch,
                       kNoAllocScratchBytes, info, stream);
}

}  // extern "C"
