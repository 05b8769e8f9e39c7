// emu_host.cu -- the split-emulation DGEMM on operands in host memory.
//
// The device buffer holds packed copies of the stored A and B (leading dimension =
// rows), the m x n result and the emulation workspace.  Every step is stream-ordered
// on the caller's stream: 2-D copies in, gbd_dgemm_emu on the copies, a 2-D copy out.
#include "emu.cuh"

namespace {

constexpr size_t kAlign = 256;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct HostLayout {
  int64_t rows_a, cols_a, rows_b, cols_b;
  size_t off_a, off_b, off_c, off_ws, ws_bytes, total;
};

// packed device copies of A (rows_a x cols_a), B and C (m x n), then the workspace
HostLayout host_layout(char transa, char transb, int64_t m, int64_t n, int64_t k, int slices) {
  HostLayout L{};
  const bool ta = !(transa == 'N' || transa == 'n');
  const bool tb = !(transb == 'N' || transb == 'n');
  L.rows_a = ta ? k : m;
  L.cols_a = ta ? m : k;
  L.rows_b = tb ? n : k;
  L.cols_b = tb ? k : n;
  size_t off = 0;
  L.off_a = off; off = up(off + sizeof(double) * (size_t)L.rows_a * (size_t)L.cols_a);
  L.off_b = off; off = up(off + sizeof(double) * (size_t)L.rows_b * (size_t)L.cols_b);
  L.off_c = off; off = up(off + sizeof(double) * (size_t)m * (size_t)n);
  L.off_ws = off;
  L.ws_bytes = gbd_dgemm_emu_workspace_size(m, n, k, slices);
  L.total = up(off + L.ws_bytes);
  return L;
}

// rows x cols doubles between a leading-dimension ld_src and ld_dst layout
cudaError_t copy_2d(double* dst, int64_t ld_dst, const double* src, int64_t ld_src, int64_t rows, int64_t cols,
                    cudaMemcpyKind kind, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  return cudaMemcpy2DAsync(dst, sizeof(double) * (size_t)ld_dst, src, sizeof(double) * (size_t)ld_src,
                           sizeof(double) * (size_t)rows, (size_t)cols, kind, s);
}

}  // namespace

extern "C" {

size_t gbd_dgemm_emu_host_buffer_size(char transa, char transb, int64_t m, int64_t n, int64_t k, int slices) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return host_layout(transa, transb, m, n, k, slices).total;
}

int gbd_dgemm_emu_host(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                       double tol, void* device_buffer, size_t buffer_bytes, gbd_emu_info* info, void* stream) {
  int rc = gbd::check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (slices < 0 || slices > gbd::emu::kMaxSlices)
    return gbd::set_error(GBD_ERR_ARG, "dgemm_emu_host: slices must be 0 (automatic) or 1..%d",
                          gbd::emu::kMaxSlices);
  if (m == 0 || n == 0) return GBD_OK;  // nothing to compute or copy
  const HostLayout L = host_layout(transa, transb, m, n, k, slices);
  if (!device_buffer || buffer_bytes < L.total || (reinterpret_cast<uintptr_t>(device_buffer) & (kAlign - 1)))
    return gbd::set_error(GBD_ERR_WORKSPACE,
                          "dgemm_emu_host: the device buffer must hold %zu bytes and be 256-byte aligned", L.total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(device_buffer);
  double* dA = reinterpret_cast<double*>(base + L.off_a);
  double* dB = reinterpret_cast<double*>(base + L.off_b);
  double* dC = reinterpret_cast<double*>(base + L.off_c);
  const bool need_ab = alpha != 0.0 && k > 0;
  cudaError_t e;
  if (need_ab) {
    if ((e = copy_2d(dA, L.rows_a, A, lda, L.rows_a, L.cols_a, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return gbd::cuda_fail(e, "dgemm_emu_host: copy of A");
    if ((e = copy_2d(dB, L.rows_b, B, ldb, L.rows_b, L.cols_b, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return gbd::cuda_fail(e, "dgemm_emu_host: copy of B");
  }
  if (beta != 0.0 && (e = copy_2d(dC, m, C, ldc, m, n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return gbd::cuda_fail(e, "dgemm_emu_host: copy of C");
  // leading dimensions of the packed copies (at least 1, as BLAS requires)
  const int64_t lda_d = L.rows_a > 1 ? L.rows_a : 1, ldb_d = L.rows_b > 1 ? L.rows_b : 1;
  rc = gbd_dgemm_emu(transa, transb, m, n, k, alpha, dA, lda_d, dB, ldb_d, beta, dC, m, slices, tol,
                     base + L.off_ws, L.ws_bytes, info, stream);
  if (rc) return rc;
  if ((e = copy_2d(C, ldc, dC, m, m, n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return gbd::cuda_fail(e, "dgemm_emu_host: copy of C back");
  return GBD_OK;
}

}  // extern "C"
