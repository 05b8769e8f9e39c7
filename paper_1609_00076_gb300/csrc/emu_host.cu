// emu_host.cu -- the emulated DGEMMs (split or modular) on operands in host memory.
//
// The device buffer holds packed copies of the stored A and B (leading dimension =
// rows), the m x n result and the emulation workspace.  Every step is stream-ordered
// on the caller's stream: 2-D copies in, gbd_dgemm_emu or gbd_dgemm_emu_mod on the
// copies, a 2-D copy out.
#include "emu.cuh"

namespace {

constexpr size_t kAlign = 256;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct HostLayout {
  int64_t rows_a, cols_a, rows_b, cols_b;
  size_t off_a, off_b, off_c, off_ws, ws_bytes, total;
};

// packed device copies of A (rows_a x cols_a), B and C (m x n), then the workspace of the
// split (modular = false: `digits` slices) or modular (`digits` integer bits) emulation
HostLayout host_layout(char transa, char transb, int64_t m, int64_t n, int64_t k, int digits, bool modular) {
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
  L.ws_bytes = modular ? gbd_dgemm_emu_mod_workspace_size(m, n, k, digits) : gbd_dgemm_emu_workspace_size(m, n, k, digits);
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

// copies in, the emulated product, the copy out
int host_call(bool modular, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int digits, double tol,
              void* device_buffer, size_t buffer_bytes, gbd_emu_info* info, void* stream) {
  const char* name = modular ? "dgemm_emu_mod_host" : "dgemm_emu_host";
  int rc = gbd::check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (modular ? (digits < -1 || digits > 62) : (digits < 0 || digits > gbd::emu::kMaxSlices))
    return gbd::set_error(GBD_ERR_ARG, "%s: %s out of range", name, modular ? "bits" : "slices");
  if (m == 0 || n == 0) return GBD_OK;  // nothing to compute or copy
  const HostLayout L = host_layout(transa, transb, m, n, k, digits, modular);
  if (!device_buffer || buffer_bytes < L.total || (reinterpret_cast<uintptr_t>(device_buffer) & (kAlign - 1)))
    return gbd::set_error(GBD_ERR_WORKSPACE, "%s: the device buffer must hold %zu bytes and be 256-byte aligned",
                          name, L.total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(device_buffer);
  double* dA = reinterpret_cast<double*>(base + L.off_a);
  double* dB = reinterpret_cast<double*>(base + L.off_b);
  double* dC = reinterpret_cast<double*>(base + L.off_c);
  const bool need_ab = alpha != 0.0 && k > 0;
  cudaError_t e;
  if (need_ab) {
    if ((e = copy_2d(dA, L.rows_a, A, lda, L.rows_a, L.cols_a, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return gbd::cuda_fail(e, "emulated host call: copy of A");
    if ((e = copy_2d(dB, L.rows_b, B, ldb, L.rows_b, L.cols_b, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return gbd::cuda_fail(e, "emulated host call: copy of B");
  }
  if (beta != 0.0 && (e = copy_2d(dC, m, C, ldc, m, n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return gbd::cuda_fail(e, "emulated host call: copy of C");
  // leading dimensions of the packed copies (at least 1, as BLAS requires)
  const int64_t lda_d = L.rows_a > 1 ? L.rows_a : 1, ldb_d = L.rows_b > 1 ? L.rows_b : 1;
  rc = modular ? gbd_dgemm_emu_mod(transa, transb, m, n, k, alpha, dA, lda_d, dB, ldb_d, beta, dC, m, digits, tol,
                                   base + L.off_ws, L.ws_bytes, info, stream)
               : gbd_dgemm_emu(transa, transb, m, n, k, alpha, dA, lda_d, dB, ldb_d, beta, dC, m, digits, tol,
                               base + L.off_ws, L.ws_bytes, info, stream);
  if (rc) return rc;
  if ((e = copy_2d(C, ldc, dC, m, m, n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return gbd::cuda_fail(e, "emulated host call: copy of C back");
  return GBD_OK;
}

}  // namespace

extern "C" {

size_t gbd_dgemm_emu_host_buffer_size(char transa, char transb, int64_t m, int64_t n, int64_t k, int slices) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return host_layout(transa, transb, m, n, k, slices, false).total;
}

size_t gbd_dgemm_emu_mod_host_buffer_size(char transa, char transb, int64_t m, int64_t n, int64_t k, int bits) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return host_layout(transa, transb, m, n, k, bits, true).total;
}

int gbd_dgemm_emu_host(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int slices,
                       double tol, void* device_buffer, size_t buffer_bytes, gbd_emu_info* info, void* stream) {
  return host_call(false, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, tol, device_buffer,
                   buffer_bytes, info, stream);
}

int gbd_dgemm_emu_mod_host(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                           int64_t ldc, int bits, double tol, void* device_buffer, size_t buffer_bytes,
                           gbd_emu_info* info, void* stream) {
  return host_call(true, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits, tol, device_buffer,
                   buffer_bytes, info, stream);
}

}  // extern "C"
