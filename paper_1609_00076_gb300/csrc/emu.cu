// emu.cu -- host side of the split emulation: workspace sizing, slice-count
// selection and the launch sequence of gbd_dgemm_emu.
#include <cmath>
#include <cstdint>

#include <cstring>

#include "emu.cuh"

namespace gbd {
namespace emu {
namespace {

constexpr double kU = 1.1102230246251565e-16;  // 2^-53

// A-priori relative error of s slices (digits of b bits), as a fraction of
// |alpha| (|op(A)||op(B)|)_ij, for row/column magnitude sums mu, nu (in units of
// 2^sigma_i, 2^tau_j) and inner dimension k:
//   |err_ij| <= |alpha| 2^(sigma_i + tau_j - s b) (mu_i + nu_j + (s-1)(1+2^-b) k)
// and (|op(A)||op(B)|)_ij is estimated as 2^(sigma_i + tau_j) mu_i nu_j / k, with a
// safety factor of 8 for the estimate.
double relative_bound(int s, double mu_min, double nu_min, int64_t k) {
  const double kk = (double)k;
  const double trunc = std::ldexp(1.0, -s * kDigitBits) * (2.0 * kk + (s - 1) * (1.0 + std::ldexp(1.0, -kDigitBits)) * kk);
  const double ab = mu_min * nu_min / kk / 8.0;
  return ab > 0.0 ? trunc / ab : INFINITY;
}

}  // namespace

int choose_slices(double tol, double mu_min, double nu_min, int64_t k, double* bound) {
  for (int s = 1; s <= kMaxSlices; ++s) {
    const double b = relative_bound(s, mu_min, nu_min, k);
    if (b <= tol || s == kMaxSlices) {
      if (bound) *bound = b;
      return s;
    }
  }
  return kMaxSlices;
}

}  // namespace emu
}  // namespace gbd

extern "C" {

size_t gbd_dgemm_emu_workspace_size(int64_t m, int64_t n, int64_t k, int slices) {
  if (m < 0 || n < 0 || k < 0) return 0;
  if (slices <= 0 || slices > gbd::emu::kMaxSlices) slices = gbd::emu::kMaxSlices;
  return gbd::emu::layout(m, n, k, slices, nullptr, nullptr);
}

int gbd_dgemm_emu(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                  int64_t ldc, int slices, double tol, void* workspace, size_t workspace_bytes,
                  gbd_emu_info* info, void* stream) {
  using namespace gbd;
  using namespace gbd::emu;
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  const bool timing = info && info->record_phases;
  if (info) {
    info->prep_ms = 0.0;
    info->gemm_ms = 0.0;
    info->slices = 0;
    info->digit_bits = kDigitBits;
    info->products = 0;
    info->mu_min = 0.0;
    info->nu_min = 0.0;
    info->bound_est = 0.0;
  }
  if (slices < 0 || slices > kMaxSlices)
    return set_error(GBD_ERR_ARG, "dgemm_emu: slices must be 0 (automatic) or 1..%d", kMaxSlices);
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (alpha == 0.0 || k == 0) return scale_c(m, n, beta, C, ldc, s);
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim || (m + 63) / 64 > 65535 || (n + 63) / 64 > 65535)
    return set_error(GBD_ERR_LIMIT, "dgemm_emu: m, n below 4194240 and k below 2^31 are supported");
  rc = current_device(nullptr, nullptr);
  if (rc) return rc;

  const int s_ws = slices ? slices : kMaxSlices;
  const size_t need = layout(m, n, k, s_ws, nullptr, nullptr);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return set_error(GBD_ERR_WORKSPACE, "dgemm_emu: workspace must be 256-byte aligned and hold %zu bytes", need);
  Workspace ws;
  layout(m, n, k, s_ws, workspace, &ws);

  const int ta = trans_code(transa), tb = trans_code(transb);
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  struct EventGuard {
    cudaEvent_t* e;
    ~EventGuard() {
      for (int i = 0; i < 3; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  if (timing) {
    cudaError_t ee;
    for (int i = 0; i < 3; ++i)
      if ((ee = cudaEventCreate(&ev[i])) != cudaSuccess) return cuda_fail(ee, "dgemm_emu: cudaEventCreate");
    if ((ee = cudaEventRecord(ev[0], s)) != cudaSuccess) return cuda_fail(ee, "dgemm_emu: cudaEventRecord");
  }
  // op(A) rows: A[p*lda + i] when 'N' (rows contiguous), A[i*lda + p] when 'T'
  // op(B)^T rows (= columns j of op(B)): B[j*ldb + p] when 'N', B[p*ldb + j] when 'T'
  cudaError_t e;
  // both operand sides in one launch per step: op(A) (m rows of k) and op(B)^T (n rows of k)
  PrepPair pp;
  memset(&pp, 0, sizeof(pp));
  PrepJob& ja = pp.j[0];
  PrepJob& jb = pp.j[1];
  ja.X = A; ja.ld = lda; ja.R = m; ja.K = k; ja.rows_contig = ta == 0;
  ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = slices == 0 ? ws.muA : nullptr; ja.D = ws.DA; ja.kp = ws.kp;
  jb.X = B; jb.ld = ldb; jb.R = n; jb.K = k; jb.rows_contig = tb != 0;
  jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = slices == 0 ? ws.muB : nullptr; jb.D = ws.DB; jb.kp = ws.kp;
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);
  if ((rc = launch_exponents_pair(pp, exp_blocks, ws.ysum, ws.zero_bytes, s))) return rc;

  int s_use = slices;
  double bound = 0.0, mu_min = 0.0, nu_min = 0.0;
  if (slices == 0) {
    if ((rc = launch_magnitudes_pair(pp, exp_blocks, s))) return rc;
    if ((rc = launch_min_stats(ws.muA, m, ws.muB, n, ws.badA, ws.badB, ws.stats, s))) return rc;
    float st[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(st, ws.stats, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu: reading the magnitude statistics");
    mu_min = st[0] < 1e38f ? st[0] : 0.0;
    nu_min = st[1] < 1e38f ? st[1] : 0.0;
    const double target = tol > 0.0 ? tol : 2.0 * (double)k * kU;
    s_use = (mu_min > 0.0 && nu_min > 0.0) ? choose_slices(target, mu_min, nu_min, k, &bound) : 1;
  }
  ja.slices = s_use;
  jb.slices = s_use;
  if ((rc = launch_split_pair(pp, split_blocks, s))) return rc;
  // the slice tensors are laid out for s_use slices from the start of each region
  GemmParams gp;
  gp.m = m; gp.n = n; gp.k = k;
  gp.slices = s_use;
  gp.alpha = alpha; gp.beta = beta;
  gp.C = C; gp.ldc = ldc;
  gp.sigA = ws.sigA; gp.sigB = ws.sigB; gp.badA = ws.badA; gp.badB = ws.badB;
  if (timing && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu: cudaEventRecord");
  if ((rc = launch_slice_gemm(gp, ws, s))) return rc;
  if (timing) {
    float t0 = 0.f, t1 = 0.f;
    if ((e = cudaEventRecord(ev[2], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[2])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t0, ev[0], ev[1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t1, ev[1], ev[2])) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu: phase timing");
    info->prep_ms = t0;
    info->gemm_ms = t1;
  }
  if (info) {
    info->slices = s_use;
    info->products = s_use * (s_use + 1) / 2;
    info->mu_min = mu_min;
    info->nu_min = nu_min;
    info->bound_est = bound;
  }
  return GBD_OK;
}

}  // extern "C"
