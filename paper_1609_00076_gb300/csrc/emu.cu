// emu.cu -- host side of the split emulation: workspace sizing, the certified
// slice-count choice and the launch sequence of gbd_dgemm_emu.
#include <cmath>
#include <cstdint>

#include <cstring>

#include "emu.cuh"

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
    const int rp = info->record_phases;
    memset(info, 0, sizeof(*info));
    info->record_phases = rp;
    info->digit_bits = kDigitBits;
  }
  if (slices < 0 || slices > kMaxSlices)
    return set_error(GBD_ERR_ARG, "dgemm_emu: slices must be 0 (automatic) or 1..%d", kMaxSlices);
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (alpha == 0.0 || k == 0) return scale_c(m, n, beta, C, ldc, s);
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim || (m + 63) / 64 > 65535 || (n + 63) / 64 > 65535)
    return set_error(GBD_ERR_LIMIT, "dgemm_emu: m, n below 4194240 and k below 2^31 are supported");
  int sms = 0;
  rc = current_device(nullptr, &sms);
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
  ja.emin = slices == 0 ? ws.eminA : nullptr;
  jb.emin = slices == 0 ? ws.eminB : nullptr;
  ja.st = ws.st[0];
  jb.st = ws.st[1];
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);

  int s_use = slices, exact = 0;
  double bound = 0.0, rho = 0.0, gamma = 0.0;
  if (slices == 0) {
    // the certified choice: one pass for the exponents, magnitude sums and FP8 magnitude planes (in
    // the slices' place), then the planes' product
    if ((e = cudaMemsetAsync(ws.cert, 0, sizeof(unsigned int) * kCertWords, s)) != cudaSuccess ||
        (ws.zero_bytes && (e = cudaMemsetAsync(ws.ysum, 0, ws.zero_bytes, s)) != cudaSuccess))
      return cuda_fail(e, "dgemm_emu: clearing the certification words");
    const int prec = cert_prec_default();
    if ((rc = launch_statplane_pair(pp, split_blocks, ws.cert + kCertTexA, ws.cert + kCertNormA, s))) return rc;
    if (prec == kCertBF16 && (rc = launch_magplane_pair(pp, prec, ws.cert + kCertTexA, split_blocks, s))) return rc;
    if ((rc = launch_cert(m, n, k, prec, ws.DA, ws.DB, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB, ws.eminA,
                          ws.eminB, ws.cert, nullptr, 0, sms, s)))
      return rc;
    unsigned int cw[kCertWords] = {};
    if ((e = cudaMemcpyAsync(cw, ws.cert, sizeof(cw), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu: reading the certification");
    cert_rho_gamma(cw, &rho, &gamma);
    const double target = tol > 0.0 ? tol : 2.0 * (double)k * kUnitRoundoff;
    s_use = cert_split_slices(rho, gamma, (int)cw[kCertTexA], (int)cw[kCertTexB], k, target, &bound, &exact);
    if (s_use > kMaxSlices && prec == kCertFP8) {  // the FP8 planes' looser bound: certify again with BF16 planes
      unsigned int* w2 = ws.cert + kCertRetry;
      if ((rc = launch_magplane_pair(pp, kCertBF16, w2 + kCertTexA, split_blocks, s))) return rc;
      if ((rc = launch_cert(m, n, k, kCertBF16, ws.DA, ws.DB, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB,
                            ws.eminA, ws.eminB, w2, nullptr, 0, sms, s)))
        return rc;
      if ((e = cudaMemcpyAsync(cw, w2, sizeof(unsigned int) * kCertRetry, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "dgemm_emu: reading the certification");
      cert_rho_gamma(cw, &rho, &gamma);
      s_use = cert_split_slices(rho, gamma, (int)cw[kCertTexA], (int)cw[kCertTexB], k, target, &bound, &exact);
    }
    if (s_use > kMaxSlices) {  // no slice count can be certified: the FP64 tensor-core path
      if (timing && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu: cudaEventRecord");
      if ((rc = gbd_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream))) return rc;
      if (info) {
        info->path = GBD_PATH_NATIVE;
        info->rho = rho;
        info->gamma = gamma;
        info->bound = 0.0;
        if (timing) {
          float t0 = 0.f, t1 = 0.f;
          if ((e = cudaEventRecord(ev[2], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[2])) != cudaSuccess ||
              (e = cudaEventElapsedTime(&t0, ev[0], ev[1])) != cudaSuccess ||
              (e = cudaEventElapsedTime(&t1, ev[1], ev[2])) != cudaSuccess)
            return cuda_fail(e, "dgemm_emu: phase timing");
          info->prep_ms = t0;
          info->gemm_ms = t1;
        }
      }
      return GBD_OK;
    }
  }
  if (slices != 0 && (rc = launch_exponents_pair(pp, exp_blocks, ws.ysum, ws.zero_bytes, s))) return rc;
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
    info->path = GBD_PATH_SPLIT;
    info->slices = s_use;
    info->products = s_use * (s_use + 1) / 2;
    info->exact = exact;
    info->rho = rho;
    info->gamma = gamma;
    info->bound = bound;
  }
  return GBD_OK;
}

}  // extern "C"
