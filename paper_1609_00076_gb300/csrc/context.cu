// context.cu -- the library context: one device, its properties, and a pool of workspaces
// owned by the library (one per stream, grown with stream-ordered allocations), behind the
// dgemm argument list of the paper (Section 1.2) plus the method and the accuracy target.
//
// A workspace is reused only by later calls on the same stream, which run after the earlier
// ones in stream order; growing it frees the old block in that stream's order too
// (cudaFreeAsync), so no call waits for another.  Calls on different streams get different
// workspaces and may run concurrently.
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>

#include "emu.cuh"

struct gbd_ctx {
  int device = 0;
  int sms = 0;
  std::mutex mu;
  struct Block {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::unordered_map<cudaStream_t, Block> pool;
};

namespace gbd {
namespace {

constexpr size_t kPoolAlign = 256;

// makes the context's device current for the duration of a call
struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    int cur = -1;
    if (ok && cudaGetDevice(&cur) == cudaSuccess && cur != prev && prev >= 0) cudaSetDevice(prev);
  }
};

bool valid_method(int method) {
  return method == GBD_METHOD_NATIVE || method == GBD_METHOD_SPLIT || method == GBD_METHOD_MODULAR ||
         method == GBD_METHOD_AUTO;
}

size_t method_workspace(int method, int64_t m, int64_t n, int64_t k) {
  switch (method) {
    case GBD_METHOD_NATIVE: return 0;
    case GBD_METHOD_SPLIT: return gbd_dgemm_emu_workspace_size(m, n, k, 0);
    case GBD_METHOD_MODULAR: return gbd_dgemm_emu_mod_workspace_size(m, n, k, 0);
    default: {  // automatic: the modular attempt, then the split one, in the same block
      const size_t a = gbd_dgemm_emu_mod_workspace_size(m, n, k, 0), b = gbd_dgemm_emu_workspace_size(m, n, k, 0);
      return a > b ? a : b;
    }
  }
}

// a workspace of at least `bytes` for work on `stream` (stream-ordered growth)
int pool_get(gbd_ctx* ctx, cudaStream_t stream, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return GBD_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  gbd_ctx::Block& b = ctx->pool[stream];
  if (b.bytes < bytes) {
    cudaError_t e;
    if (b.p && (e = cudaFreeAsync(b.p, stream)) != cudaSuccess) return cuda_fail(e, "context: cudaFreeAsync");
    b.p = nullptr;
    b.bytes = 0;
    const size_t want = (bytes + kPoolAlign - 1) & ~(kPoolAlign - 1);
    if ((e = cudaMallocAsync(&b.p, want, stream)) != cudaSuccess) {
      b.p = nullptr;
      return set_error(GBD_ERR_WORKSPACE, "context: cudaMallocAsync of %zu bytes failed: %s", want,
                       cudaGetErrorString(e));
    }
    b.bytes = want;
  }
  *out = b.p;
  return GBD_OK;
}

}  // namespace
}  // namespace gbd

extern "C" {

int gbd_create(gbd_ctx** out, int device) {
  using namespace gbd;
  if (!out) return set_error(GBD_ERR_ARG, "gbd_create: out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "gbd_create: cudaGetDeviceCount");
  if (device < 0 || device >= count) return set_error(GBD_ERR_DEVICE, "gbd_create: no device %d", device);
  DeviceScope scope(device);
  if (!scope.ok) return set_error(GBD_ERR_CUDA, "gbd_create: cannot make device %d current", device);
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  gbd_ctx* ctx = new (std::nothrow) gbd_ctx();
  if (!ctx) return set_error(GBD_ERR_WORKSPACE, "gbd_create: host allocation failed");
  ctx->device = device;
  ctx->sms = sms;
  *out = ctx;
  return GBD_OK;
}

void gbd_destroy(gbd_ctx* ctx) {
  if (!ctx) return;
  {
    gbd::DeviceScope scope(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto& kv : ctx->pool)
      if (kv.second.p) cudaFreeAsync(kv.second.p, kv.first);  // after the stream's last call
    ctx->pool.clear();
  }
  delete ctx;
}

int gbd_workspace_size(const gbd_ctx* ctx, int method, int64_t m, int64_t n, int64_t k, size_t* bytes) {
  (void)ctx;  // the sizes depend on the problem alone
  using namespace gbd;
  if (!bytes) return set_error(GBD_ERR_ARG, "gbd_workspace_size: bytes is NULL");
  *bytes = 0;
  if (!valid_method(method)) return set_error(GBD_ERR_ARG, "gbd_workspace_size: method %d", method);
  if (m < 0) return 3;
  if (n < 0) return 4;
  if (k < 0) return 5;
  *bytes = method_workspace(method, m, n, k);
  return GBD_OK;
}

int gbd_ctx_dgemm(gbd_ctx* ctx, int method, char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                  double tol, gbd_emu_info* info, void* stream) {
  using namespace gbd;
  if (!ctx) return set_error(GBD_ERR_ARG, "gbd_ctx_dgemm: context is NULL");
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (!valid_method(method)) return set_error(GBD_ERR_ARG, "gbd_ctx_dgemm: method %d", method);
  DeviceScope scope(ctx->device);
  if (!scope.ok) return set_error(GBD_ERR_CUDA, "gbd_ctx_dgemm: cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (method == GBD_METHOD_NATIVE) {
    if (info) {
      const int rp = info->record_phases;
      memset(info, 0, sizeof(*info));
      info->record_phases = rp;
      info->path = (m && n && k && alpha != 0.0) ? GBD_PATH_NATIVE : GBD_PATH_NONE;
    }
    return gbd_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
  }
  const bool quick = m == 0 || n == 0 || k == 0 || alpha == 0.0;
  void* ws = nullptr;
  const size_t need = quick ? 0 : method_workspace(method, m, n, k);
  if ((rc = pool_get(ctx, s, need, &ws))) return rc;
  if (method == GBD_METHOD_SPLIT)
    return gbd_dgemm_emu(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, ws, need, info, stream);
  rc = gbd_dgemm_emu_mod(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, ws, need, info, stream);
  if (method == GBD_METHOD_MODULAR || rc != GBD_ERR_LIMIT) return rc;
  // automatic: the target needs more than 16 moduli (C is untouched); the split emulation
  // certifies up to 9 slices and otherwise computes natively
  return gbd_dgemm_emu(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, ws, need, info, stream);
}

int gbd_ctx_dgemm_grouped(gbd_ctx* ctx, const gbd_problem* probs, int count, int* slices_used, void* stream) {
  using namespace gbd;
  if (!ctx) return set_error(GBD_ERR_ARG, "gbd_ctx_dgemm_grouped: context is NULL");
  DeviceScope scope(ctx->device);
  if (!scope.ok) return set_error(GBD_ERR_CUDA, "gbd_ctx_dgemm_grouped: cannot make device %d current", ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t need = gbd_dgemm_grouped_workspace_size(probs, count);
  void* ws = nullptr;
  int rc = pool_get(ctx, s, need, &ws);
  if (rc) return rc;
  return gbd_dgemm_grouped(probs, count, ws, need, slices_used, stream);
}

int gbd_sync_error(gbd_ctx* ctx, void* stream) {
  using namespace gbd;
  if (!ctx) return set_error(GBD_ERR_ARG, "gbd_sync_error: context is NULL");
  DeviceScope scope(ctx->device);
  if (!scope.ok) return set_error(GBD_ERR_CUDA, "gbd_sync_error: cannot make device %d current", ctx->device);
  return gbd_check_device_error(stream);
}

size_t gbd_ctx_pool_bytes(gbd_ctx* ctx) {
  if (!ctx) return 0;
  std::lock_guard<std::mutex> lk(ctx->mu);
  size_t total = 0;
  for (const auto& kv : ctx->pool) total += kv.second.bytes;
  return total;
}

}  // extern "C"
