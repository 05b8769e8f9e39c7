// runtime.cu -- host-side plumbing of the library: error text, argument checks,
// device checks, the device error word and tensor-map encoding.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gbd {

namespace {
thread_local char g_msg[512] = "no error";

// Error word set by bounded device-side waits (one per device context; never
// allocated, so reading it needs no set-up beyond the symbol address).
__device__ unsigned int g_device_error = 0;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned int* g_err_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
int g_dev_ok[kMaxDevices] = {};  // 0 unknown, 1 ok, -1 not sm_103

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

// A bounded wait that nothing completes: the watchdog path of every kernel, exercised
// on purpose.  One thread waits on a fresh mbarrier's first phase for limit_ns, gives up,
// sets kErrWaitTma in the error word and the kernel ends normally.
__global__ void k_watchdog_selftest(unsigned int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(&bar, 0)) return;  // never: no thread arrives
    if ((it & 255u) == 0u && global_ns() - t0 > limit_ns) {
      atomicOr(err, kErrWaitTma);
      return;
    }
  }
}

// The FP64 tensor-core rate: every warp runs `iters` rounds of eight independent
// mma.sync.m16n8k16.f64 on register fragments (4096 flops each); the sums keep the
// results live.
__device__ double g_probe_sink;  // written only to keep the probe's products live

__global__ void __launch_bounds__(256) k_fp64_mma_probe(int64_t iters) {
  double a[8], b[4], d[8][4];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = 1.0 + 1e-3 * (threadIdx.x + q);
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = 1.0 - 1e-3 * (threadIdx.x + q);
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) d[r][q] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) dmma_16x8x16(d[r], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += d[r][q];
  if (s == 1234.5) g_probe_sink = s;  // practically never: only keeps the products alive
}

__global__ void k_scale_c(int64_t m, int64_t n, double beta, double* C, int64_t ldc) {
  const int64_t total = m * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    double* c = C + j * ldc + i;
    *c = (beta == 0.0) ? 0.0 : beta * *c;  // beta == 0: C is not read
  }
}
}  // namespace

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return set_error(GBD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int trans_code(char t) {
  if (t == 'N' || t == 'n') return 0;
  if (t == 'T' || t == 't' || t == 'C' || t == 'c') return 1;
  return -1;
}

int check_dgemm_args(char transa, char transb, int64_t m, int64_t n, int64_t k, int64_t lda,
                     int64_t ldb, int64_t ldc) {
  const int ta = trans_code(transa), tb = trans_code(transb);
  auto mx = [](int64_t a) { return a > 1 ? a : (int64_t)1; };
  int bad = 0;
  if (ta < 0) bad = 1;
  else if (tb < 0) bad = 2;
  else if (m < 0) bad = 3;
  else if (n < 0) bad = 4;
  else if (k < 0) bad = 5;
  else if (lda < mx(ta ? k : m)) bad = 8;
  else if (ldb < mx(tb ? n : k)) bad = 10;
  else if (ldc < mx(m)) bad = 13;
  if (bad) set_error(bad, "dgemm: parameter %d had an illegal value", bad);
  return bad;
}

int current_device(int* device, int* num_sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(GBD_ERR_DEVICE, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev_ok[dev] == 0) {
    int major = 0, minor = 0, sms = 0;
    if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return cuda_fail(e, "cudaDeviceGetAttribute");
    g_dev_ok[dev] = (major == 10 && minor == 3) ? 1 : -1;
    g_sm_count[dev] = sms;
    if (g_dev_ok[dev] < 0)
      return set_error(GBD_ERR_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a",
                       dev, major, minor);
  }
  if (g_dev_ok[dev] < 0) return set_error(GBD_ERR_DEVICE, "device %d is not sm_103", dev);
  if (device) *device = dev;
  if (num_sms) *num_sms = g_sm_count[dev];
  return GBD_OK;
}

// ---- page-locked staging for host-to-device table copies ----
namespace {
struct StagingBlock {
  void* p = nullptr;
  size_t bytes = 0;
  int device = -1;
  cudaEvent_t ev = nullptr;  // recorded after the block's last copies
  bool in_use = false;
};
std::mutex g_staging_mu;
std::vector<StagingBlock> g_staging;
constexpr size_t kStagingMin = (size_t)64 << 10;
}  // namespace

int staging_get(size_t bytes, int* handle, void** ptr) {
  *handle = -1;
  *ptr = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "staging: cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_staging_mu);
  for (size_t i = 0; i < g_staging.size(); ++i) {
    StagingBlock& b = g_staging[i];
    if (b.in_use || b.device != dev || b.bytes < bytes) continue;
    if (cudaEventQuery(b.ev) != cudaSuccess) continue;  // its copies have not run yet
    b.in_use = true;
    *handle = (int)i;
    *ptr = b.p;
    return GBD_OK;
  }
  StagingBlock b;
  b.bytes = kStagingMin;
  while (b.bytes < bytes) b.bytes *= 2;
  b.device = dev;
  if ((e = cudaHostAlloc(&b.p, b.bytes, cudaHostAllocDefault)) != cudaSuccess)
    return cuda_fail(e, "staging: cudaHostAlloc");
  if ((e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming)) != cudaSuccess) {
    cudaFreeHost(b.p);
    return cuda_fail(e, "staging: cudaEventCreate");
  }
  b.in_use = true;
  g_staging.push_back(b);
  *handle = (int)g_staging.size() - 1;
  *ptr = b.p;
  return GBD_OK;
}

int staging_put(int handle, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_staging_mu);
  if (handle < 0 || handle >= (int)g_staging.size()) return GBD_OK;
  StagingBlock& b = g_staging[handle];
  cudaError_t e = cudaEventRecord(b.ev, stream);
  b.in_use = false;
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "staging: cudaEventRecord");
}

unsigned int* device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_err_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    g_err_ptr[dev] = static_cast<unsigned int*>(p);
  }
  return g_err_ptr[dev];
}

int encode_tmap(CUtensorMap* out, CUtensorMapDataType dtype, int rank, const void* base,
                const uint64_t* dims, const uint64_t* pitches_bytes, const uint32_t* box,
                CUtensorMapSwizzle swizzle) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                       cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return set_error(GBD_ERR_CUDA, "cuTensorMapEncodeTiled entry point not found");
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
  }
  if (rank < 1 || rank > 5) return set_error(GBD_ERR_ARG, "tensor map rank %d", rank);
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = pitches_bytes[i];
  }
  CUresult r = g_encode(out, dtype, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(GBD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d): rank %d dims %llu x %llu box %u x %u",
                     (int)r, rank, (unsigned long long)dims[0], (unsigned long long)dims[1], box[0], box[1]);
  return GBD_OK;
}

int encode_tmap_2d(CUtensorMap* out, CUtensorMapDataType dtype, const void* base, uint64_t inner,
                   uint64_t outer, uint64_t pitch_bytes, uint32_t box_inner, uint32_t box_outer,
                   CUtensorMapSwizzle swizzle) {
  const uint64_t dims[2] = {inner, outer};
  const uint64_t pitches[1] = {pitch_bytes};
  const uint32_t box[2] = {box_inner, box_outer};
  return encode_tmap(out, dtype, 2, base, dims, pitches, box, swizzle);
}

int scale_c(int64_t m, int64_t n, double beta, double* C, int64_t ldc, cudaStream_t stream) {
  if (m == 0 || n == 0 || beta == 1.0) return GBD_OK;
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  const int64_t total = m * n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  k_scale_c<<<(unsigned)blocks, 256, 0, stream>>>(m, n, beta, C, ldc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "scale kernel launch");
}

}  // namespace gbd

extern "C" {

int gbd_version(void) { return 100; }  // 0.1.0

const char* gbd_last_error(void) { return gbd::g_msg; }

int gbd_fp64_mma_probe(int64_t iters, double* tflops, void* stream) {
  using namespace gbd;
  if (iters < 1 || !tflops) return set_error(GBD_ERR_ARG, "fp64_mma_probe: iters >= 1 and a result pointer");
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    return cuda_fail(e, "fp64_mma_probe: cudaEventCreate");
  const int blocks = 4 * sms, threads = 256;
  k_fp64_mma_probe<<<blocks, threads, 0, s>>>(iters / 8 + 1);  // warm-up
  cudaEventRecord(e0, s);
  k_fp64_mma_probe<<<blocks, threads, 0, s>>>(iters);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "fp64_mma_probe: timing");
  const double flops = 4096.0 * 8.0 * (double)iters * (double)(blocks * threads / 32);
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return GBD_OK;
}

int gbd_watchdog_selftest(int limit_ms, void* stream) {
  if (limit_ms < 1 || limit_ms > 10000) return gbd::set_error(GBD_ERR_ARG, "watchdog: limit_ms must be in 1..10000");
  int rc = gbd::current_device(nullptr, nullptr);
  if (rc) return rc;
  unsigned int* err = gbd::device_error_word();
  if (!err) return gbd::set_error(GBD_ERR_CUDA, "device error word not reachable");
  gbd::k_watchdog_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err, (unsigned long long)limit_ms * 1000000ull);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : gbd::cuda_fail(e, "watchdog self-test launch");
}

int gbd_check_device_error(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return gbd::cuda_fail(e, "cudaStreamSynchronize");
  unsigned int* p = gbd::device_error_word();
  if (!p) return gbd::set_error(GBD_ERR_CUDA, "device error word not reachable");
  unsigned int v = 0, zero = 0;
  if ((e = cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return gbd::cuda_fail(e, "read device error word");
  if (v == 0) return GBD_OK;
  if ((e = cudaMemcpy(p, &zero, sizeof(zero), cudaMemcpyHostToDevice)) != cudaSuccess)
    return gbd::cuda_fail(e, "clear device error word");
  if (v == gbd::kErrModRange)
    return gbd::set_error(GBD_ERR_LIMIT,
                          "a modular call in device-side automatic mode needed more than 16 moduli (its C is NaN)");
  return gbd::set_error(GBD_ERR_TIMEOUT, "a bounded device wait gave up (error bits 0x%x)", v);
}

}  // extern "C"
