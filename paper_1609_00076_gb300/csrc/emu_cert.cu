// emu_cert.cu -- the certified precision choice of both emulations of DGEMM.
//
// The a-priori truncation bound of element (i, j) is, in units of 2^(sigma_i + tau_j),
//   split (s slices of 7 bits):  2^-7s (mu_i + nu_j + (s - 1)(1 + 2^-7) k)
//   modular (t integer bits):    2^(-t-1) (mu_i + nu_j + k 2^(-t-1))
// and it has to stay within (tol - r u) G^_ij, G^_ij = sum_p |a^_ip||b^_pj| the scaled
// (|op(A)||op(B)|)_ij and r u the allowance for the final roundings.  A choice that meets this
// for every element needs G^_ij, an m x n x k quantity: this file bounds it from below with
// one BF16 product on the tensor cores of the magnitude planes (emu_split.cu, MagWriter), and
// reduces over the elements
//     rho = max (mu_i + nu_j) / G_ij,   gamma = max 1 / G_ij     (G_ij <= G^_ij)
// so that the choice needs only max of 2^(-t-1) (rho + k 2^(-t-1) gamma) <= tol - r u (and the
// split form).  Elements whose plane product is exactly zero have no error term (each term of
// |A||B| has a zero factor, which both emulations represent exactly) and are skipped.
//
// The lower bound: the planes hold v = RZ(max(|a^|, w) 2^S) with w = 2^(-63-S), so
//   sum_p v_a v_b 2^-2S <= G^ + k (2 w + w^2)
// and the FP32 accumulation of the non-negative BF16 products (exact in FP32) overshoots the
// exact sum by at most (number of accumulation steps) x 17 x 2^-24 of it; with at most 16384
// terms per chunk this is far below delta = min(k, 16384) 2^-19, so
//   G^_ij >= L_ij (1 - delta) 2^-2S - k (2w + w^2)
// with L_ij the FP32 result; chunk results are added rounding downward and every step of the
// epilogue rounds toward the safe side (__fmul_rd, __fsub_rd, __fdiv_ru).  S is the largest
// scale that keeps k 2^(2S) below 2^124 (no overflow of the FP32 accumulator).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "emu.cuh"
#include "tcgen05.cuh"

namespace gbd {
namespace emu {
namespace {

using namespace tc;

constexpr int kCBM = 128, kCBN = 128;
constexpr int kCStages = 6;
constexpr int kCEpiWarps = 16;  // 4 x 4 warps over 128 TMEM lanes x 128 columns
constexpr int kCThreads = 64 + 32 * kCEpiWarps;
constexpr int kCTmemCols = 2 * kCBN;         // two accumulators
constexpr int kCertChunkBlocks = 256;        // k-blocks of 64 per FP32 accumulation chunk (16384)
constexpr int kCCols = kCBN / (kCEpiWarps / 4);  // columns per epilogue thread

struct CertArgs {
  int64_t m, n;
  int nkb, tiles_m, num_tiles, group_m;
  float f;         // (1 - delta) 2^-2S, rounded down
  float slack;     // k (2 w + w^2), rounded up
  float mu_scale;  // upper-bound factor of the magnitude sums
  const unsigned long long* muA;  // [m] sum_p |a^_ip| in 32.32 fixed point
  const unsigned long long* muB;  // [n]
  const int* badA;
  const int* badB;
  const int* sigA;
  const int* sigB;
  unsigned int* words;  // [0] max rho, [1] max gamma (bits of non-negative floats)
  double* L;            // optional [m x n] output G_ij 2^(sigma_i + tau_j), leading dimension ldl
  int64_t ldl;
  unsigned int* err;
};

struct CSmem {
  static constexpr int kABytes = kCBM * kBK * 2;
  static constexpr int kBBytes = kCBN * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + kCStages * kABytes;
  static constexpr int kOffBar = kOffB + kCStages * kBBytes;
  static constexpr int kNumBars = 2 * kCStages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kBytes = kOffTmemSlot + 16;
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

// an upper bound of a magnitude sum held in 32.32 fixed point
__device__ __forceinline__ float mu_upper(unsigned long long q, float scale) {
  return __fmaf_ru((float)((double)q * 0x1p-32), scale, 0x1p-20f);
}

__global__ void __launch_bounds__(kCThreads, 1)
    k_cert_gemm(const __grid_constant__ CertArgs p, const __grid_constant__ CUtensorMap tmA,
                const __grid_constant__ CUtensorMap tmB) {
  using L = CSmem;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + kCStages;
  uint64_t* acc_full = bars + 2 * kCStages;
  uint64_t* acc_empty = bars + 2 * kCStages + 2;
  uint64_t* done = bars + 2 * kCStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmemSlot);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    for (int i = 0; i < kCStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 32 * kCEpiWarps);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(kCTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      const uint32_t bytes = (uint32_t)(L::kABytes + L::kBBytes);
      for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
        int tm, tn;
        tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
        for (int kb = 0; kb < p.nkb; ++kb) {
          mbar_wait(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
          mbar_arrive_expect_tx(&full[stage], bytes);
          tma_load_3d(smem + L::kOffA + stage * L::kABytes, &tmA, &full[stage], kb * kBK, tm * kCBM, 0);
          tma_load_3d(smem + L::kOffB + stage * L::kBBytes, &tmB, &full[stage], kb * kBK, tn * kCBN, 0);
          if (++stage == kCStages) { stage = 0; phase ^= 1u; }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kCBM, kCBN);
      uint32_t stage = 0, phase = 0, chunk = 0;
      const uint32_t a_base = smem_u32(smem + L::kOffA), b_base = smem_u32(smem + L::kOffB);
      for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x)
        for (int i0 = 0; i0 < p.nkb; i0 += kCertChunkBlocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
          tc_fence_after();
          const uint32_t dtm = tmem_base + buf * kCBN;
          const int i1 = min(p.nkb, i0 + kCertChunkBlocks);
          for (int it = i0; it < i1; ++it) {
            mbar_wait(&full[stage], phase, p.err, kErrWaitTma);
            tc_fence_after();
            const uint64_t da = smem_desc_sw128(a_base + stage * L::kABytes);
            const uint64_t db = smem_desc_sw128(b_base + stage * L::kBBytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              umma_bf16(dtm, da + 2 * kk, db + 2 * kk, idesc, (it > i0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[stage]);
            if (++stage == kCStages) { stage = 0; phase ^= 1u; }
          }
          umma_commit(&acc_full[buf]);
        }
      if (chunk > 0) {  // a CTA without a tile issued nothing and has nothing to wait for
        umma_commit(done);
        mbar_wait(done, 0, p.err, kErrWaitMma);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue ------------------------------
    const int quad = warp & 3;            // TMEM lanes 32 quad .. 32 quad + 31
    const int part = (warp - 2) >> 2;     // columns kCCols part ..
    const int row = quad * 32 + lane;
    const int col0 = part * kCCols;
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    float rmax = 0.0f, gmax = 0.0f;
    uint32_t chunk = 0;
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
      int tm, tn;
      tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
      const int64_t i = (int64_t)tm * kCBM + row;
      const int64_t jc0 = (int64_t)tn * kCBN + col0;
      float acc[kCCols];
      bool first = true;
      for (int i0 = 0; i0 < p.nkb; i0 += kCertChunkBlocks, ++chunk) {
        const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
        mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
        tc_fence_after();
        const uint32_t taddr = trow + buf * kCBN + col0;
#pragma unroll
        for (int q = 0; q < kCCols / 16; ++q) {
          uint32_t v[16];
          tmem_ld_16(taddr + q * 16, v);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            acc[q * 16 + jj] = first ? __uint_as_float(v[jj]) : __fadd_rd(acc[q * 16 + jj], __uint_as_float(v[jj]));
        }
        first = false;
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
      }
      if (i < p.m) {
        const bool rbad = p.badA[i] != 0;
        const float mui = rbad ? 0.0f : mu_upper(p.muA[i], p.mu_scale);
        const int si = p.L ? (p.sigA[i] == kExpEmpty ? 0 : p.sigA[i]) : 0;
#pragma unroll
        for (int c = 0; c < kCCols; ++c) {  // fully unrolled: acc stays in registers
          const int64_t j = jc0 + c;
          if (j < p.n) {
            if (rbad || p.badB[j] != 0) {  // a NaN row or column of the result: no bound applies
              if (p.L) p.L[i + j * p.ldl] = __longlong_as_double(0x7FF8000000000000ll);
              continue;
            }
            const float Lc = acc[c];
            float G = 0.0f;
            if (Lc > 0.0f) {
              G = __fsub_rd(__fmul_rd(Lc, p.f), p.slack);
              float rho = INFINITY, gam = INFINITY;
              if (G > 0.0f) {
                rho = __fdiv_ru(__fadd_ru(mui, mu_upper(p.muB[j], p.mu_scale)), G);
                gam = __frcp_ru(G);
              }
              rmax = fmaxf(rmax, rho);
              gmax = fmaxf(gmax, gam);
            }
            if (p.L) {
              const int tj = p.sigB[j] == kExpEmpty ? 0 : p.sigB[j];
              p.L[i + j * p.ldl] = G > 0.0f ? ldexp((double)G, si + tj) : 0.0;
            }
          }
        }
      }
    }
    // non-negative floats order as their bit patterns
    const unsigned rb = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
    const unsigned gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));
    if (lane == 0) {
      if (rb) atomicMax(p.words + 0, rb);
      if (gb) atomicMax(p.words + 1, gb);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kCTmemCols)
                 : "memory");
  }
}

float float_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
}
float float_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

}  // namespace

int plane_scale(int64_t k) {
  int kb = 0;
  while (((int64_t)1 << kb) < k) ++kb;
  return (124 - kb) / 2;
}

int launch_cert(int64_t m, int64_t n, int64_t k, const uint16_t* PA, const uint16_t* PB, int64_t kp,
                const unsigned long long* muA, const unsigned long long* muB, const int* badA, const int* badB,
                const int* sigA, const int* sigB, unsigned int* words, double* Lout, int64_t ldl, int sms,
                cudaStream_t stream) {
  if (m <= 0 || n <= 0 || k <= 0) return GBD_OK;
  const int S = plane_scale(k);
  CertArgs a;
  memset(&a, 0, sizeof(a));
  a.m = m;
  a.n = n;
  a.nkb = (int)((k + kBK - 1) / kBK);
  const double delta = (double)(k < 16384 ? k : 16384) * std::ldexp(1.0, -19);
  a.f = float_down(std::ldexp(1.0 - delta, -2 * S));
  const double w = std::ldexp(1.0, -63 - S);
  a.slack = float_up((double)k * (2.0 * w + w * w) * (1.0 + std::ldexp(1.0, -40)));
  const double nkr = (double)((k + 1023) / 1024);
  a.mu_scale = float_up(1.0 + std::ldexp(1.0, -10) + nkr * std::ldexp(1.0, -22));
  a.muA = muA;
  a.muB = muB;
  a.badA = badA;
  a.badB = badB;
  a.sigA = sigA;
  a.sigB = sigB;
  a.words = words;
  a.L = Lout;
  a.ldl = ldl;
  a.err = device_error_word();
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, 1u};
  const uint64_t pA[2] = {(uint64_t)kp * 2, (uint64_t)m * kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, (uint32_t)kCBM, 1u};
  int rc = encode_tmap(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, PA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, 1u};
  const uint64_t pB[2] = {(uint64_t)kp * 2, (uint64_t)n * kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, (uint32_t)kCBN, 1u};
  rc = encode_tmap(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, PB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  a.tiles_m = (int)((m + kCBM - 1) / kCBM);
  const int64_t tiles = (int64_t)a.tiles_m * ((n + kCBN - 1) / kCBN);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  const int grid = (int)(tiles < sms ? tiles : sms);
  a.group_m = group_rows(grid, kCBM, kCBN, a.tiles_m);
  cudaError_t e = cudaFuncSetAttribute(k_cert_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, CSmem::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(certification gemm)");
  k_cert_gemm<<<grid, kCThreads, CSmem::kAlloc, stream>>>(a, tmA, tmB);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "certification gemm launch");
}

}  // namespace emu
}  // namespace gbd

extern "C" {

size_t gbd_abs_product_lower_bound_workspace_size(int64_t m, int64_t n, int64_t k) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return gbd::emu::layout(m, n, k, 1, nullptr, nullptr, false);
}

int gbd_abs_product_lower_bound(char transa, char transb, int64_t m, int64_t n, int64_t k, const double* A,
                                int64_t lda, const double* B, int64_t ldb, double* L, int64_t ldl, void* workspace,
                                size_t workspace_bytes, void* stream) {
  using namespace gbd;
  using namespace gbd::emu;
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldl);
  if (rc) return rc == 13 ? 11 : rc;  // ldl is argument 11 of this list
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k == 0) return scale_c(m, n, 0.0, L, ldl, s);  // an empty sum: L = 0
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim)
    return set_error(GBD_ERR_LIMIT, "abs_product_lower_bound: m, n and k below 2^31 are supported");
  int sms = 0;
  if ((rc = current_device(nullptr, &sms))) return rc;
  const size_t need = layout(m, n, k, 1, nullptr, nullptr, false);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return set_error(GBD_ERR_WORKSPACE,
                     "abs_product_lower_bound: workspace must be 256-byte aligned and hold %zu bytes", need);
  Workspace ws;
  layout(m, n, k, 1, workspace, &ws, false);
  PrepPair pp;
  memset(&pp, 0, sizeof(pp));
  PrepJob& ja = pp.j[0];
  PrepJob& jb = pp.j[1];
  ja.X = A; ja.ld = lda; ja.R = m; ja.K = k; ja.rows_contig = trans_code(transa) == 0;
  ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = ws.muA; ja.D = ws.DA; ja.kp = ws.kp;
  jb.X = B; jb.ld = ldb; jb.R = n; jb.K = k; jb.rows_contig = trans_code(transb) != 0;
  jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = ws.muB; jb.D = ws.DB; jb.kp = ws.kp;
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);
  if ((rc = launch_exponents_pair(pp, exp_blocks, nullptr, 0, s))) return rc;
  if ((rc = launch_magnitudes_pair(pp, exp_blocks, s))) return rc;
  cudaError_t e = cudaMemsetAsync(ws.cert, 0, sizeof(unsigned int) * kCertWords, s);
  if (e != cudaSuccess) return cuda_fail(e, "abs_product_lower_bound: clearing the certification words");
  if ((rc = launch_magplane_pair(pp, plane_scale(k), ws.cert + 2, split_blocks, s))) return rc;
  return launch_cert(m, n, k, ws.DA, ws.DB, ws.kp, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB, ws.cert, L,
                     ldl, sms, s);
}

}  // extern "C"
