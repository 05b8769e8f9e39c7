// emu_mod.cu -- the modular emulation of DGEMM (Ozaki, Uchino and Imamura, "Ozaki Scheme
// II: a GEMM-oriented emulation of floating-point matrix multiplication using an integer
// modular technique", 2025) on the 5th-generation tensor cores.
//
//   1. sigma_i, tau_j: the row and column exponents of the split emulation (emu_split.cu).
//   2. A' = rint(a 2^(t - sigma_i)), B' = rint(b 2^(t - tau_j)) (integers, |.| <= 2^t), and
//      their symmetric residues modulo n pairwise coprime moduli p_l <= 256, written as BF16
//      slices (emu_split.cu, k_residue_pair).
//   3. For every modulus: the residue product on tcgen05.mma with 1024-deep exact FP32
//      chunks drained into int32, reduced modulo p_l; the epilogue stores one byte per
//      element, u_l = (residue x c_l) mod p_l with c_l = (M/p_l)^-1 mod p_l.
//   4. k_crt: C' = sum_l u_l (M/p_l) mod M, the unique integer of (-M/2, M/2] congruent to
//      the products; it equals A'B' because M > 2 k 2^(2t) >= 2 max|A'B'|.  Then
//      C := fma(alpha 2^(tau_j - 2t), fl(C') 2^sigma_i, beta C0), fl correctly rounded.
// There is no FP64 arithmetic in the products: n GEMMs replace the s(s+1)/2 of the split
// emulation.  All waits are bounded (2 s) and set the device error word when they give up.
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "emu.cuh"
#include "tcgen05.cuh"

namespace gbd {
namespace emu {
namespace {

using namespace tc;

constexpr int kBM = 128, kBN = 128;
constexpr int kStages = 6;
constexpr int kEpiWarps = 16;  // 4 x 4 warps over 128 TMEM lanes x 128 columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kCols = kBN / (kEpiWarps / 4);  // columns per epilogue thread
constexpr int kTmemCols = 2 * kBN;             // two accumulators
constexpr int kReduceChunks = 64;              // int32 stays exact for 64 chunks of 1024 k

struct Smem {
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = kBN * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + kStages * kABytes;
  static constexpr int kOffBar = kOffB + kStages * kBBytes;
  static constexpr int kNumBars = 2 * kStages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kBytes = kOffTmemSlot + 16;
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

struct ModArgs {
  int64_t m, n;
  int nkb, nmod;
  int tiles_m, num_tiles, group_m;
  int p[kMaxModuli];  // moduli
  int c[kMaxModuli];  // (M/p_l)^-1 mod p_l
  uint8_t* U;         // [nmod][n][m] bytes u_l
  unsigned int* err;
};

// v mod p in [0, p) for a 32-bit integer of either sign
__device__ __forceinline__ int mod_nonneg(int v, int p) {
  int r = v % p;
  return r < 0 ? r + p : r;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mod_gemm(const ModArgs p, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
  using L = Smem;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = bars + 2 * kStages + 2;
  uint64_t* done = bars + 2 * kStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmemSlot);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 32 * kEpiWarps);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(kTmemCols)
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
        for (int l = 0; l < p.nmod; ++l)
          for (int kb = 0; kb < p.nkb; ++kb) {
            mbar_wait(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
            mbar_arrive_expect_tx(&full[stage], bytes);
            tma_load_3d(smem + L::kOffA + stage * L::kABytes, &tmA, &full[stage], kb * kBK, tm * kBM, l);
            tma_load_3d(smem + L::kOffB + stage * L::kBBytes, &tmB, &full[stage], kb * kBK, tn * kBN, l);
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kBM, kBN);
      uint32_t stage = 0, phase = 0, chunk = 0;
      const uint32_t a_base = smem_u32(smem + L::kOffA), b_base = smem_u32(smem + L::kOffB);
      for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x)
        for (int l = 0; l < p.nmod; ++l)
          for (int i0 = 0; i0 < p.nkb; i0 += kChunkBlocks, ++chunk) {
            const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
            mbar_wait(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
            tc_fence_after();
            const uint32_t dtm = tmem_base + buf * kBN;
            const int i1 = min(p.nkb, i0 + kChunkBlocks);
            for (int it = i0; it < i1; ++it) {
              mbar_wait(&full[stage], phase, p.err, kErrWaitTma);
              tc_fence_after();
              const uint64_t da = smem_desc_sw128(a_base + stage * L::kABytes);
              const uint64_t db = smem_desc_sw128(b_base + stage * L::kBBytes);
#pragma unroll
              for (int kk = 0; kk < kBK / 16; ++kk)
                umma_bf16(dtm, da + 2 * kk, db + 2 * kk, idesc, (it > i0 || kk > 0) ? 1u : 0u);
              umma_commit(&empty[stage]);
              if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
            umma_commit(&acc_full[buf]);
          }
      umma_commit(done);
      mbar_wait(done, 0, p.err, kErrWaitMma);
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue ----------------------------------
    // each modulus: exact int32 sums of the drained chunks, then one residue byte
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int part = ew >> 2;
    const int row = quad * 32 + lane;
    const int col0 = part * kCols;
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    const int64_t plane = p.m * p.n;
    uint32_t chunk = 0;
    int acc[kCols];
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
      int tm, tn;
      tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
      const int64_t i = (int64_t)tm * kBM + row;
      const int64_t jc0 = (int64_t)tn * kBN + col0;
      for (int l = 0; l < p.nmod; ++l) {
        const int pm = p.p[l];
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = 0;
        int nch = 0;
        for (int i0 = 0; i0 < p.nkb; i0 += kChunkBlocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
          tc_fence_after();
          const uint32_t taddr = trow + buf * kBN + col0;
#pragma unroll
          for (int q = 0; q < kCols / 16; ++q) {
            uint32_t v[16];
            tmem_ld_16(taddr + q * 16, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[q * 16 + jj] += __float2int_rn(__uint_as_float(v[jj]));
          }
          tc_fence_before();
          mbar_arrive(&acc_empty[buf]);
          if (++nch == kReduceChunks) {  // keep the running sums inside int32
            nch = 0;
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] = mod_nonneg(acc[c], pm);
          }
        }
        const int cl = p.c[l];
        uint8_t* u = p.U + (int64_t)l * plane + jc0 * p.m + i;
        if (i < p.m) {
#pragma unroll
          for (int c = 0; c < kCols; ++c)
            if (jc0 + c < p.n) u[(int64_t)c * p.m] = (uint8_t)((mod_nonneg(acc[c], pm) * cl) % pm);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kTmemCols)
                 : "memory");
  }
}

// ---- the two-SM form: 256 x 256 tiles on a CTA pair (tcgen05 cta_group::2) ----
// Each CTA stages 128 rows of A and 128 rows of op(B)^T per k-block; the leader's single
// MMA thread multiplies the pair's 256 x 64 by 64 x 256 into both CTAs' TMEM (128 lanes x
// 256 columns each), so every staged byte feeds twice the flops of the one-SM form.
constexpr int k2BM = 256, k2BN = 256;
constexpr int k2Stages = 6;
constexpr int k2EpiWarps = 16;  // 4 x 4 warps over 128 TMEM lanes x 256 columns
constexpr int k2Threads = 64 + 32 * k2EpiWarps;
constexpr int k2Cols = k2BN / (k2EpiWarps / 4);
constexpr int k2TmemCols = 2 * k2BN;

struct Smem2 {
  static constexpr int kABytes = 128 * kBK * 2;
  static constexpr int kBBytes = 128 * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + k2Stages * kABytes;
  static constexpr int kOffBar = kOffB + k2Stages * kBBytes;
  static constexpr int kNumBars = 2 * k2Stages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kBytes = kOffTmemSlot + 16;
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(k2Threads, 1)
    k_mod_gemm_pair(const ModArgs p, const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB) {
  using L = Smem2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + k2Stages;
  uint64_t* acc_full = bars + 2 * k2Stages;
  uint64_t* acc_empty = bars + 2 * k2Stages + 2;
  uint64_t* done = bars + 2 * k2Stages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmemSlot);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int num_pairs = gridDim.x / 2, pair_id = blockIdx.x / 2;

  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    for (int i = 0; i < k2Stages; ++i) {
      mbar_init(&full[i], 1);   // the leader's producer arrives (with both CTAs' bytes)
      mbar_init(&empty[i], 1);  // one commit per phase, multicast to both CTAs
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 2 * 32 * k2EpiWarps);  // every epilogue thread of both CTAs
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(k2TmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // the peer's barriers are initialised and its TMEM is allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer (both CTAs) ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      const uint32_t pair_bytes = (uint32_t)(2 * (L::kABytes + L::kBBytes));
      for (int tile = pair_id; tile < p.num_tiles; tile += num_pairs) {
        int tm, tn;
        tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
        const int m0 = tm * k2BM + (int)rank * 128;
        const int nb0 = tn * k2BN + (int)rank * 128;
        for (int l = 0; l < p.nmod; ++l)
          for (int kb = 0; kb < p.nkb; ++kb) {
            mbar_wait_cluster(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
            if (leader) mbar_arrive_expect_tx(&full[stage], pair_bytes);
            const uint32_t fbar = map_to_rank(smem_u32(&full[stage]), 0);
            tma_load_3d_pair(smem + L::kOffA + stage * L::kABytes, &tmA, fbar, kb * kBK, m0, l);
            tma_load_3d_pair(smem + L::kOffB + stage * L::kBBytes, &tmB, fbar, kb * kBK, nb0, l);
            if (++stage == k2Stages) { stage = 0; phase ^= 1u; }
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer (leader CTA) ------------------------------
    if (leader && lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(k2BM, k2BN);
      uint32_t stage = 0, phase = 0, chunk = 0;
      const uint32_t a_base = smem_u32(smem + L::kOffA), b_base = smem_u32(smem + L::kOffB);
      for (int tile = pair_id; tile < p.num_tiles; tile += num_pairs)
        for (int l = 0; l < p.nmod; ++l)
          for (int i0 = 0; i0 < p.nkb; i0 += kChunkBlocks, ++chunk) {
            const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
            mbar_wait_cluster(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
            tc_fence_after();
            const uint32_t dtm = tmem_base + buf * k2BN;
            const int i1 = min(p.nkb, i0 + kChunkBlocks);
            for (int it = i0; it < i1; ++it) {
              mbar_wait_cluster(&full[stage], phase, p.err, kErrWaitTma);
              tc_fence_after();
              const uint64_t da = smem_desc_sw128(a_base + stage * L::kABytes);
              const uint64_t db = smem_desc_sw128(b_base + stage * L::kBBytes);
#pragma unroll
              for (int kk = 0; kk < kBK / 16; ++kk)
                umma_bf16_pair(dtm, da + 2 * kk, db + 2 * kk, idesc, (it > i0 || kk > 0) ? 1u : 0u);
              umma_commit_pair(&empty[stage]);  // frees this stage in both CTAs
              if (++stage == k2Stages) { stage = 0; phase ^= 1u; }
            }
            umma_commit_pair(&acc_full[buf]);  // chunk complete in both CTAs' TMEM
          }
      umma_commit_pair(done);
      mbar_wait_cluster(done, 0, p.err, kErrWaitMma);
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue (both CTAs) ------------------------------
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int part = ew >> 2;
    const int row = quad * 32 + lane;
    const int col0 = part * k2Cols;
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    const int64_t plane = p.m * p.n;
    uint32_t empty_remote[2];
    empty_remote[0] = map_to_rank(smem_u32(&acc_empty[0]), 0);
    empty_remote[1] = map_to_rank(smem_u32(&acc_empty[1]), 0);
    uint32_t chunk = 0;
    int acc[k2Cols];
    for (int tile = pair_id; tile < p.num_tiles; tile += num_pairs) {
      int tm, tn;
      tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
      const int64_t i = (int64_t)tm * k2BM + rank * 128 + row;
      const int64_t jc0 = (int64_t)tn * k2BN + col0;
      for (int l = 0; l < p.nmod; ++l) {
        const int pm = p.p[l];
#pragma unroll
        for (int c = 0; c < k2Cols; ++c) acc[c] = 0;
        int nch = 0;
        for (int i0 = 0; i0 < p.nkb; i0 += kChunkBlocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
          tc_fence_after();
          const uint32_t taddr = trow + buf * k2BN + col0;
#pragma unroll
          for (int q = 0; q < k2Cols / 16; ++q) {
            uint32_t v[16];
            tmem_ld_16(taddr + q * 16, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[q * 16 + jj] += __float2int_rn(__uint_as_float(v[jj]));
          }
          tc_fence_before();
          mbar_arrive_remote(empty_remote[buf]);
          if (++nch == kReduceChunks) {  // keep the running sums inside int32
            nch = 0;
#pragma unroll
            for (int c = 0; c < k2Cols; ++c) acc[c] = mod_nonneg(acc[c], pm);
          }
        }
        const int cl = p.c[l];
        uint8_t* u = p.U + (int64_t)l * plane + jc0 * p.m + i;
        if (i < p.m) {
#pragma unroll
          for (int c = 0; c < k2Cols; ++c)
            if (jc0 + c < p.n) u[(int64_t)c * p.m] = (uint8_t)((mod_nonneg(acc[c], pm) * cl) % pm);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA leaves while the pair still uses its shared memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(k2TmemCols)
                 : "memory");
  }
}

// ---- Chinese remainder reconstruction and the FP64 result ----
struct CrtArgs {
  int64_t m, n, ldc;
  int nmod, t;
  uint64_t mp_lo[kMaxModuli], mp_hi[kMaxModuli];  // M / p_l
  float inv[kMaxModuli];                          // 1 / p_l
  uint64_t M_lo, M_hi, half_lo, half_hi;          // M and floor(M/2)
  double alpha, beta;
  double* C;
  const int* sigA;
  const int* sigB;
  const int* badA;
  const int* badB;
  const uint8_t* U;
};

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 make_u128(uint64_t hi, uint64_t lo) { return ((u128)hi << 64) | lo; }

// a 128-bit integer of either sign as the nearest double (ties to even)
__device__ __forceinline__ double i128_to_double(u128 v) {
  const bool neg = (uint64_t)(v >> 127) != 0;
  const u128 a = neg ? (u128)0 - v : v;
  const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
  if (hi == 0 && lo < (1ull << 53)) {
    const double d = (double)lo;
    return neg ? -d : d;
  }
  const int nbits = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  const int shift = nbits - 53;  // >= 1
  uint64_t mant = (uint64_t)(a >> shift);
  const u128 rem = a & (((u128)1 << shift) - 1), half = (u128)1 << (shift - 1);
  int e = shift;
  if (rem > half || (rem == half && (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++e;
    }
  }
  const double d = ldexp((double)mant, e);  // mant < 2^53, e < 128: exact
  return neg ? -d : d;
}

__global__ void __launch_bounds__(256) k_crt(const __grid_constant__ CrtArgs a) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.m) return;
  const int sig = a.sigA[row] == kExpEmpty ? 0 : a.sigA[row];
  const bool bad_r = a.badA[row] != 0;
  const u128 M = make_u128(a.M_hi, a.M_lo), half = make_u128(a.half_hi, a.half_lo);
  const int64_t plane = a.m * a.n;
  for (int64_t col = blockIdx.y; col < a.n; col += gridDim.y) {
    const int64_t e = col * a.m + row;
    u128 s = 0;
    float qf = 0.0f;
    for (int l = 0; l < a.nmod; ++l) {
      const uint32_t u = a.U[(int64_t)l * plane + e];
      s += (u128)u * make_u128(a.mp_hi[l], a.mp_lo[l]);  // modulo 2^128
      qf += (float)u * a.inv[l];
    }
    // sum_l u_l (M/p_l) = C'_u + q M with q = floor(sum_l u_l/p_l); the float estimate of q
    // is off by at most one, which the range of the difference reveals
    u128 cu = s - (u128)(uint64_t)floorf(qf) * M;
    if ((uint64_t)(cu >> 127)) cu += M;  // q was one too large
    else if (cu >= M) cu -= M;           // one too small
    const u128 v = cu > half ? cu - M : cu;  // the symmetric representative
    const double x = i128_to_double(v);
    const int tau = a.sigB[col] == kExpEmpty ? 0 : a.sigB[col];
    double w = a.beta != 0.0 ? a.beta * a.C[col * a.ldc + row] : 0.0;
    if (bad_r || a.badB[col]) w = __longlong_as_double(0x7FF8000000000000ll);
    else w = fma(ldexp(a.alpha, tau - 2 * a.t), ldexp(x, sig), w);
    a.C[col * a.ldc + row] = w;
  }
}

// ---- host side ----
struct ModWorkspace {
  int* sigA;
  int* sigB;
  int* badA;
  int* badB;
  unsigned long long* muA;
  unsigned long long* muB;
  float* stats;
  uint16_t* DA;  // [nmod][m][kp]
  uint16_t* DB;  // [nmod][n][kp]
  uint8_t* U;    // [nmod][n][m]
  int64_t kp;
};

size_t mod_layout(int64_t m, int64_t n, int64_t k, int nmod, void* base, ModWorkspace* ws) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t kp = (k + 7) / 8 * 8;
  size_t off = 0;
  const size_t o_sigA = off; off = up(off + sizeof(int) * (size_t)m);
  const size_t o_sigB = off; off = up(off + sizeof(int) * (size_t)n);
  const size_t o_badA = off; off = up(off + sizeof(int) * (size_t)m);
  const size_t o_badB = off; off = up(off + sizeof(int) * (size_t)n);
  const size_t o_muA = off; off = up(off + sizeof(unsigned long long) * (size_t)m);
  const size_t o_muB = off; off = up(off + sizeof(unsigned long long) * (size_t)n);
  const size_t o_stats = off; off = up(off + sizeof(float) * 4);
  const size_t o_DA = off; off = up(off + 2 * (size_t)nmod * (size_t)m * (size_t)kp);
  const size_t o_DB = off; off = up(off + 2 * (size_t)nmod * (size_t)n * (size_t)kp);
  const size_t o_U = off; off = up(off + (size_t)nmod * (size_t)m * (size_t)n);
  if (base && ws) {
    char* b = static_cast<char*>(base);
    ws->sigA = reinterpret_cast<int*>(b + o_sigA);
    ws->sigB = reinterpret_cast<int*>(b + o_sigB);
    ws->badA = reinterpret_cast<int*>(b + o_badA);
    ws->badB = reinterpret_cast<int*>(b + o_badB);
    ws->muA = reinterpret_cast<unsigned long long*>(b + o_muA);
    ws->muB = reinterpret_cast<unsigned long long*>(b + o_muB);
    ws->stats = reinterpret_cast<float*>(b + o_stats);
    ws->DA = reinterpret_cast<uint16_t*>(b + o_DA);
    ws->DB = reinterpret_cast<uint16_t*>(b + o_DB);
    ws->U = reinterpret_cast<uint8_t*>(b + o_U);
    ws->kp = kp;
  }
  return off;
}

typedef unsigned __int128 hu128;

// product of the first n moduli
hu128 moduli_product(int n) {
  hu128 M = 1;
  for (int l = 0; l < n; ++l) M *= (hu128)kModuli[l];
  return M;
}

// fewest moduli whose product exceeds 2 k 2^(2t) >= 2 max |A'B'|; 0 when none is enough
int moduli_for(int t, int64_t k) {
  if (t < 1 || k < 1) return 0;
  // k > 2^(kb-1): from 2t + kb >= 126 on, 2 k 2^(2t) > 2^126 exceeds every product;
  // below it, 2 k 2^(2t) < 2^127 is computed exactly
  int kb = 0;
  while (((int64_t)1 << kb) < k) ++kb;
  if (2 * t + kb >= 126) return 0;
  const hu128 need = ((hu128)2 * (hu128)k) << (2 * t);
  for (int n = 1; n <= kMaxModuli; ++n)
    if (moduli_product(n) > need) return n;
  return 0;
}

int64_t inverse_mod(int64_t a, int64_t p) {  // a^-1 mod p, gcd(a, p) = 1
  int64_t t = 0, nt = 1, r = p, nr = ((a % p) + p) % p;
  while (nr) {
    const int64_t q = r / nr;
    int64_t x = t - q * nt; t = nt; nt = x;
    x = r - q * nr; r = nr; nr = x;
  }
  return t < 0 ? t + p : t;
}

// Estimated componentwise relative error of t integer bits, from the magnitude statistics
// (as the slice count of the split emulation): 2^(-t-1) (2k + k 2^(-t-1)) / (mu nu / (8k)).
double mod_relative_bound(int t, double mu_min, double nu_min, int64_t k) {
  const double kd = (double)k;
  return ldexp(1.0, -t - 1) * (2.0 * kd + kd * ldexp(1.0, -t - 1)) / (mu_min * nu_min / kd / 8.0);
}

int choose_bits(double tol, double mu_min, double nu_min, int64_t k, double* bound) {
  for (int t = 1; t <= 62; ++t) {
    const double b = mod_relative_bound(t, mu_min, nu_min, k);
    if (b <= tol) {
      if (bound) *bound = b;
      return t;
    }
  }
  return 63;
}

// Relative throughput per SM of the two-SM form over the one-SM form when both fill the GPU
constexpr double kModPairGain = 1.2;

int launch_mod_gemm(int64_t m, int64_t n, int64_t k, int nmod, const int* pc, const ModWorkspace& ws, int sms,
                    cudaStream_t stream) {
  // GBD_EMU_KERNEL=pair|single overrides the choice (tests and tuning).  Otherwise the expected
  // time in units of one 128 x 128 tile on one SM: whole waves of tiles over the SMs (or SM
  // pairs), a 256 x 256 tile being four units on two SMs at kModPairGain.
  const char* force = getenv("GBD_EMU_KERNEL");
  const int64_t tiles1 = ((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN);
  const int64_t tiles2 = ((m + k2BM - 1) / k2BM) * ((n + k2BN - 1) / k2BN);
  const int64_t pairs_avail = sms / 2 > 0 ? sms / 2 : 1;
  const double t_one = (double)((tiles1 + sms - 1) / sms);
  const double t_pair = (double)((tiles2 + pairs_avail - 1) / pairs_avail) * 2.0 / kModPairGain;
  const bool pair = force ? force[0] == 'p' : t_pair < t_one;
  const int bm = pair ? 128 : kBM;  // rows of A (and of op(B)^T) one CTA stages
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, (uint64_t)nmod};
  const uint64_t pA[2] = {(uint64_t)ws.kp * 2, (uint64_t)m * ws.kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, (uint32_t)bm, 1u};
  int rc = encode_tmap(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, (uint64_t)nmod};
  const uint64_t pB[2] = {(uint64_t)ws.kp * 2, (uint64_t)n * ws.kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, (uint32_t)(pair ? 128 : kBN), 1u};
  rc = encode_tmap(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  ModArgs a;
  memset(&a, 0, sizeof(a));
  a.m = m; a.n = n;
  a.nkb = (int)((k + kBK - 1) / kBK);
  a.nmod = nmod;
  const int tbm = pair ? k2BM : kBM, tbn = pair ? k2BN : kBN;
  a.tiles_m = (int)((m + tbm - 1) / tbm);
  const int64_t tiles = (int64_t)a.tiles_m * ((n + tbn - 1) / tbn);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  for (int l = 0; l < nmod; ++l) {
    a.p[l] = kModuli[l];
    a.c[l] = pc[l];
  }
  a.U = ws.U;
  a.err = device_error_word();
  cudaError_t e;
  if (pair) {
    const int pairs = (int)(tiles < pairs_avail ? tiles : pairs_avail);
    a.group_m = group_rows(pairs, k2BM, k2BN, a.tiles_m);
    e = cudaFuncSetAttribute(k_mod_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm pair)");
    k_mod_gemm_pair<<<(unsigned)(2 * pairs), k2Threads, Smem2::kAlloc, stream>>>(a, tmA, tmB);
  } else {
    const int grid = (int)(tiles < sms ? tiles : sms);
    a.group_m = group_rows(grid, kBM, kBN, a.tiles_m);
    e = cudaFuncSetAttribute(k_mod_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm)");
    k_mod_gemm<<<grid, kThreads, Smem::kAlloc, stream>>>(a, tmA, tmB);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "modular gemm launch");
}

}  // namespace
}  // namespace emu
}  // namespace gbd

extern "C" {

size_t gbd_dgemm_emu_mod_workspace_size(int64_t m, int64_t n, int64_t k, int bits) {
  if (m < 0 || n < 0 || k < 0) return 0;
  int nmod = gbd::emu::kMaxModuli;
  if (bits > 0) {
    const int nm = gbd::emu::moduli_for(bits, k > 0 ? k : 1);
    if (nm > 0) nmod = nm;
  }
  return gbd::emu::mod_layout(m, n, k, nmod, nullptr, nullptr);
}

int gbd_dgemm_emu_mod_moduli(int bits, int64_t k, int* moduli) {
  const int n = gbd::emu::moduli_for(bits, k);
  if (moduli)
    for (int l = 0; l < n; ++l) moduli[l] = gbd::emu::kModuli[l];
  return n;
}

int gbd_dgemm_emu_mod(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int bits,
                      double tol, void* workspace, size_t workspace_bytes, gbd_emu_info* info, void* stream) {
  using namespace gbd;
  using namespace gbd::emu;
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (info) {
    const int rp = info->record_phases;
    memset(info, 0, sizeof(*info));
    info->record_phases = rp;
  }
  if (bits < 0 || bits > 62) return set_error(GBD_ERR_ARG, "dgemm_emu_mod: bits must be 0 (automatic) or 1..62");
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (alpha == 0.0 || k == 0) return scale_c(m, n, beta, C, ldc, s);
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim)
    return set_error(GBD_ERR_LIMIT, "dgemm_emu_mod: m, n and k below 2^31 are supported");
  int sms = 0;
  if ((rc = current_device(nullptr, &sms))) return rc;
  int nmod_ws = kMaxModuli;
  if (bits > 0) {
    nmod_ws = moduli_for(bits, k);
    if (nmod_ws == 0)
      return set_error(GBD_ERR_LIMIT, "dgemm_emu_mod: %d bits need more than %d moduli at k = %lld", bits,
                       kMaxModuli, (long long)k);
  }
  const size_t need = mod_layout(m, n, k, nmod_ws, nullptr, nullptr);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return set_error(GBD_ERR_WORKSPACE, "dgemm_emu_mod: workspace must be 256-byte aligned and hold %zu bytes",
                     need);
  ModWorkspace ws;
  mod_layout(m, n, k, nmod_ws, workspace, &ws);
  const int ta = (transa == 'N' || transa == 'n') ? 0 : 1, tb = (transb == 'N' || transb == 'n') ? 0 : 1;

  // exponents (and, in automatic mode, the magnitude statistics) of both sides
  PrepPair pp;
  memset(&pp, 0, sizeof(pp));
  PrepJob& ja = pp.j[0];
  PrepJob& jb = pp.j[1];
  ja.X = A; ja.ld = lda; ja.R = m; ja.K = k; ja.rows_contig = ta == 0;
  ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = bits == 0 ? ws.muA : nullptr; ja.D = ws.DA; ja.kp = ws.kp;
  jb.X = B; jb.ld = ldb; jb.R = n; jb.K = k; jb.rows_contig = tb != 0;
  jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = bits == 0 ? ws.muB : nullptr; jb.D = ws.DB; jb.kp = ws.kp;
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);
  if ((rc = launch_exponents_pair(pp, exp_blocks, nullptr, 0, s))) return rc;
  int t = bits;
  double bound = 0.0, mu_min = 0.0, nu_min = 0.0;
  cudaError_t e;
  if (bits == 0) {
    if ((rc = launch_magnitudes_pair(pp, exp_blocks, s))) return rc;
    if ((rc = launch_min_stats(ws.muA, m, ws.muB, n, ws.badA, ws.badB, ws.stats, s))) return rc;
    float st[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(st, ws.stats, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu_mod: reading statistics");
    mu_min = st[0] < 1e38f ? st[0] : 0.0;
    nu_min = st[1] < 1e38f ? st[1] : 0.0;
    const double target = tol > 0.0 ? tol : 2.0 * (double)k * 1.1102230246251565e-16;
    t = (mu_min > 0.0 && nu_min > 0.0) ? choose_bits(target, mu_min, nu_min, k, &bound) : 1;
  }
  const int nmod = moduli_for(t, k);
  if (nmod == 0)
    return set_error(GBD_ERR_LIMIT,
                     "dgemm_emu_mod: the accuracy target needs %d integer bits, beyond %d moduli at k = %lld "
                     "(gbd_dgemm_emu covers it)",
                     t, kMaxModuli, (long long)k);

  // residues of both sides
  ModSplit ms;
  memset(&ms, 0, sizeof(ms));
  ms.n = nmod;
  ms.t = t;
  for (int l = 0; l < nmod; ++l) {
    const int pm = kModuli[l];
    ms.p[l] = pm;
    ms.inv[l] = 1.0f / (float)pm;
    uint32_t w = 1, lo = 0, hi = 0;  // 256^d mod p
    for (int d = 0; d < 8; ++d) {
      if (d < 4) lo |= (w % (uint32_t)pm) << (8 * d);
      else hi |= (w % (uint32_t)pm) << (8 * (d - 4));
      w = (w * 256u) % (uint32_t)pm;
    }
    ms.wlo[l] = lo;
    ms.whi[l] = hi;
  }
  if ((rc = launch_residue_pair(pp, ms, split_blocks, s))) return rc;

  // products modulo each modulus, then the reconstruction
  const hu128 M = moduli_product(nmod);
  int pc[kMaxModuli];
  CrtArgs ca;
  memset(&ca, 0, sizeof(ca));
  for (int l = 0; l < nmod; ++l) {
    const hu128 Mp = M / (hu128)kModuli[l];
    pc[l] = (int)inverse_mod((int64_t)(Mp % (hu128)kModuli[l]), kModuli[l]);
    ca.mp_lo[l] = (uint64_t)Mp;
    ca.mp_hi[l] = (uint64_t)(Mp >> 64);
    ca.inv[l] = 1.0f / (float)kModuli[l];
  }
  if ((rc = launch_mod_gemm(m, n, k, nmod, pc, ws, sms, s))) return rc;
  ca.m = m; ca.n = n; ca.ldc = ldc;
  ca.nmod = nmod; ca.t = t;
  ca.M_lo = (uint64_t)M; ca.M_hi = (uint64_t)(M >> 64);
  const hu128 half = M / 2;
  ca.half_lo = (uint64_t)half; ca.half_hi = (uint64_t)(half >> 64);
  ca.alpha = alpha; ca.beta = beta; ca.C = C;
  ca.sigA = ws.sigA; ca.sigB = ws.sigB; ca.badA = ws.badA; ca.badB = ws.badB;
  ca.U = ws.U;
  const unsigned gy = (unsigned)(n < 65535 ? n : 65535);
  k_crt<<<dim3((unsigned)((m + 255) / 256), gy), 256, 0, s>>>(ca);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "reconstruction launch");
  if (info) {
    info->slices = nmod;
    info->digit_bits = t;
    info->products = nmod;
    info->mu_min = mu_min;
    info->nu_min = nu_min;
    info->bound_est = bound;
  }
  return GBD_OK;
}

}  // extern "C"
