// emu_cert.cu -- the certified precision choice of both emulations of DGEMM.
//
// The a-priori truncation bound of element (i, j) is, in units of 2^(sigma_i + tau_j),
//   split (s slices of 7 bits):  2^-7s (mu_i + nu_j + (s - 1)(1 + 2^-7) k)
//   modular (t integer bits):    2^(-t-1) (mu_i + nu_j + k 2^(-t-1))
// and it has to stay within (tol - r u) G^_ij, G^_ij = sum_p |a^_ip||b^_pj| the scaled
// (|op(A)||op(B)|)_ij and r u the allowance for the final roundings.  A choice that meets this
// for every element needs G^_ij, an m x n x k quantity: this file bounds it from below with
// one product on the tensor cores of the magnitude planes (emu_split.cu, MagWriter), in FP8 E5M2
// (kind::f8f6f4, the emulations' default) or in BF16 (kind::f16, tighter), and
// reduces over the elements
//     rho = rhoA + rhoB >= max (mu_i + nu_j) / G_ij,   gamma = max 1 / G_ij     (G_ij <= G^_ij)
// with rhoA = max_i mu_i / min_j G_ij and rhoB = max_j nu_j / min_i G_ij, so that the choice needs
// only 2^(-t-1) (rho + k 2^(-t-1) gamma) <= tol - r u (and the split form).  Elements whose plane product is exactly zero have no error term (each term of
// |A||B| has a zero factor, which both emulations represent exactly) and are skipped.
//
// The lower bound: the planes hold v = RZ(max(|a^|, w) 2^S) with w = 2^(-63-S) (BF16) or 2^(-14-S)
// (E5M2, S = 15), so
//   sum_p v_a v_b 2^-2S <= G^ + k (2 w + w^2)
// and the FP32 accumulation of the non-negative products (exact in FP32) overshoots the
// exact sum by at most (number of accumulation steps) x 17 x 2^-24 of it, an MMA step adding 16
// products; a chunk of c terms (16384 in the one-SM form, the whole k <= 65536 in the pair form)
// stays far below delta = c 2^-19, so
//   G^_ij >= L_ij (1 - delta) 2^-2S - k (2w + w^2)
// with L_ij the FP32 result; chunk results are added rounding downward and every step of the
// epilogue rounds toward the safe side (__fmul_rd, __fsub_rd, __fdiv_ru).  S is the largest
// scale that keeps k 2^(2S) below 2^124 (no overflow of the FP32 accumulator).
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "emu.cuh"
#include "tcgen05.cuh"

namespace gbd {
namespace emu {
namespace {

using namespace tc;

// PAIR = false: 128 x 128 tiles on one SM (cta_group::1).  PAIR = true: 256 x 256 tiles on a
// CTA pair (cta_group::2): each CTA stages 128 rows of both planes per k-block and holds 128 rows
// x 256 columns of the tile in its TMEM, so every staged byte feeds twice the products.
template <bool PAIR, bool FP8 = false>
struct CertCfg {
  static constexpr int BM = PAIR ? 256 : 128;  // tile rows (both CTAs of a pair)
  static constexpr int BN = PAIR ? 256 : 128;  // tile columns
  static constexpr int kStages = 6;
  static constexpr int kEpiWarps = 16;                // 4 x 4 warps over 128 TMEM lanes x BN columns
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static constexpr int kTmemCols = 2 * BN;           // two accumulators
  static constexpr int kCols = BN / (kEpiWarps / 4);  // columns per epilogue thread
  static constexpr int kKB = FP8 ? 128 : kBK;         // k elements per stage: 128 bytes of a row
  static constexpr int kABytes = 128 * 128;           // per CTA and stage: 128 rows of 128 bytes
  static constexpr int kBBytes = 128 * 128;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + kStages * kABytes;
  static constexpr int kOffBar = kOffB + kStages * kBBytes;
  static constexpr int kNumBars = 2 * kStages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kBytes = kOffTmemSlot + 16;
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};
// k-blocks of 64 per FP32 accumulation chunk: the one-SM form drains 16384-deep chunks into
// registers; the pair form accumulates the whole inner dimension in TMEM (k <= kCertPairMaxK)
constexpr int kCertChunkBlocks = 256;
constexpr int64_t kCertPairMaxK = 65536;


// an upper bound of a magnitude sum held in 32.32 fixed point
__device__ __forceinline__ float mu_upper(unsigned long long q, float scale) {
  return __fmaf_ru((float)((double)q * 0x1p-32), scale, 0x1p-20f);
}

// TABLE (one-SM form): the tiles of several problems, each with its own arguments and maps in a
// table entry (entries in tile order); the maxima go to each problem's words tile by tile.
template <bool PAIR, bool FP8, bool TABLE = false>
__global__ void __launch_bounds__(CertCfg<PAIR>::kThreads, 1)
    k_cert_gemm(const __grid_constant__ CertArgs p, const __grid_constant__ CUtensorMap tmA,
                const __grid_constant__ CUtensorMap tmB, const CertTableEntry* __restrict__ table = nullptr,
                int count = 0, int total_tiles = 0, const unsigned int* __restrict__ run_if = nullptr) {
  static_assert(!(PAIR && TABLE), "grouped certification runs on one SM per tile");
  using L = CertCfg<PAIR, FP8>;
  if (!TABLE && p.gate && p.gate->feasible) return;  // the retry of a certification that succeeded
  if (TABLE && run_if && *run_if == 0u) return;     // a grouped retry that no problem needs
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + L::kStages;
  uint64_t* acc_full = bars + 2 * L::kStages;
  uint64_t* acc_empty = bars + 2 * L::kStages + 2;
  uint64_t* done = bars + 2 * L::kStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmemSlot);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int unit = PAIR ? (int)(blockIdx.x / 2) : (int)blockIdx.x;   // tile sequence of this CTA (pair)
  const int units = PAIR ? (int)(gridDim.x / 2) : (int)gridDim.x;

  const int num_tiles = TABLE ? total_tiles : p.num_tiles;
  // the arguments and the tile coordinates of tile `tile` (grouped: of its problem)
  auto tile_args = [&](int tile, int& cur, int& tm, int& tn) -> const CertArgs* {
    if constexpr (!TABLE) {
      tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
      return &p;  // a __grid_constant__ parameter: its address is that of the parameter itself
    } else {
      while (cur + 1 < count && table[cur + 1].tile_begin <= tile) ++cur;
      const CertArgs* q = &table[cur].a;
      tile_coords(tile - (int)table[cur].tile_begin, q->tiles_m, q->group_m, q->num_tiles, tm, tn);
      return q;
    }
  };
  // grouped retry: the tiles of a problem whose plan is already feasible are skipped by every role
  auto skipped = [&](const CertArgs& q) { return TABLE && q.gate && q.gate->feasible; };

  if (warp == 0 && lane == 0) {
    if (!TABLE) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
    }
    for (int i = 0; i < L::kStages; ++i) {
      mbar_init(&full[i], 1);   // PAIR: the leader's producer arrives with both CTAs' bytes
      mbar_init(&empty[i], 1);  // one commit per phase (multicast to both CTAs of a pair)
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], (PAIR ? 2 : 1) * 32 * L::kEpiWarps);  // every epilogue thread (of both CTAs)
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "n"(L::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "n"(L::kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync_all();  // the peer's barriers are initialised and its TMEM is allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      int cur = 0;
      for (int tile = unit; tile < num_tiles; tile += units) {
        int tm, tn;
        const CertArgs& q = *tile_args(tile, cur, tm, tn);
        if (skipped(q)) continue;
        const CUtensorMap* ma = TABLE ? &table[cur].tmA : &tmA;
        const CUtensorMap* mb = TABLE ? &table[cur].tmB : &tmB;
        if (TABLE) {  // maps written into global memory before the launch: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ma) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mb) : "memory");
        }
        const int m0 = tm * L::BM + (int)rank * 128, n0 = tn * L::BN + (int)rank * 128;
        for (int kb = 0; kb < q.nkb; ++kb) {
          if (PAIR) {
            mbar_wait_cluster(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
            if (leader) mbar_arrive_expect_tx(&full[stage], (uint32_t)(2 * (L::kABytes + L::kBBytes)));
            const uint32_t fbar = map_to_rank(smem_u32(&full[stage]), 0);
            tma_load_3d_pair(smem + L::kOffA + stage * L::kABytes, ma, fbar, kb * L::kKB, m0, 0);
            tma_load_3d_pair(smem + L::kOffB + stage * L::kBBytes, mb, fbar, kb * L::kKB, n0, 0);
          } else {
            mbar_wait(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
            mbar_arrive_expect_tx(&full[stage], (uint32_t)(L::kABytes + L::kBBytes));
            tma_load_3d(smem + L::kOffA + stage * L::kABytes, ma, &full[stage], kb * L::kKB, m0, 0);
            tma_load_3d(smem + L::kOffB + stage * L::kBBytes, mb, &full[stage], kb * L::kKB, n0, 0);
          }
          if (++stage == L::kStages) { stage = 0; phase ^= 1u; }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer (the leader of a pair) --------------------------------
    if (leader && lane == 0) {
      constexpr uint32_t idesc = FP8 ? idesc_e5m2(L::BM, L::BN) : idesc_bf16(L::BM, L::BN);
      uint32_t stage = 0, phase = 0, chunk = 0;
      const uint32_t a_base = smem_u32(smem + L::kOffA), b_base = smem_u32(smem + L::kOffB);
      int cur = 0;
      for (int tile = unit; tile < num_tiles; tile += units) {
        int tm, tn;
        const CertArgs& q = *tile_args(tile, cur, tm, tn);
        if (skipped(q)) continue;
        for (int i0 = 0; i0 < q.nkb; i0 += q.chunk_blocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          if (PAIR) mbar_wait_cluster(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
          else mbar_wait(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
          tc_fence_after();
          const uint32_t dtm = tmem_base + buf * L::BN;
          const int i1 = min(q.nkb, i0 + q.chunk_blocks);
          for (int it = i0; it < i1; ++it) {
            if (PAIR) mbar_wait_cluster(&full[stage], phase, p.err, kErrWaitTma);
            else mbar_wait(&full[stage], phase, p.err, kErrWaitTma);
            tc_fence_after();
            const uint64_t da = smem_desc_sw128(a_base + stage * L::kABytes);
            const uint64_t db = smem_desc_sw128(b_base + stage * L::kBBytes);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of every row per instruction
              const uint32_t acc = (it > i0 || kk > 0) ? 1u : 0u;
              if (FP8) {
                if (PAIR) umma_fp8_pair(dtm, da + 2 * kk, db + 2 * kk, idesc, acc);
                else umma_fp8(dtm, da + 2 * kk, db + 2 * kk, idesc, acc);
              } else {
                if (PAIR) umma_bf16_pair(dtm, da + 2 * kk, db + 2 * kk, idesc, acc);
                else umma_bf16(dtm, da + 2 * kk, db + 2 * kk, idesc, acc);
              }
            }
            if (PAIR) umma_commit_pair(&empty[stage]);  // frees this stage in both CTAs
            else umma_commit(&empty[stage]);
            if (++stage == L::kStages) { stage = 0; phase ^= 1u; }
          }
          if (PAIR) umma_commit_pair(&acc_full[buf]);  // the chunk is complete in both CTAs' TMEM
          else umma_commit(&acc_full[buf]);
        }
      }
      if (chunk > 0) {  // a CTA without a tile issued nothing and has nothing to wait for
        if (PAIR) {
          umma_commit_pair(done);
          mbar_wait_cluster(done, 0, p.err, kErrWaitMma);
        } else {
          umma_commit(done);
          mbar_wait(done, 0, p.err, kErrWaitMma);
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue ------------------------------
    constexpr int COLS = L::kCols;
    const int quad = warp & 3;            // TMEM lanes 32 quad .. 32 quad + 31
    const int part = (warp - 2) >> 2;     // columns COLS part ..
    const int row = quad * 32 + lane;
    const int col0 = part * COLS;
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    uint32_t empty_remote[2] = {0u, 0u};
    if (PAIR) {
      empty_remote[0] = map_to_rank(smem_u32(&acc_empty[0]), 0);
      empty_remote[1] = map_to_rank(smem_u32(&acc_empty[1]), 0);
    }
    // Per element, with G_ij its lower bound and 1/theta_i, 1/phi_j upper bounds of the reciprocal
    // of the smallest non-zero scaled entry of row i and column j:
    //   T1 = min(nu_j / G_ij, 1/theta_i),  T2 = min(mu_i / G_ij, 1/phi_j),
    //   T3 = min(1 / G_ij, 1 / (k theta_i phi_j)),
    // every term rounded up (without a usable G_ij only the spread terms remain).  The words hold
    // rhoA = max T2, rhoB = max T1 and gamma = max T3, so that for every element
    //   (its error bound) / G_ij <= 2^(-t-1) (rhoA + rhoB + k 2^(-t-1) gamma)     (modular).
    float rmaxA = 0.0f, rmaxB = 0.0f, gmax = 0.0f;
    // 1/theta as a power of two from the row's exponent sigma and its smallest one (inf above 2^127)
    auto inv_spread = [](int sig, int em) -> float {
      if (em == kEminNone) return 0.0f;  // no non-zero entry: no term
      const int x = (sig == kExpEmpty ? 0 : sig) + 1 - em;
      return x > 127 ? INFINITY : __int_as_float((127 + x) << 23);
    };
    auto certify = [&](const CertArgs& p, int64_t i, int64_t jc0, const float (&acc)[32]) {
      const bool row_ok = i < p.m && p.badA[i] == 0;
      const int si = (i < p.m) ? p.sigA[i] : 0;
      const float mui = row_ok ? mu_upper(p.muA[i], p.mu_scale) : 0.0f;
      const float cth = row_ok ? inv_spread(si, p.eminA[i]) : 0.0f;
      // this lane's column of the 32: its magnitude sum and spread, handed round by shuffles
      const int64_t jl = jc0 + lane;
      const bool col_ok = jl < p.n && p.badB[jl] == 0;
      const float nu_l = col_ok ? mu_upper(p.muB[jl], p.mu_scale) : 0.0f;
      const float cph_l = col_ok ? inv_spread(p.sigB[jl], p.eminB[jl]) : 0.0f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {  // fully unrolled: acc stays in registers
        const int64_t j = jc0 + c;
        const float nuj = __shfl_sync(0xffffffffu, nu_l, c);
        const float cph = __shfl_sync(0xffffffffu, cph_l, c);
        const bool ok = row_ok && j < p.n && p.badB[j] == 0;
        float G = 0.0f;
        if (ok && acc[c] > 0.0f) {
          G = __fsub_rd(__fmul_rd(acc[c], p.f), p.slack);
          float t1 = cth, t2 = cph, t3 = __fmul_ru(__fmul_ru(cth, cph), p.kinv);
          if (G > 0.0f) {
            const float inv = __frcp_ru(G);
            t1 = fminf(t1, __fmul_ru(nuj, inv));
            t2 = fminf(t2, __fmul_ru(mui, inv));
            t3 = fminf(t3, inv);
          }
          rmaxB = fmaxf(rmaxB, t1);
          rmaxA = fmaxf(rmaxA, t2);
          gmax = fmaxf(gmax, t3);
        }
        if (p.L && i < p.m && j < p.n) {
          double out = 0.0;
          if (!ok) out = __longlong_as_double(0x7FF8000000000000ll);  // a NaN row or column: no bound
          else if (G > 0.0f) out = ldexp((double)G, (si == kExpEmpty ? 0 : si) +
                                                        (p.sigB[j] == kExpEmpty ? 0 : p.sigB[j]));
          p.L[i + j * p.ldl] = out;
        }
      }
    };
    // the maxima into a problem's words (grouped: after every tile, the next may be another's)
    auto flush = [&](unsigned int* words) {  // non-negative floats (and +inf) order as their bits
      const unsigned ra = __reduce_max_sync(0xffffffffu, __float_as_uint(rmaxA));
      const unsigned rb = __reduce_max_sync(0xffffffffu, __float_as_uint(rmaxB));
      const unsigned gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));
      if (lane == 0) {
        if (ra) atomicMax(words + kCertRhoA, ra);
        if (rb) atomicMax(words + kCertRhoB, rb);
        if (gb) atomicMax(words + kCertGamma, gb);
      }
      rmaxA = rmaxB = gmax = 0.0f;
    };
    uint32_t chunk = 0;
    int cur = 0;
    for (int tile = unit; tile < num_tiles; tile += units) {
      int tm, tn;
      const CertArgs& p = *tile_args(tile, cur, tm, tn);
      if (skipped(p)) continue;
      const int64_t i = (int64_t)tm * L::BM + (int)rank * 128 + row;
      const int64_t jc0 = (int64_t)tn * L::BN + col0;
      if (p.chunk_blocks >= p.nkb) {
        // one chunk: the columns straight from TMEM, 32 at a time
        const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
        ++chunk;
        mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
        tc_fence_after();
#pragma unroll 1
        for (int h = 0; h < COLS; h += 32) {
          float acc[32];
          const uint32_t taddr = trow + buf * L::BN + col0 + h;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint32_t v[16];
            tmem_ld_16(taddr + q * 16, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[q * 16 + jj] = __uint_as_float(v[jj]);
          }
          certify(p, i, jc0 + h, acc);
        }
        tc_fence_before();
        if (PAIR) mbar_arrive_remote(empty_remote[buf]);
        else mbar_arrive(&acc_empty[buf]);
      } else if (!PAIR) {
        // several chunks (one-SM form, COLS = 32): their results added in registers, rounding down
        static_assert(PAIR || COLS == 32, "the one-SM epilogue holds 32 columns per thread");
        float acc[32];
        bool first = true;
        for (int i0 = 0; i0 < p.nkb; i0 += p.chunk_blocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
          tc_fence_after();
          const uint32_t taddr = trow + buf * L::BN + col0;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
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
        certify(p, i, jc0, acc);
      }
      if (TABLE) flush(p.words);
    }
    if (!TABLE) flush(p.words);
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync_all();  // neither CTA leaves while the pair still uses its shared memory
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(L::kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(L::kTmemCols)
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

int cert_prec_default() {
  const char* e = getenv("GBD_CERT_DTYPE");  // bf16 | fp8 (tests and tuning)
  return (e && (e[0] == 'b' || e[0] == 'B')) ? kCertBF16 : kCertFP8;
}

int plane_scale(int64_t k, int prec) {
  if (prec == kCertFP8) return 15;  // |v| < 2^15 within E5M2's range; k 2^30 < 2^124 for every k < 2^31
  int kb = 0;
  while (((int64_t)1 << kb) < k) ++kb;
  return (124 - kb) / 2;
}

int64_t plane_pitch(int64_t k, int prec) {
  return prec == kCertFP8 ? (k + 15) / 16 * 16 : (k + 7) / 8 * 8;
}

namespace {

template <bool PAIR, bool FP8>
int launch_cert_kernel(const CertArgs& a, const CUtensorMap& tmA, const CUtensorMap& tmB, int grid,
                       cudaStream_t stream) {
  using L = CertCfg<PAIR, FP8>;
  auto kern = k_cert_gemm<PAIR, FP8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(certification gemm)");
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(L::kThreads, 1, 1);
  cfg.dynamicSmemBytes = L::kAlloc;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PAIR ? 2 : 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = PAIR ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, kern, a, tmA, tmB, static_cast<const CertTableEntry*>(nullptr), 0, 0,
                         static_cast<const unsigned int*>(nullptr));
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "certification gemm launch");
}

}  // namespace

int launch_cert(int64_t m, int64_t n, int64_t k, int prec, const void* PA, const void* PB,
                const unsigned long long* muA, const unsigned long long* muB, const int* badA, const int* badB,
                const int* sigA, const int* sigB, const int* eminA, const int* eminB, unsigned int* words,
                double* Lout, int64_t ldl, int sms, cudaStream_t stream, const ModPlan* gate) {
  if (m <= 0 || n <= 0 || k <= 0) return GBD_OK;
  const bool fp8 = prec == kCertFP8;
  const int S = plane_scale(k, prec);
  const int64_t pitch = plane_pitch(k, prec);
  const int kkb = fp8 ? 128 : kBK;  // k elements per k-block
  CertArgs a;
  memset(&a, 0, sizeof(a));
  a.m = m;
  a.n = n;
  a.nkb = (int)((k + kkb - 1) / kkb);
  // the floor of the planes, w = 2^(-63-S) (BF16) or 2^(-14-S) (E5M2's smallest normal)
  const double w = std::ldexp(1.0, (fp8 ? -14 : -63) - S);
  a.slack = float_up((double)k * (2.0 * w + w * w) * (1.0 + std::ldexp(1.0, -40)));
  // the magnitude sums' FP32 roundings: within 2^-10 relatively for every 1024-deep block of terms
  // and 2^-22 for every one of at most ceil(k/64) partial sums merged (tiles of the one-pass
  // statistics; the magnitude pass's 1024-deep blocks are fewer)
  const double nkt = (double)((k + 63) / 64);
  a.mu_scale = float_up(1.0 + std::ldexp(1.0, -10) + nkt * std::ldexp(1.0, -22));
  a.muA = muA;
  a.muB = muB;
  a.badA = badA;
  a.badB = badB;
  a.sigA = sigA;
  a.sigB = sigB;
  a.eminA = eminA;
  a.eminB = eminB;
  a.kinv = float_up(1.0 / (double)k);
  a.gate = gate;
  a.words = words;
  a.L = Lout;
  a.ldl = ldl;
  a.err = device_error_word();
  // one-SM 128 x 128 tiles or CTA-pair 256 x 256 tiles, by whole waves of tiles (a pair tile is four
  // one-SM tiles on two SMs at about 1.2 times the rate per SM)
  const int64_t tiles1 = ((m + 127) / 128) * ((n + 127) / 128);
  const int64_t tiles2 = ((m + 255) / 256) * ((n + 255) / 256);
  const int64_t pairs_avail = sms / 2 > 0 ? sms / 2 : 1;
  const double t_one = (double)((tiles1 + sms - 1) / sms);
  const double t_pair = (double)((tiles2 + pairs_avail - 1) / pairs_avail) * 2.0 / 1.2;
  const char* force = getenv("GBD_CERT_KERNEL");  // pair | single (tests and tuning)
  const bool pair = k <= kCertPairMaxK && sms >= 2 && (force ? force[0] == 'p' : t_pair < t_one);
  // the accumulation chunk and the overshoot bound of its FP32 accumulation
  a.chunk_blocks = pair ? a.nkb : kCertChunkBlocks * kBK / kkb;
  const int64_t chunk_k = (int64_t)a.chunk_blocks * kkb < k ? (int64_t)a.chunk_blocks * kkb : k;
  const double delta = (double)chunk_k * std::ldexp(1.0, -19);
  a.f = float_down(std::ldexp(1.0 - delta, -2 * S));
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint64_t eb = fp8 ? 1 : 2;
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, 1u};
  const uint64_t pA[2] = {(uint64_t)pitch * eb, (uint64_t)m * pitch * eb};
  const uint32_t bA[3] = {(uint32_t)kkb, 128u, 1u};
  int rc = encode_tmap(&tmA, dt, 3, PA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, 1u};
  const uint64_t pB[2] = {(uint64_t)pitch * eb, (uint64_t)n * pitch * eb};
  const uint32_t bB[3] = {(uint32_t)kkb, 128u, 1u};
  rc = encode_tmap(&tmB, dt, 3, PB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const int bm = pair ? 256 : 128, bn = pair ? 256 : 128;
  a.tiles_m = (int)((m + bm - 1) / bm);
  const int64_t tiles = (int64_t)a.tiles_m * ((n + bn - 1) / bn);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  if (pair) {
    const int64_t pairs = tiles < pairs_avail ? tiles : pairs_avail;
    a.group_m = group_rows((int)pairs, bm, bn, a.tiles_m);
    return fp8 ? launch_cert_kernel<true, true>(a, tmA, tmB, (int)(2 * pairs), stream)
               : launch_cert_kernel<true, false>(a, tmA, tmB, (int)(2 * pairs), stream);
  }
  const int grid = (int)(tiles < sms ? tiles : sms);
  a.group_m = group_rows(grid, bm, bn, a.tiles_m);
  return fp8 ? launch_cert_kernel<false, true>(a, tmA, tmB, grid, stream)
             : launch_cert_kernel<false, false>(a, tmA, tmB, grid, stream);
}

int make_cert_entry(int64_t m, int64_t n, int64_t k, int prec, const void* PA, const void* PB,
                    const unsigned long long* muA, const unsigned long long* muB, const int* badA, const int* badB,
                    const int* sigA, const int* sigB, const int* eminA, const int* eminB, unsigned int* words,
                    const ModPlan* gate, CertTableEntry* e) {
  memset(e, 0, sizeof(*e));
  CertArgs& a = e->a;
  const bool fp8 = prec == kCertFP8;
  const int S = plane_scale(k, prec);
  const int64_t pitch = plane_pitch(k, prec);
  const int kkb = fp8 ? 128 : kBK;  // k elements per k-block
  const uint64_t eb = fp8 ? 1 : 2;
  a.m = m;
  a.n = n;
  a.nkb = (int)((k + kkb - 1) / kkb);
  a.chunk_blocks = kCertChunkBlocks * kBK / kkb;  // 16384 deep, as the one-SM form of single calls
  const int64_t chunk_k = (int64_t)a.chunk_blocks * kkb < k ? (int64_t)a.chunk_blocks * kkb : k;
  a.f = float_down(std::ldexp(1.0 - (double)chunk_k * std::ldexp(1.0, -19), -2 * S));
  const double w = std::ldexp(1.0, (fp8 ? -14 : -63) - S);
  a.slack = float_up((double)k * (2.0 * w + w * w) * (1.0 + std::ldexp(1.0, -40)));
  a.mu_scale = float_up(1.0 + std::ldexp(1.0, -10) + (double)((k + 63) / 64) * std::ldexp(1.0, -22));
  a.muA = muA;
  a.muB = muB;
  a.badA = badA;
  a.badB = badB;
  a.sigA = sigA;
  a.sigB = sigB;
  a.eminA = eminA;
  a.eminB = eminB;
  a.kinv = float_up(1.0 / (double)k);
  a.gate = gate;
  a.words = words;
  a.err = device_error_word();
  a.tiles_m = (int)((m + 127) / 128);
  a.num_tiles = a.tiles_m * (int)((n + 127) / 128);
  a.group_m = a.tiles_m;  // within one problem the tiles walk down the rows
  const CUtensorMapDataType dt = fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, 1u};
  const uint64_t pA[2] = {(uint64_t)pitch * eb, (uint64_t)m * pitch * eb};
  const uint32_t box[3] = {(uint32_t)kkb, 128u, 1u};
  int rc = encode_tmap(&e->tmA, dt, 3, PA, dA, pA, box, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, 1u};
  const uint64_t pB[2] = {(uint64_t)pitch * eb, (uint64_t)n * pitch * eb};
  return encode_tmap(&e->tmB, dt, 3, PB, dB, pB, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

int launch_cert_grouped(const CertTableEntry* table_dev, int count, int total_tiles, int prec, int sms,
                        cudaStream_t stream, const unsigned int* run_if) {
  if (count <= 0 || total_tiles <= 0) return GBD_OK;
  using L = CertCfg<false, true>;  // the same shared memory and threads in both precisions
  auto kern = prec == kCertFP8 ? k_cert_gemm<false, true, true> : k_cert_gemm<false, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped certification)");
  CertArgs dummy_args;
  memset(&dummy_args, 0, sizeof(dummy_args));
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  const int grid = total_tiles < sms ? total_tiles : sms;
  kern<<<grid, L::kThreads, L::kAlloc, stream>>>(dummy_args, dummy, dummy, table_dev, count, total_tiles, run_if);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "grouped certification launch");
}

}  // namespace emu
}  // namespace gbd

extern "C" {

size_t gbd_abs_product_lower_bound_workspace_size(int64_t m, int64_t n, int64_t k) {
  if (m < 0 || n < 0 || k < 0) return 0;
  return gbd::emu::layout(m, n, k, 1, nullptr, nullptr, false);
}

int gbd_abs_product_lower_bound(char transa, char transb, int64_t m, int64_t n, int64_t k, const double* A,
                                int64_t lda, const double* B, int64_t ldb, double* L, int64_t ldl, int fp8,
                                void* workspace, size_t workspace_bytes, void* stream) {
  using namespace gbd;
  using namespace gbd::emu;
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldl);
  if (rc) return rc == 13 ? 11 : rc;  // ldl is argument 11 of this list
  if (fp8 != 0 && fp8 != 1) return 12;
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
  ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = ws.muA; ja.D = ws.DA; ja.kp = ws.kp; ja.emin = ws.eminA;
  jb.X = B; jb.ld = ldb; jb.R = n; jb.K = k; jb.rows_contig = trans_code(transb) != 0;
  jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = ws.muB; jb.D = ws.DB; jb.kp = ws.kp; jb.emin = ws.eminB;
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);
  if ((rc = launch_exponents_pair(pp, exp_blocks, nullptr, 0, s))) return rc;
  if ((rc = launch_magnitudes_pair(pp, exp_blocks, s))) return rc;
  cudaError_t e = cudaMemsetAsync(ws.cert, 0, sizeof(unsigned int) * kCertWords, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.eminA, 0x7F, sizeof(int) * (size_t)(m + n), s);
  if (e != cudaSuccess) return cuda_fail(e, "abs_product_lower_bound: clearing the certification words");
  const int prec = fp8 ? kCertFP8 : kCertBF16;
  if ((rc = launch_magplane_pair(pp, prec, ws.cert + kCertTexA, split_blocks, s))) return rc;
  return launch_cert(m, n, k, prec, ws.DA, ws.DB, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB, ws.eminA,
                     ws.eminB, ws.cert, L, ldl, sms, s);
}

}  // extern "C"
