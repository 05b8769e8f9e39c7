// emu_mod.cu -- the modular emulation of DGEMM (Ozaki, Uchino and Imamura, "Ozaki Scheme
// II: a GEMM-oriented emulation of floating-point matrix multiplication using an integer
// modular technique", 2025) on the 5th-generation tensor cores.
//
//   1. sigma_i, tau_j: the row and column exponents of the split emulation (emu_split.cu).
//   2. A' = rint(a 2^(t - sigma_i)), B' = rint(b 2^(t - tau_j)) (integers, |.| <= 2^t), and
//      their residues modulo n pairwise coprime moduli p_l <= 256, written as BF16 slices
//      (emu_split.cu, k_residue_pair).
//   3. For every modulus: the residue product on tcgen05.mma with 1024-deep exact FP32
//      chunks drained into int32, reduced modulo p_l; the epilogue parks one byte per
//      element, u_l = (residue x c_l) mod p_l with c_l = (M/p_l)^-1 mod p_l, in a per-CTA slot.
//   4. In the same epilogue, while the next tile's products run: C' = sum_l u_l (M/p_l) mod M,
//      the unique integer of (-M/2, M/2] congruent to the products; it equals A'B' because
//      M > 2 k 2^(2t) >= 2 max|A'B'|.  Then C := fma(alpha 2^(tau_j - 2t), fl(C') 2^sigma_i,
//      beta C0), fl correctly rounded.
// There is no FP64 arithmetic in the products: n GEMMs replace the s(s+1)/2 of the split
// emulation.  All waits are bounded (2 s) and set the device error word when they give up.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "emu.cuh"
#include "tcgen05.cuh"

namespace gbd {
namespace emu {
namespace {

using namespace tc;

constexpr int kReduceChunks = 63;  // 63 chunks of 1024 k (each below 2^24) plus a residue stay below 2^30
// The parked residues: for every 128 x 128 block of C (row block rb, column block cb, block
// rb * nbn + cb) and modulus l, one plane of [column / 4][row][4 columns] bytes, so that a thread
// moves four columns in one word and a warp 128 contiguous bytes
constexpr int64_t kParkBlock = 128 * 128;

// the reconstruction constants of the first n moduli (M = p_0 ... p_(n-1), W_l = M / p_l,
// c_l = W_l^-1 mod p_l): with r_l = C' mod p_l in [0, p_l), X = sum_l r_l V_l, V_l = c_l W_l < M,
// is congruent to C' modulo M, and X / M = sum_l r_l c_l / p_l
// V_l and e_l = ceil(c_l 2^16 / p_l) enter as bytes, four moduli per word, for the byte dot
// products of dp4a: wp[G][d] holds byte d of V_4G .. V_4G+3, ep[G][d] byte d of e_4G .. e_4G+3;
// sum_l r_l e_l / 2^16 exceeds X / M by less than 1/16
struct CrtSet {
  uint32_t wp[kMaxModuli / 4][16];
  uint32_t ep[kMaxModuli / 4][2];
  uint32_t M[4];  // M in 32-bit limbs, least significant first
  uint32_t H[4];  // M / 2 - 1 (M is even: p_0 = 256)
};
struct CrtConsts {
  CrtSet set[kMaxModuli];  // set[n - 1]: the constants for the first n moduli
};

// multi-word arithmetic on 32-bit limbs (least significant first) for the constants, at compile time
constexpr void limbs_mul_small(uint32_t (&x)[5], uint32_t f) {
  uint64_t carry = 0;
  for (int j = 0; j < 5; ++j) {
    const uint64_t t = (uint64_t)x[j] * f + carry;
    x[j] = (uint32_t)t;
    carry = t >> 32;
  }
}
constexpr uint32_t limbs_div_small(uint32_t (&x)[5], uint32_t d) {  // x := x / d, returns x mod d
  uint64_t rem = 0;
  for (int j = 4; j >= 0; --j) {
    const uint64_t t = (rem << 32) | x[j];
    x[j] = (uint32_t)(t / d);
    rem = t % d;
  }
  return (uint32_t)rem;
}
constexpr uint32_t inverse_small(uint32_t a, uint32_t p) {  // a^-1 mod p, gcd(a, p) = 1
  int64_t t = 0, nt = 1, r = p, nr = a % p;
  while (nr != 0) {
    const int64_t q = r / nr;
    const int64_t x = t - q * nt;
    t = nt;
    nt = x;
    const int64_t y = r - q * nr;
    r = nr;
    nr = y;
  }
  return (uint32_t)(t < 0 ? t + p : t);
}
constexpr CrtConsts make_crt_consts() {
  CrtConsts k{};
  for (int nn = 1; nn <= kMaxModuli; ++nn) {
    CrtSet& cs = k.set[nn - 1];
    uint32_t M[5] = {1u, 0u, 0u, 0u, 0u};
    for (int l = 0; l < nn; ++l) limbs_mul_small(M, (uint32_t)kModuli[l]);
    for (int l = 0; l < nn; ++l) {
      const uint32_t p = (uint32_t)kModuli[l];
      uint32_t W[5] = {M[0], M[1], M[2], M[3], M[4]};
      limbs_div_small(W, p);  // exact: p divides M
      uint32_t Wr[5] = {W[0], W[1], W[2], W[3], W[4]};
      const uint32_t c = inverse_small(limbs_div_small(Wr, p), p);
      limbs_mul_small(W, c);  // V_l = c_l W_l < M
      const uint32_t e = (uint32_t)((((uint64_t)c << 16) + p - 1) / p);  // below 2^16
      const int G = l / 4, b = 8 * (l % 4);
      for (int d = 0; d < 16; ++d) cs.wp[G][d] |= ((W[d / 4] >> (8 * (d % 4))) & 0xFFu) << b;
      for (int d = 0; d < 2; ++d) cs.ep[G][d] |= ((e >> (8 * d)) & 0xFFu) << b;
    }
    uint32_t H[5] = {M[0], M[1], M[2], M[3], M[4]};
    limbs_div_small(H, 2u);
    for (int j = 0; j < 5; ++j) {  // H := M / 2 - 1
      if (H[j] != 0u) {
        --H[j];
        break;
      }
      H[j] = 0xFFFFFFFFu;
    }
    for (int j = 0; j < 4; ++j) {
      cs.M[j] = M[j];
      cs.H[j] = H[j];
    }
  }
  return k;
}
// in constant memory: the specialisations address them as immediate operands
__constant__ CrtConsts kCrt = make_crt_consts();

struct ModArgs {
  int64_t m, n;
  int nkb;
  int tiles_m, num_tiles, group_m;
  int tri;  // 0: all of C; 1: only the tiles that meet its lower triangle (i >= j), 2: its
            // upper one (m = n), by rows of tiles
  int p[kMaxModuli];         // moduli
  uint32_t bar[kMaxModuli];  // floor(2^32 / p_l), for Barrett reduction
  float pinv[kMaxModuli];    // fl(1 / p_l) in FP32 (the reduction of a single exact FP32 chunk)
  const ModPlan* plan;       // the call's n (and whether the target was reachable)
  uint8_t* park;             // [blocks][park_mods][kParkBlock] the residues of the products
  int park_mods;             // moduli the park array holds per block
  int nbn;                   // 128-column blocks of C
  // split over moduli (one-SM form, few tiles): each tile's moduli in `groups` work units
  int groups;
  unsigned int* err;
};

// tile t of a triangle of tiles, by rows: (r, c) with c <= r, t = r (r + 1) / 2 + c
__device__ __forceinline__ void tri_tile(int t, int& r, int& c) {
  int q = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // corrected below
  while ((int64_t)(q + 1) * (q + 2) / 2 <= t) ++q;
  while (q > 0 && (int64_t)q * (q + 1) / 2 > t) --q;
  r = q;
  c = t - (int)((int64_t)q * (q + 1) / 2);
}

// the coordinates of tile `tile` of a launch: group-M rows over all tiles, or, for a triangular
// output, the tiles that meet the triangle, by rows
__device__ __forceinline__ void raster_coords(int tri, int tile, int tiles_m, int group_m, int num_tiles, int& tm,
                                              int& tn) {
  if (tri == 0) {
    tile_coords(tile, tiles_m, group_m, num_tiles, tm, tn);
    return;
  }
  int r, c;
  tri_tile(tile, r, c);
  tm = tri == 1 ? r : c;
  tn = tri == 1 ? c : r;
}

// the coordinates, in 128 x 128 tiles, of tile `tile` of a one-SM launch
__device__ __forceinline__ void tile128_coords(const ModArgs& p, int tile, int& tm, int& tn) {
  raster_coords(p.tri, tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
}

// the moduli [l0, l1) of work unit g of `groups` (at most nmod units per tile)
__device__ __forceinline__ void unit_range(int g, int groups, int nmod, int& l0, int& l1) {
  l0 = (int)((int64_t)g * nmod / groups);
  l1 = (int)((int64_t)(g + 1) * nmod / groups);
}

// x mod p for 0 <= x < 2^32 (Barrett: with b = floor(2^32/p), floor(x b / 2^32) is floor(x/p) or
// one less)
__device__ __forceinline__ uint32_t mod_barrett(uint32_t x, uint32_t p, uint32_t b) {
  uint32_t r = x - __umulhi(x, b) * p;
  return r >= p ? r - p : r;
}
// v mod p in [0, p) for |v| < 2^30 (shifted by p 2^23, which lies in [2^30, 2^31], into [0, 2^32))
__device__ __forceinline__ int mod_nonneg(int v, uint32_t p, uint32_t b) {
  return (int)mod_barrett((uint32_t)v + (p << 23), p, b);
}

// A grouped launch's table as the product kernels look units up in it: per entry its first tile,
// k-blocks, tile rows and tiles, and its plan's moduli count (0 for an infeasible plan).  Each CTA
// copies it into shared memory at its start when it fits (kTabCache entries), so that finding a
// unit's problem costs shared-memory reads instead of a chain of dependent global loads (table
// entry, plan); larger tables are read in global memory.
struct TabInfo {
  int tile_begin, nkb, tiles_m, group_m, num_tiles, nmod;
};
constexpr int kTabCache = 1024;
struct TabView {
  const ModTableEntry* table;
  const TabInfo* tab;  // the shared-memory copy, or null
  int count;
  __device__ __forceinline__ int begin(int i) const { return tab ? tab[i].tile_begin : (int)table[i].tile_begin; }
  __device__ __forceinline__ TabInfo info(int i) const {
    if (tab) return tab[i];
    const ModTableEntry& e = table[i];
    const ModPlan* pl = e.plan;
    return TabInfo{(int)e.tile_begin, e.nkb, e.tiles_m, e.group_m, e.num_tiles, pl->feasible ? pl->n : 0};
  }
  // the entry of `tile`, from entry cur on (the tiles a walk asks for increase)
  __device__ __forceinline__ int find(int tile, int cur) const {
    while (cur + 1 < count && begin(cur + 1) <= tile) ++cur;
    return cur;
  }
};
// the copy (every thread of the CTA takes part; a __syncthreads() must follow before its use)
__device__ __forceinline__ void tab_fill(TabInfo* tab, const ModTableEntry* table, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const ModTableEntry& e = table[i];
    const ModPlan* pl = e.plan;
    tab[i] = TabInfo{(int)e.tile_begin, e.nkb, e.tiles_m, e.group_m, e.num_tiles, pl->feasible ? pl->n : 0};
  }
}

// v mod p for an FP32 integer |v| <= 2^24 (one exact 1024-deep chunk), as the FP32 number
// 2^23 + r whose low byte is r in [0, p): with inv = fl(1/p), |v inv - v/p| <= 2^24 2^-24 / p < 0.01,
// so q = rint(v inv) (one fma against 1.5 2^23) is within 0.51 of v/p and r = v - p q (exact in
// one fma) lies in (-0.51 p, 0.51 p); p is added when r is negative.
__device__ __forceinline__ uint32_t mod_f32_byte(float v, float pf, float inv) {
  const float q = fmaf(v, inv, 12582912.0f) - 12582912.0f;
  const float r = fmaf(-pf, q, v);
  return __float_as_uint(r + (r < 0.0f ? 8388608.0f + pf : 8388608.0f));
}

// The epilogue of the product kernels.  Each thread owns one TMEM lane (a row of the CTA's 128)
// and COLS columns of the TBN-wide tile.  Per modulus: drain the 1024-deep chunks into int32
// sums (reduced modulo p_l every kReduceChunks chunks), reduce modulo p_l and park the residues,
// one byte each, in the block's plane of the park array (k_mod_crt rebuilds C from them).
// SPLIT: the work units are (tile, group of moduli); PAIR: (tile, modulus), modulus-major (unit u
// is modulus u / num_tiles of tile u % num_tiles); TABLE: the tiles belong to the problems of a
// grouped launch (table entries in tile order), and a tile whose problem's plan is infeasible is
// skipped (another kernel computes that problem).
// ONE: a modulus of one chunk (k <= 1024) is reduced in FP32 never (0), always (1: the launch's k
// is that small) or when its problem's k is (2)
template <int EPI_WARPS, int TBN, bool PAIR, bool TABLE, bool SPLIT, int ONE = 2>
__device__ __forceinline__ void mod_park(const ModArgs& p, int nmod, uint32_t tmem_base, uint64_t* acc_full,
                                         uint64_t* acc_empty, int warp, int lane, int unit0, int unit_step,
                                         int units, int row_off, const ModTableEntry* table = nullptr,
                                         int count = 0, const TabInfo* tab = nullptr) {
  const TabView tv{table, tab, count};
  constexpr int COLS = TBN / (EPI_WARPS / 4);
  constexpr int kGroups = COLS / 4;
  static_assert(COLS % 4 == 0 && 128 % COLS == 0, "a thread's columns lie in one 128-column block");
  const int ew = warp - 2;
  const int quad = warp & 3;
  const int part = ew >> 2;
  const int row = quad * 32 + lane;
  const int col0 = part * COLS;
  const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
  uint32_t empty_remote[2] = {0u, 0u};
  if (PAIR) {
    empty_remote[0] = map_to_rank(smem_u32(&acc_empty[0]), 0);
    empty_remote[1] = map_to_rank(smem_u32(&acc_empty[1]), 0);
  }
  const int groups = SPLIT ? min(p.groups, nmod) : 1;
  uint32_t chunk = 0;
  int acc[COLS];
  int cur = 0;      // grouped: the table entry of the current tile (a CTA's tiles increase)
  int cur_l = -1;   // grouped pairs: the modulus of the current sweep (the tiles restart with it)
  for (int u = unit0; u < units; u += unit_step) {
    const int tile = SPLIT ? u / groups : PAIR ? u % p.num_tiles : u;
    int l0 = 0, l1 = nmod, nkb = p.nkb, tm, tn;
    uint8_t* park = p.park;
    int pmods = p.park_mods, nbn = p.nbn;
    int64_t pm = p.m, pn = p.n;
    if (SPLIT) unit_range(u % groups, groups, nmod, l0, l1);
    if (PAIR) {
      l0 = u / p.num_tiles;
      l1 = l0 + 1;
    }
    if (TABLE) {
      if (PAIR && l0 != cur_l) {
        cur = 0;
        cur_l = l0;
      }
      cur = tv.find(tile, cur);
      const TabInfo ti = tv.info(cur);
      if (ti.nmod == 0) continue;  // an infeasible plan: computed by the FP64 kernel instead
      if (PAIR) {
        if (l0 >= ti.nmod) continue;  // this problem has fewer moduli than the launch's largest
      } else {
        l1 = ti.nmod;
      }
      nkb = ti.nkb;
      tile_coords(tile - ti.tile_begin, ti.tiles_m, ti.group_m, ti.num_tiles, tm, tn);
      const ModTableEntry& e = table[cur];
      park = e.park;
      pmods = e.park_mods;
      nbn = e.nbn;
      pm = e.m;
      pn = e.n;
    } else if (PAIR) {
      raster_coords(p.tri, tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
    } else {
      tile128_coords(p, tile, tm, tn);
    }
    // this thread's 128 x 128 block of C; a block wholly outside C is not parked
    const int rb = PAIR ? 2 * tm + (row_off >> 7) : tm;
    const int cb = PAIR ? 2 * tn + (col0 >> 7) : tn;
    const bool inside = (int64_t)rb * 128 < pm && (int64_t)cb * 128 < pn;
    uint8_t* const pb = park + ((int64_t)rb * nbn + cb) * pmods * kParkBlock + (int64_t)((col0 & 127) / 4) * 512 +
                        row * 4;
    for (int l = l0; l < l1; ++l) {
      const uint32_t pmod = (uint32_t)p.p[l], bm = p.bar[l];
      if (ONE == 1 || (ONE == 2 && nkb <= kChunkBlocks)) {
        // one chunk: its exact FP32 sums reduced in FP32 and parked slice by slice, each 16-column
        // TMEM load issued before the previous slice's arithmetic; the buffer is freed at the end
        const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
        ++chunk;
        mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
        tc_fence_after();
        const uint32_t taddr = trow + buf * TBN + col0;
        const float pf = (float)pmod, inv = p.pinv[l];
        unsigned int* const dst = reinterpret_cast<unsigned int*>(pb + (int64_t)l * kParkBlock);
        uint32_t va[16], vb[16];
        tmem_ld_16_issue(taddr, va);
#pragma unroll
        for (int q = 0; q < COLS / 16; ++q) {
          uint32_t(&cur)[16] = (q & 1) ? vb : va;
          uint32_t(&nxt)[16] = (q & 1) ? va : vb;
          tmem_wait_ld_16(cur);
          if (q + 1 < COLS / 16) tmem_ld_16_issue(taddr + (q + 1) * 16, nxt);
          uint32_t b[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) b[jj] = mod_f32_byte(__uint_as_float(cur[jj]), pf, inv);
          if (inside) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const uint32_t lo = __byte_perm(b[4 * g], b[4 * g + 1], 0x0040u);
              const uint32_t hi = __byte_perm(b[4 * g + 2], b[4 * g + 3], 0x0040u);
              __stcs(dst + (4 * q + g) * 128, __byte_perm(lo, hi, 0x5410u));  // read once, by the reconstruction
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (PAIR) mbar_arrive_remote(empty_remote[buf]);
          else mbar_arrive(&acc_empty[buf]);
        }
        continue;
      }
      if constexpr (ONE != 1) {  // int32 sums over the chunks, reduced modulo p_l every kReduceChunks
#pragma unroll
        for (int c = 0; c < COLS; ++c) acc[c] = 0;
        int nch = 0;
        for (int i0 = 0; i0 < nkb; i0 += kChunkBlocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
          tc_fence_after();
          const uint32_t taddr = trow + buf * TBN + col0;
#pragma unroll
          for (int q = 0; q < COLS / 16; ++q) {
            uint32_t v[16];
            tmem_ld_16(taddr + q * 16, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) acc[q * 16 + jj] += __float2int_rn(__uint_as_float(v[jj]));
          }
          // the warp's TMEM loads are complete (waited on) and fenced: one arrive per warp frees the
          // buffer (a release-ordered remote arrive per thread stalled the epilogue on its fences)
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (PAIR) mbar_arrive_remote(empty_remote[buf]);
            else mbar_arrive(&acc_empty[buf]);
          }
          if (++nch == kReduceChunks) {  // keep the running sums below 2^30 in magnitude
            nch = 0;
#pragma unroll
            for (int c = 0; c < COLS; ++c) acc[c] = mod_nonneg(acc[c], pmod, bm);
          }
        }
        if (inside) {
          unsigned int* const dst = reinterpret_cast<unsigned int*>(pb + (int64_t)l * kParkBlock);
#pragma unroll
          for (int g = 0; g < kGroups; ++g) {
            uint32_t w = 0u;
#pragma unroll
            for (int b = 0; b < 4; ++b) w |= (uint32_t)mod_nonneg(acc[4 * g + b], pmod, bm) << (8 * b);
            __stcs(dst + g * 128, w);  // read once, by the reconstruction
          }
        }
      }
    }
  }
}

// ---- the one-SM form: 128 x 128 tiles ----
constexpr int kBM = 128, kBN = 128;
constexpr int kStages = 6;
constexpr int kEpiWarps = 16;  // 4 x 4 warps over 128 TMEM lanes x 128 columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kTmemCols = 2 * kBN;  // two accumulators

struct Smem {
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = kBN * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + kStages * kABytes;
  static constexpr int kOffBar = kOffB + kStages * kBBytes;
  static constexpr int kNumBars = 2 * kStages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kOffTab = kOffTmemSlot + 16;  // grouped launches: the table's copy
  static constexpr int kBytes = kOffTab + kTabCache * (int)sizeof(TabInfo);
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

// SPLIT: the work units are (tile, group of moduli) instead of tiles (few-tile problems).
// TABLE: the tiles of several problems (a grouped launch): entries in tile order, each with its
// problem's residue maps and device plan; tiles of an infeasible plan are skipped.
template <bool SPLIT, bool TABLE = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_mod_gemm(const __grid_constant__ ModArgs p, const __grid_constant__ CUtensorMap tmA,
               const __grid_constant__ CUtensorMap tmB, const ModTableEntry* __restrict__ table = nullptr,
               int count = 0) {
  static_assert(!(SPLIT && TABLE), "the grouped form has whole tiles as work units");
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
      mbar_init(&acc_empty[i], kEpiWarps);  // one arrive per epilogue warp
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
  TabInfo* const tab_s = reinterpret_cast<TabInfo*>(smem + L::kOffTab);
  const bool tab_cached = TABLE && count <= kTabCache;
  if (tab_cached) tab_fill(tab_s, table, count);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const ModPlan plan = *p.plan;  // written by k_mod_plan earlier on the stream (grouped: the first problem's)
  const int nmod = plan.n;
  // work units: tiles, or (tile, group of moduli) with at most nmod groups per tile
  const int groups = SPLIT ? min(p.groups, nmod) : 1;
  const int units = p.num_tiles * groups;
  // grouped: the moduli count and k-blocks of unit u's problem (0 moduli: skipped), its maps
  const TabView tv{table, tab_cached ? tab_s : nullptr, count};
  auto table_unit = [&](int u, int& cur, int& tm, int& tn, int& nm, int& nkb, const CUtensorMap*& ma,
                        const CUtensorMap*& mb) {
    cur = tv.find(u, cur);
    const TabInfo ti = tv.info(cur);
    nm = ti.nmod;
    nkb = ti.nkb;
    tile_coords(u - ti.tile_begin, ti.tiles_m, ti.group_m, ti.num_tiles, tm, tn);
    ma = &table[cur].tmA;
    mb = &table[cur].tmB;
  };

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      const uint32_t bytes = (uint32_t)(L::kABytes + L::kBBytes);
      int cur = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int tile = u / groups;
        int l0 = 0, l1 = nmod, nkb = p.nkb;
        if (SPLIT) unit_range(u % groups, groups, nmod, l0, l1);
        int tm, tn;
        const CUtensorMap* ma = &tmA;
        const CUtensorMap* mb = &tmB;
        if (TABLE) {
          table_unit(u, cur, tm, tn, l1, nkb, ma, mb);
          if (l1 == 0) continue;
          // maps written into global memory before the launch: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ma) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mb) : "memory");
        } else {
          tile128_coords(p, tile, tm, tn);
        }
        for (int l = l0; l < l1; ++l)
          for (int kb = 0; kb < nkb; ++kb) {
            mbar_wait(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
            mbar_arrive_expect_tx(&full[stage], bytes);
            tma_load_3d(smem + L::kOffA + stage * L::kABytes, ma, &full[stage], kb * kBK, tm * kBM, l);
            tma_load_3d(smem + L::kOffB + stage * L::kBBytes, mb, &full[stage], kb * kBK, tn * kBN, l);
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
      int cur = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        int l0 = 0, l1 = nmod, nkb = p.nkb;
        if (SPLIT) unit_range(u % groups, groups, nmod, l0, l1);
        if (TABLE) {
          int tm, tn;
          const CUtensorMap *ma, *mb;
          table_unit(u, cur, tm, tn, l1, nkb, ma, mb);
        }
        for (int l = l0; l < l1; ++l)
          for (int i0 = 0; i0 < nkb; i0 += kChunkBlocks, ++chunk) {
            const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
            mbar_wait(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
            tc_fence_after();
            const uint32_t dtm = tmem_base + buf * kBN;
            const int i1 = min(nkb, i0 + kChunkBlocks);
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
      }
      if (chunk > 0) {  // a CTA without a unit issued nothing and has nothing to wait for
        umma_commit(done);
        mbar_wait(done, 0, p.err, kErrWaitMma);
      }
    }
    __syncwarp();
  } else {
    mod_park<kEpiWarps, kBN, false, TABLE, SPLIT>(p, nmod, tmem_base, acc_full, acc_empty, warp, lane, blockIdx.x,
                                                  gridDim.x, units, 0, table, count, tab_cached ? tab_s : nullptr);
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
constexpr int k2TmemCols = 2 * k2BN;
static_assert(kBM == 128 && kBN == 128 && k2BN == 256, "the park array is laid out in 128 x 128 blocks");

struct Smem2 {
  static constexpr int kABytes = 128 * kBK * 2;
  static constexpr int kBBytes = 128 * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + k2Stages * kABytes;
  static constexpr int kOffBar = kOffB + k2Stages * kBBytes;
  static constexpr int kNumBars = 2 * k2Stages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kOffTab = kOffTmemSlot + 16;  // grouped launches: the table's copy
  static constexpr int kBytes = kOffTab + kTabCache * (int)sizeof(TabInfo);
  static constexpr int kAlloc = kBytes + 1024;
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

// TABLE: the tiles of several problems (a grouped launch, `count` table entries whose tiles are
// numbered in order, 256 x 256 each), their moduli swept together up to the largest count of any
// plan (*nmax); a unit beyond its own problem's count, or of an infeasible plan, is skipped.
// ONE as for mod_park (single products: 1 when k <= 1024, else 0; grouped: 2)
template <bool TABLE, int ONE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(k2Threads, 1)
    k_mod_gemm_pair(const __grid_constant__ ModArgs p, const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, const ModTableEntry* __restrict__ table = nullptr,
                    int count = 0, const unsigned int* __restrict__ nmax = nullptr) {
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
    if (!TABLE) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
    }
    for (int i = 0; i < k2Stages; ++i) {
      mbar_init(&full[i], 1);   // the leader's producer arrives (with both CTAs' bytes)
      mbar_init(&empty[i], 1);  // one commit per phase, multicast to both CTAs
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 2 * k2EpiWarps);  // one arrive per epilogue warp of both CTAs
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
  TabInfo* const tab_s = reinterpret_cast<TabInfo*>(smem + L::kOffTab);
  const bool tab_cached = TABLE && count <= kTabCache;
  if (tab_cached) tab_fill(tab_s, table, count);
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // the peer's barriers are initialised and its TMEM is allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // single product: the call's plan; grouped: the largest moduli count of the problems' plans
  // (written by the plan kernels earlier on the stream; 0 when no plan is feasible)
  const int nmod = TABLE ? (int)*nmax : p.plan->n;
  // work units (tile, modulus), modulus-major: the pairs sweep the tiles of one modulus's planes
  // together, so a band of them stays in L2, and every pair has work down to the last wave
  const int units = p.num_tiles * nmod;
  // grouped: unit u's problem (table cursor `cur`, restarted with each modulus `cur_l`), its tile
  // coordinates, k-blocks and residue maps; false when the unit is skipped
  const TabView tv{table, tab_cached ? tab_s : nullptr, count};
  auto table_unit = [&](int u, int& cur, int& cur_l, int& tm, int& tn, int& nkb, const CUtensorMap*& ma,
                        const CUtensorMap*& mb) {
    const int tile = u % p.num_tiles, l = u / p.num_tiles;
    if (l != cur_l) {
      cur = 0;
      cur_l = l;
    }
    cur = tv.find(tile, cur);
    const TabInfo ti = tv.info(cur);
    if (l >= ti.nmod) return false;  // an infeasible plan (no moduli), or fewer moduli than l + 1
    nkb = ti.nkb;
    tile_coords(tile - ti.tile_begin, ti.tiles_m, ti.group_m, ti.num_tiles, tm, tn);
    ma = &table[cur].tmA;
    mb = &table[cur].tmB;
    return true;
  };

  if (warp == 0) {
    // ------------------------------ TMA producer (both CTAs) ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      const uint32_t pair_bytes = (uint32_t)(2 * (L::kABytes + L::kBBytes));
      int cur = 0, cur_l = -1;
      for (int u = pair_id; u < units; u += num_pairs) {
        const int l = u / p.num_tiles;
        int tm, tn, nkb = p.nkb;
        const CUtensorMap* ma = &tmA;
        const CUtensorMap* mb = &tmB;
        if (TABLE) {
          if (!table_unit(u, cur, cur_l, tm, tn, nkb, ma, mb)) continue;
          // maps written into global memory before the launch: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ma) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mb) : "memory");
        } else {
          raster_coords(p.tri, u % p.num_tiles, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
        }
        const int m0 = tm * k2BM + (int)rank * 128;
        const int nb0 = tn * k2BN + (int)rank * 128;
        for (int kb = 0; kb < nkb; ++kb) {
          mbar_wait_cluster(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
          if (leader) mbar_arrive_expect_tx(&full[stage], pair_bytes);
          const uint32_t fbar = map_to_rank(smem_u32(&full[stage]), 0);
          tma_load_3d_pair(smem + L::kOffA + stage * L::kABytes, ma, fbar, kb * kBK, m0, l);
          tma_load_3d_pair(smem + L::kOffB + stage * L::kBBytes, mb, fbar, kb * kBK, nb0, l);
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
      int cur = 0, cur_l = -1;
      for (int u = pair_id; u < units; u += num_pairs) {
        int nkb = p.nkb;
        if (TABLE) {
          int tm, tn;
          const CUtensorMap *ma, *mb;
          if (!table_unit(u, cur, cur_l, tm, tn, nkb, ma, mb)) continue;
        }
        for (int i0 = 0; i0 < nkb; i0 += kChunkBlocks, ++chunk) {
          const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
          mbar_wait_cluster(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
          tc_fence_after();
          const uint32_t dtm = tmem_base + buf * k2BN;
          const int i1 = min(nkb, i0 + kChunkBlocks);
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
      }
      if (chunk > 0) {  // a pair without a unit issued nothing and has nothing to wait for
        umma_commit_pair(done);
        mbar_wait_cluster(done, 0, p.err, kErrWaitMma);
      }
    }
    __syncwarp();
  } else {
    mod_park<k2EpiWarps, k2BN, true, TABLE, false, ONE>(p, nmod, tmem_base, acc_full, acc_empty, warp, lane, pair_id,
                                                   num_pairs, units, (int)rank * 128, table, count,
                                                   tab_cached ? tab_s : nullptr);
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

// ---- the reconstruction: C from the parked residues ----
// One CTA of 256 threads per 128 x 128 block of C at a time: thread (row, g) rebuilds the four
// columns 4g .. 4g+3 of its row from one word per modulus, g = threadIdx.x / 128 + 2 i.  A warp
// reads 128 contiguous bytes per modulus and writes 32 consecutive rows of a column.
// C := fma(alpha 2^(tau_j - 2t), fl(C') 2^sigma_i, beta C0), fl correctly rounded (ties to even)
// and the scaling as ldexp; NaN for a row or column with a non-finite entry, and everywhere when
// the plan found the target unreachable.  The arithmetic is on 32-bit limbs, specialised for the
// number of moduli N (L = 3 limbs while M < 2^95, that is N <= 12, else 4), so that the
// constants are immediate operands; when beta = 0 and alpha 2^(tau_j - 2t) is a power of two
// (alpha a power of two) the result is assembled from integers, without FP64 arithmetic.
constexpr int kCrtThreads = 256;

template <int L>
__device__ __forceinline__ void limbs_add(uint32_t (&x)[L], const uint32_t (&y)[L]) {
  if constexpr (L == 3) {
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]));
  } else {
    asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.cc.u32 %2, %2, %6;\n\taddc.u32 %3, %3, %7;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]));
  }
}
template <int L>
__device__ __forceinline__ void limbs_sub(uint32_t (&x)[L], const uint32_t (&y)[L]) {
  if constexpr (L == 3) {
    asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]));
  } else {
    asm("sub.cc.u32 %0, %0, %4;\n\tsubc.cc.u32 %1, %1, %5;\n\tsubc.cc.u32 %2, %2, %6;\n\tsubc.u32 %3, %3, %7;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]));
  }
}

// fl(C') for the residues T (four moduli per word, modulus 4G + b in byte b of T[G]): the sign,
// the unbiased exponent E of the rounded value and its 53-bit significand with the implicit bit
// (mant in [2^52, 2^53], 2^53 when the rounding carried), or zero.  X = sum_l r_l V_l modulo
// 2^(32 L) from the byte sums S_d = sum_l r_l (byte d of V_l) < 2^20 (four moduli per dp4a), as
// X = sum_k 2^(32 k) (A_k + 2^16 B_k), A_k = S_4k + 2^8 S_4k+1, B_k = S_4k+2 + 2^8 S_4k+3 (each
// below 2^29): limb k is A_k + (B_k << 16 mod 2^32) + (B_k-1 >> 16) plus the carry of limb k - 1,
// the first two terms summed with carries (the third keeps A_k below 2^30).  Qe = floor(sum_l
// r_l e_l / 2^16 + 1/2) is round(X / M) or one more, and one more only when X - Qe M <= -M/2:
// then M is added back.  The result lies in (-M/2, M/2].
template <int N>
__device__ __forceinline__ bool crt_round(const CrtSet& S, const uint32_t (&T)[(N + 3) / 4], uint32_t& sign, int& E,
                                          uint64_t& mant) {
  constexpr int L = N <= 12 ? 3 : 4;
  constexpr int NG = (N + 3) / 4;
  uint32_t a[L], lo[L], bprev = 0u;
#pragma unroll
  for (int k = 0; k < L; ++k) {
    uint32_t s1 = 0u, s3 = 0u;
#pragma unroll
    for (int G = 0; G < NG; ++G) {
      s1 = __dp4a(T[G], S.wp[G][4 * k + 1], s1);
      s3 = __dp4a(T[G], S.wp[G][4 * k + 3], s3);
    }
    uint32_t A = s1 << 8, B = s3 << 8;
#pragma unroll
    for (int G = 0; G < NG; ++G) {
      A = __dp4a(T[G], S.wp[G][4 * k], A);
      B = __dp4a(T[G], S.wp[G][4 * k + 2], B);
    }
    a[k] = A + (bprev >> 16);
    lo[k] = B << 16;
    bprev = B;
  }
  uint32_t x[L];
#pragma unroll
  for (int k = 0; k < L; ++k) x[k] = a[k];
  limbs_add<L>(x, lo);
  uint32_t qh = 0u;
#pragma unroll
  for (int G = 0; G < NG; ++G) qh = __dp4a(T[G], S.ep[G][1], qh);
  uint32_t qe = (qh << 8) + (1u << 15);
#pragma unroll
  for (int G = 0; G < NG; ++G) qe = __dp4a(T[G], S.ep[G][0], qe);
  // X - Qe M
  const uint32_t Q = qe >> 16;
  uint32_t qm[L];
  uint64_t t = (uint64_t)Q * S.M[0];
  qm[0] = (uint32_t)t;
#pragma unroll
  for (int j = 1; j < L; ++j) {
    t = (t >> 32) + (uint64_t)Q * S.M[j];
    qm[j] = (uint32_t)t;
  }
  limbs_sub<L>(x, qm);
  // X - Qe M <= -M/2 exactly when X - Qe M + (M/2 - 1) is negative
  uint32_t h[L];
#pragma unroll
  for (int j = 0; j < L; ++j) h[j] = x[j];
  uint32_t hc[L];
#pragma unroll
  for (int j = 0; j < L; ++j) hc[j] = S.H[j];
  limbs_add<L>(h, hc);
  const uint32_t fix = 0u - (h[L - 1] >> 31);
  uint32_t mm[L];
#pragma unroll
  for (int j = 0; j < L; ++j) mm[j] = S.M[j] & fix;
  limbs_add<L>(x, mm);
  // sign and magnitude
  sign = x[L - 1] >> 31;
  const uint32_t neg = 0u - sign;
  uint32_t sg[L];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    x[j] ^= neg;
    sg[j] = j == 0 ? sign : 0u;
  }
  limbs_add<L>(x, sg);
  // normalise: the leading one to bit 32 L - 1
  int lz = 0;
#pragma unroll
  for (int step = 0; step < L - 1; ++step) {
    if (x[L - 1] == 0u) {
#pragma unroll
      for (int j = L - 1; j > 0; --j) x[j] = x[j - 1];
      x[0] = 0u;
      lz += 32;
    }
  }
  if (x[L - 1] == 0u) return false;  // C' = 0
  const int c = __clz((int)x[L - 1]);
#pragma unroll
  for (int j = L - 1; j > 0; --j) x[j] = __funnelshift_l(x[j - 1], x[j], c);
  x[0] <<= c;
  lz += c;
  E = 32 * L - 1 - lz;
  // the top 53 bits, rounded to nearest, ties to even, on the 32 L - 53 bits below
  const uint64_t m = ((uint64_t)x[L - 1] << 21) | (x[L - 2] >> 11);
  uint32_t sticky = x[L - 2] & 0x3FFu;
#pragma unroll
  for (int j = 0; j < L - 2; ++j) sticky |= x[j];
  const uint32_t half = (x[L - 2] >> 10) & 1u;
  mant = m + (half & ((sticky != 0u) | (uint32_t)(m & 1u)));
  return true;
}

template <int N>
__device__ __forceinline__ void crt_rows(const CrtJob& job, bool nan_out, int rb, int cb) {
  const CrtSet& S = kCrt.set[N - 1];
  // the job's fields in registers (the stores to C cannot alias them then)
  const int64_t m = job.m, n = job.n, ldc = job.ldc;
  const double beta = job.beta;
  const int tri = job.tri;
  double* const C = job.C;
  const double* const cs = job.cs;
  const int row = threadIdx.x & 127;
  const int64_t i = (int64_t)rb * 128 + row;
  if (i >= m) return;
  const int sg = job.sigA[i];
  const int sig = sg == kExpEmpty ? 0 : sg;
  const bool bad = nan_out || job.badA[i] != 0;
  const bool beta0 = beta == 0.0;
  const uint8_t* const pb = job.park + ((int64_t)rb * job.nbn + cb) * job.park_mods * kParkBlock + row * 4;
  for (int g = threadIdx.x >> 7; g < 32; g += kCrtThreads / 128) {
    const int64_t j0 = (int64_t)cb * 128 + 4 * g;
    if (j0 >= n) break;
    constexpr int NG = (N + 3) / 4;
    uint32_t w[4 * NG];
#pragma unroll
    for (int l = 0; l < N; ++l)
      w[l] = __ldcs(reinterpret_cast<const unsigned int*>(pb + (int64_t)l * kParkBlock + g * 512));
#pragma unroll
    for (int l = N; l < 4 * NG; ++l) w[l] = 0u;
    // word l holds column 4g + q's residue modulo p_l in byte q: a 4 x 4 byte transpose per group
    // of four moduli gives each column its residues, four moduli per word (byte b: modulus 4G + b)
    uint32_t T[4][NG];
#pragma unroll
    for (int G = 0; G < NG; ++G) {
      const uint32_t t01 = __byte_perm(w[4 * G], w[4 * G + 1], 0x5140u);      // bytes 0, 1 of both
      const uint32_t t23 = __byte_perm(w[4 * G + 2], w[4 * G + 3], 0x5140u);
      const uint32_t u01 = __byte_perm(w[4 * G], w[4 * G + 1], 0x7362u);      // bytes 2, 3 of both
      const uint32_t u23 = __byte_perm(w[4 * G + 2], w[4 * G + 3], 0x7362u);
      T[0][G] = __byte_perm(t01, t23, 0x5410u);
      T[1][G] = __byte_perm(t01, t23, 0x7632u);
      T[2][G] = __byte_perm(u01, u23, 0x5410u);
      T[3][G] = __byte_perm(u01, u23, 0x7632u);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t jj = j0 + q;
      const bool in = jj < n && (tri == 0 || (tri == 1 ? jj <= i : jj >= i));
      if (!in) continue;
      const double csv = cs[jj];
      const uint64_t cbits = (uint64_t)__double_as_longlong(csv);
      double* const dst = C + jj * ldc + i;
      if (bad || (cbits << 1) > 0xFFE0000000000000ull) {  // a non-finite row or column (NaN scale)
        *dst = __longlong_as_double(0x7FF8000000000000ll);
        continue;
      }
      uint32_t sign;
      int E;
      uint64_t mant;
      const bool nz = crt_round<N>(S, T[q], sign, E, mant);
      // y = fl(C') 2^sigma_i: its bits while it is a normal number (the rounding's carry moves
      // into the exponent field)
      const int ey = E + sig + 1023;  // biased exponent before the carry
      const uint64_t ybits = nz ? ((uint64_t)(ey - 1) << 52) + mant : 0ull;
      const bool y_normal = !nz || (ey >= 1 && (ybits >> 52) <= 2046);
      const int ecs = (int)((cbits >> 52) & 0x7FF);
      if (beta0 && y_normal && (cbits & 0x000FFFFFFFFFFFFFull) == 0 && ecs >= 1 && ecs <= 2046) {
        // alpha 2^(tau_j - 2t) = +-2^(ecs - 1023): an exact scaling while the result stays normal
        if (!nz) {
          *dst = 0.0;  // fma(cs, +0, +0) = +0
          continue;
        }
        const int eo = (int)(ybits >> 52) + ecs - 1023;
        if (eo >= 1 && eo <= 2046) {
          const uint64_t ob = (ybits + ((uint64_t)(int64_t)(ecs - 1023) << 52)) |
                              ((uint64_t)(sign ^ (uint32_t)(cbits >> 63)) << 63);
          *dst = __longlong_as_double((long long)ob);
          continue;
        }
      }
      double y = 0.0;
      if (nz) {
        if (y_normal) y = __longlong_as_double((long long)ybits);
        else y = ldexp((double)mant, E - 52 + sig);  // one rounding of the exact fl(C') 2^sigma_i
        if (sign) y = -y;
      }
      const double w0 = beta0 ? 0.0 : beta * *dst;
      *dst = fma(csv, y, w0);
    }
  }
}

// each count of moduli its own function (register allocation of one specialisation at a time)
template <int N>
__device__ __noinline__ void crt_block_n(const CrtJob& j, bool nan_out, int rb, int cb) {
  crt_rows<N>(j, nan_out, rb, cb);
}

__device__ __forceinline__ void crt_block(const CrtJob& j, int64_t blk) {
  const ModPlan pl = *j.plan;
  if (!pl.feasible && j.skip_infeasible) return;
  const int rb = (int)(blk / j.nbn), cb = (int)(blk % j.nbn);
  // a triangular output: the blocks wholly outside the triangle were never multiplied
  if ((j.tri == 1 && cb > rb) || (j.tri == 2 && cb < rb)) return;
  const bool nan_out = !pl.feasible;
  switch (pl.n) {
    case 1: crt_block_n<1>(j, nan_out, rb, cb); break;
    case 2: crt_block_n<2>(j, nan_out, rb, cb); break;
    case 3: crt_block_n<3>(j, nan_out, rb, cb); break;
    case 4: crt_block_n<4>(j, nan_out, rb, cb); break;
    case 5: crt_block_n<5>(j, nan_out, rb, cb); break;
    case 6: crt_block_n<6>(j, nan_out, rb, cb); break;
    case 7: crt_block_n<7>(j, nan_out, rb, cb); break;
    case 8: crt_block_n<8>(j, nan_out, rb, cb); break;
    case 9: crt_block_n<9>(j, nan_out, rb, cb); break;
    case 10: crt_block_n<10>(j, nan_out, rb, cb); break;
    case 11: crt_block_n<11>(j, nan_out, rb, cb); break;
    case 12: crt_block_n<12>(j, nan_out, rb, cb); break;
    case 13: crt_block_n<13>(j, nan_out, rb, cb); break;
    case 14: crt_block_n<14>(j, nan_out, rb, cb); break;
    case 15: crt_block_n<15>(j, nan_out, rb, cb); break;
    default: crt_block_n<16>(j, nan_out, rb, cb); break;
  }
}

// one product (jobs == nullptr: `one`), or the jobs of a grouped launch (blocks in job order; their
// first blocks in `begins` when it holds every job, else read from the table)
__global__ void __launch_bounds__(kCrtThreads, 3) k_mod_crt(const __grid_constant__ CrtJob one,
                                                            const CrtJob* __restrict__ jobs, int count, int64_t total,
                                                            const __grid_constant__ JobBegins begins) {
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    if (!jobs) {
      crt_block(one, b);
      continue;
    }
    int lo = 0, hi = count - 1;  // the last job whose blocks begin at or before b
    const bool cached = begins.n == count;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((cached ? begins.b[mid] : jobs[mid].blk_begin) <= b) lo = mid;
      else hi = mid - 1;
    }
    crt_block(jobs[lo], b - (cached ? begins.b[lo] : jobs[lo].blk_begin));
  }
}

// alpha 2^(tau_j - 2t) for every column (NaN for a column with a non-finite entry)
__global__ void __launch_bounds__(256) k_mod_colscale(const int* __restrict__ sigB, const int* __restrict__ badB,
                                                      int64_t n, double alpha, const ModPlan* __restrict__ plan,
                                                      double* __restrict__ cs) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int t = plan->t;
  const int tau = sigB[j] == kExpEmpty ? 0 : sigB[j];
  cs[j] = badB[j] ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(alpha, tau - 2 * t);
}

typedef unsigned __int128 hu128;

// products of the first n moduli, n = 1..kMaxModuli
struct ModProducts {
  uint64_t lo[kMaxModuli], hi[kMaxModuli];
};

// fewest moduli whose product exceeds `need`; 0 when none is enough
__host__ __device__ inline int moduli_above(hu128 need, const ModProducts& mp) {
  for (int n = 1; n <= kMaxModuli; ++n)
    if ((((hu128)mp.hi[n - 1] << 64) | mp.lo[n - 1]) > need) return n;
  return 0;
}

// fewest moduli whose product exceeds 2 k 2^(2t) >= 2 max |A'B'|; 0 when none is enough
__host__ __device__ int moduli_for_products(int t, int64_t k, const ModProducts& mp) {
  if (t < 1 || k < 1) return 0;
  // k > 2^(kb-1): from 2t + kb >= 126 on, 2 k 2^(2t) > 2^126 exceeds every product;
  // below it, 2 k 2^(2t) < 2^127 is computed exactly
  int kb = 0;
  while (((int64_t)1 << kb) < k) ++kb;
  if (2 * t + kb >= 126) return 0;
  return moduli_above(((hu128)2 * (hu128)k) << (2 * t), mp);
}

// The same from the square sums: with a2 >= max_i ||a^_i||^2 and b2 >= max_j ||b^_j||^2 (rows of
// op(A), columns of op(B), scaled by 2^-sigma_i, 2^-tau_j) and the rounded integers
// A'_ip = rn(a^_ip 2^t), |A'_ip - a^_ip 2^t| <= 1/2, Cauchy-Schwarz and the triangle inequality give
//     |(A'B')_ij| <= ||A'_i|| ||B'_j|| <= 2^(2t) (sqrt(a2) + sqrt(k) 2^(-t-1)) (sqrt(b2) + sqrt(k) 2^(-t-1)),
// which is below k 2^(2t) when the rows are not all of full magnitude.  The product is formed in
// double precision (a few correctly rounded operations, covered by the factor 1 + 2^-40) and
// rounded up to an integer.
__host__ __device__ int moduli_for_norms(int t, int64_t k, float a2, float b2, const ModProducts& mp) {
  const int nk = moduli_for_products(t, k, mp);
  if (t < 1 || k < 1 || t > 62 || !(a2 >= 0.0f) || !(b2 >= 0.0f)) return nk;
  const double h = ldexp(sqrt((double)k), -t - 1);
  double x = (sqrt((double)a2) + h) * (sqrt((double)b2) + h) * (1.0 + 0x1p-40);
  if (x >= (double)k) return nk;
  const double need = ldexp(x, 2 * t + 1);  // 2 x 2^(2t) < 2 k 2^(2t) <= 2^126 unless nk == 0
  if (need >= 0x1p126) return nk;
  const double hi = floor(ldexp(need, -64));
  const double lo = ceil(need - ldexp(hi, 64));  // an integer below 2^64
  const int ncs = moduli_above(((hu128)(uint64_t)hi << 64) | (hu128)(uint64_t)lo, mp);
  return (ncs && (nk == 0 || ncs < nk)) ? ncs : nk;
}

// The call's plan, on one warp: t given (fixed_t > 0), or the certified choice from the
// certification words (cert_mod_bits: the smallest t whose a-priori bound stays within the
// target on every element, or the exactness width); then n.  When no n <= kMaxModuli suffices
// the plan is marked infeasible (n = 1, t = 1: the kernels then write NaN) and, for the
// device-side automatic mode (`flag`), the device error word records it.
// retry: the second plan, from the BF16 certification's words, only when the first was infeasible
__global__ void __launch_bounds__(32) k_mod_plan(const unsigned int* __restrict__ cert, int64_t k, double tol,
                                                  int fixed_t, const __grid_constant__ ModProducts mp,
                                                  ModPlan* __restrict__ plan, unsigned int* err, int flag,
                                                  int retry) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  // the automatic mode's square-sum bounds (written by the exponent pass into the first set)
  const float a2 = __uint_as_float(cert[kCertNormA]), b2 = __uint_as_float(cert[kCertNormB]);
  if (retry) {
    if (plan->feasible) return;
    cert += kCertRetry;
  }
  double rho = 0.0, gamma = 0.0, bound = 0.0;
  int t = fixed_t, exact = 0;
  if (fixed_t <= 0) {
    cert_rho_gamma(cert, &rho, &gamma);
    t = cert_mod_bits(rho, gamma, (int)cert[kCertTexA], (int)cert[kCertTexB], k, tol, &bound, &exact);
  }
  const int n = t > 62 ? 0 : fixed_t <= 0 ? moduli_for_norms(t, k, a2, b2, mp) : moduli_for_products(t, k, mp);
  ModPlan pl;
  pl.t = n ? t : 1;
  pl.n = n ? n : 1;
  pl.feasible = n != 0;
  pl.want = t;
  pl.exact = exact;
  pl.pad = 0;
  pl.rho = rho;
  pl.gamma = gamma;
  pl.bound = bound;
  *plan = pl;
  if (!n && flag) atomicOr(err, kErrModRange);
}

// the plans of a grouped launch, one thread per problem (as k_mod_plan; an infeasible plan needs no
// error bit: the grouped FP64 kernel computes that problem).  An infeasible plan sets flags[0] on
// the first pass and flags[1] on the final one (the retry, or the first when no retry follows).
__global__ void __launch_bounds__(128) k_mod_plan_batched(const ModPlanJob* __restrict__ jobs, int count,
                                                          const __grid_constant__ ModProducts mp, int retry,
                                                          unsigned int* __restrict__ flags, int final_pass) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const ModPlanJob j = jobs[q];
  if (retry && j.plan->feasible) return;
  const unsigned int* words = retry ? j.words + kCertRetry : j.words;
  double rho = 0.0, gamma = 0.0, bound = 0.0;
  int t = j.fixed_t, exact = 0;
  if (t <= 0) {
    cert_rho_gamma(words, &rho, &gamma);
    t = cert_mod_bits(rho, gamma, (int)words[kCertTexA], (int)words[kCertTexB], j.k, j.tol, &bound, &exact);
  }
  const int n = t > 62 ? 0
                : j.fixed_t <= 0
                    ? moduli_for_norms(t, j.k, __uint_as_float(j.words[kCertNormA]), __uint_as_float(j.words[kCertNormB]), mp)
                    : moduli_for_products(t, j.k, mp);
  ModPlan pl;
  pl.t = n ? t : 1;
  pl.n = n ? n : 1;
  pl.feasible = n != 0;
  pl.want = t;
  pl.exact = exact;
  pl.pad = 0;
  pl.rho = rho;
  pl.gamma = gamma;
  pl.bound = bound;
  *j.plan = pl;
  if (!n) {
    if (!retry) atomicOr(flags, 1u);
    if (final_pass) atomicOr(flags + 1, 1u);
  } else {
    atomicMax(flags + 2, (unsigned int)n);  // the largest moduli count, for the two-SM products
  }
}

// the column scales alpha 2^(tau_j - 2t) of a grouped launch, one block per problem
__global__ void __launch_bounds__(256) k_mod_colscale_batched(const ColJob* __restrict__ jobs) {
  const ColJob j = jobs[blockIdx.x];
  const ModPlan pl = *j.plan;
  if (!pl.feasible) return;
  for (int64_t c = threadIdx.x; c < j.n; c += blockDim.x) {
    const int tau = j.sigB[c] == kExpEmpty ? 0 : j.sigB[c];
    j.cs[c] = j.badB[c] ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(j.alpha, tau - 2 * pl.t);
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
  ModPlan* plan;
  unsigned int* cert;  // [kCertWords] the certification's maxima and exactness widths
  int* eminA;          // [m] smallest exponent of each row's non-zero entries, then eminB [n]
  int* eminB;
  StatSide st[2];      // automatic mode: the one-pass statistics' tile partials of op(A), op(B)^T
  double* cs;    // [n]
  uint16_t* DA;  // [nmod][m][kp]
  uint16_t* DB;  // [nmod][n][kp]
  uint8_t* park;  // [nbm * nbn][nmod][kParkBlock] the residues of the products
  int nbm, nbn;   // 128-row and 128-column blocks of C
  int park_mods;
  int64_t kp;
};

size_t mod_layout(int64_t m, int64_t n, int64_t k, int nmod, void* base, ModWorkspace* ws) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t kp = (k + 7) / 8 * 8;
  const int64_t nbm = (m + 127) / 128, nbn = (n + 127) / 128;
  size_t off = 0;
  const size_t o_sigA = off; off = up(off + sizeof(int) * (size_t)m);
  const size_t o_sigB = off; off = up(off + sizeof(int) * (size_t)n);
  const size_t o_badA = off; off = up(off + sizeof(int) * (size_t)m);
  const size_t o_badB = off; off = up(off + sizeof(int) * (size_t)n);
  const size_t o_muA = off; off = up(off + sizeof(unsigned long long) * (size_t)m);
  const size_t o_muB = off; off = up(off + sizeof(unsigned long long) * (size_t)n);
  const size_t o_plan = off; off = up(off + sizeof(ModPlan));
  const size_t o_cert = off; off = up(off + sizeof(unsigned int) * kCertWords);
  const size_t o_emin = off; off = up(off + sizeof(int) * (size_t)(m + n));
  const int64_t nkt = (k + 63) / 64;  // 64-wide k tiles of the one-pass statistics
  size_t o_part[2][6];
  for (int side = 0; side < 2; ++side)
    for (int f = 0; f < 6; ++f) {
      o_part[side][f] = off;
      off = up(off + 4 * (size_t)(side == 0 ? m : n) * (size_t)nkt);
    }
  const size_t o_cs = off; off = up(off + sizeof(double) * (size_t)n);
  const size_t o_DA = off; off = up(off + 2 * (size_t)nmod * (size_t)m * (size_t)kp);
  const size_t o_DB = off; off = up(off + 2 * (size_t)nmod * (size_t)n * (size_t)kp);
  const size_t o_park = off; off = up(off + (size_t)kParkBlock * (size_t)nmod * (size_t)(nbm * nbn));
  if (base && ws) {
    char* b = static_cast<char*>(base);
    ws->sigA = reinterpret_cast<int*>(b + o_sigA);
    ws->sigB = reinterpret_cast<int*>(b + o_sigB);
    ws->badA = reinterpret_cast<int*>(b + o_badA);
    ws->badB = reinterpret_cast<int*>(b + o_badB);
    ws->muA = reinterpret_cast<unsigned long long*>(b + o_muA);
    ws->muB = reinterpret_cast<unsigned long long*>(b + o_muB);
    ws->plan = reinterpret_cast<ModPlan*>(b + o_plan);
    ws->cert = reinterpret_cast<unsigned int*>(b + o_cert);
    ws->eminA = reinterpret_cast<int*>(b + o_emin);
    ws->eminB = ws->eminA + m;
    for (int side = 0; side < 2; ++side) {
      StatSide& st = ws->st[side];
      st.e = reinterpret_cast<int*>(b + o_part[side][0]);
      st.b = reinterpret_cast<int*>(b + o_part[side][1]);
      st.lo = reinterpret_cast<int*>(b + o_part[side][2]);
      st.low = reinterpret_cast<int*>(b + o_part[side][3]);
      st.s = reinterpret_cast<float*>(b + o_part[side][4]);
      st.q = reinterpret_cast<float*>(b + o_part[side][5]);
      st.nkt = (int)nkt;
    }
    ws->cs = reinterpret_cast<double*>(b + o_cs);
    ws->DA = reinterpret_cast<uint16_t*>(b + o_DA);
    ws->DB = reinterpret_cast<uint16_t*>(b + o_DB);
    ws->park = reinterpret_cast<uint8_t*>(b + o_park);
    ws->nbm = (int)nbm;
    ws->nbn = (int)nbn;
    ws->park_mods = nmod;
    ws->kp = kp;
  }
  return off;
}

// products of the first n moduli
ModProducts moduli_products() {
  ModProducts mp;
  hu128 M = 1;
  for (int l = 0; l < kMaxModuli; ++l) {
    M *= (hu128)kModuli[l];
    mp.lo[l] = (uint64_t)M;
    mp.hi[l] = (uint64_t)(M >> 64);
  }
  return mp;
}

int moduli_for(int t, int64_t k) { return moduli_for_products(t, k, moduli_products()); }

// the moduli and their Barrett constants; the rest of `a` zeroed
void mod_constants(ModArgs& a) {
  memset(&a, 0, sizeof(a));
  for (int l = 0; l < kMaxModuli; ++l) {
    a.p[l] = kModuli[l];
    a.bar[l] = (uint32_t)((1ull << 32) / (uint64_t)kModuli[l]);
    a.pinv[l] = 1.0f / (float)kModuli[l];
  }
}

// the reconstruction of one product (jobs == nullptr: `one`) or of a grouped launch's jobs
int launch_mod_crt(const CrtJob& one, const CrtJob* jobs, const CrtJob* jobs_host, int count, int64_t total, int sms,
                   cudaStream_t s) {
  if (total <= 0) return GBD_OK;
  const int64_t cap = (int64_t)sms * 8;
  const int grid = (int)(total < cap ? total : cap);
  static thread_local JobBegins begins;  // 15 KB: not on the stack
  begins.n = (jobs && count <= kBeginCache) ? count : 0;
  for (int q = 0; q < begins.n; ++q) begins.b[q] = jobs_host[q].blk_begin;
  k_mod_crt<<<grid, kCrtThreads, 0, s>>>(one, jobs, count, total, begins);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "modular reconstruction launch");
}

// the residue split parameters of every modulus (t and n come from a plan)
void mod_split_params(ModSplit& ms) {
  memset(&ms, 0, sizeof(ms));
  for (int l = 0; l < kMaxModuli; ++l) {
    const int pm = kModuli[l];
    ms.pf[l] = (float)pm;
    ms.inv[l] = 1.0f / (float)pm;
    uint32_t w = 1, lo = 0, hi = 0;  // 256^d mod p
    for (int d = 0; d < 8; ++d) {
      if (d < 4) lo |= (w % (uint32_t)pm) << (8 * d);
      else hi |= (w % (uint32_t)pm) << (8 * (d - 4));
      w = (w * 256u) % (uint32_t)pm;
    }
    ms.wlo[l] = lo;
    ms.whi[l] = hi;
    ms.wbias[l] = 0x4B000000u + ((uint32_t)pm - (8388608u % (uint32_t)pm)) % (uint32_t)pm;
  }
}

// Relative throughput per SM of the two-SM form over the one-SM form when both fill the GPU
constexpr double kModPairGain = 1.2;
// moduli assumed by the kernel choice when the device picks the count (12 at the FP64 bound for
// uniform inputs at k = 8192)
constexpr int kModTypical = 12;

// the product kernel of one call; `a` carries everything but the tile geometry; the residue
// planes hold up to nmod_ws moduli (the plan's n is at most that)
int launch_mod_gemm(int64_t m, int64_t n, int64_t k, int nmod_ws, int bits, ModArgs& a, const ModWorkspace& ws,
                    int sms, cudaStream_t stream) {
  // GBD_EMU_KERNEL=pair|single|split overrides the choice (tests and tuning).  Otherwise the
  // smallest expected time, in units of one 128 x 128 tile with all its moduli on one SM, with
  // whole waves of work units over the SMs (or SM pairs):
  //   single: units are tiles;
  //   split (one-SM, no triangle; at most 8 tiles, or fewer tiles than half the SMs with
  //     k >= 2048): units are (tile, group of moduli), at most 16 groups per tile;
  //   pair: units are (256 x 256 tile, modulus), each four quarter-tiles of one modulus on two
  //     SMs at kModPairGain.
  // The split rule's region is the measured one (256^3: 0.145 against 0.169 ms for single;
  // 256^2 x 4096: 0.25 against 0.47 ms), where it also wins the estimate.
  const char* force = getenv("GBD_EMU_KERNEL");
  const int cta_cap = sms;
  // a triangular output (m = n) covers the tiles that meet its triangle
  auto count = [&](int64_t bm, int64_t bn) {
    const int64_t tm = (m + bm - 1) / bm, tn = (n + bn - 1) / bn;
    return a.tri ? tm * (tm + 1) / 2 : tm * tn;
  };
  const int64_t tiles1 = count(kBM, kBN);
  const int64_t tiles2 = count(k2BM, k2BN);
  const int64_t pairs_avail = cta_cap / 2 > 0 ? cta_cap / 2 : 1;
  const int nm = bits > 0 ? nmod_ws : kModTypical;
  auto waves = [](int64_t units, int64_t slots) { return (double)((units + slots - 1) / slots); };
  const double t_one = waves(tiles1, cta_cap);
  int64_t groups = (cta_cap + tiles1 - 1) / tiles1;  // the kernel keeps at most nmod of them
  if (groups > kMaxModuli) groups = kMaxModuli;
  const int64_t g_eff = groups < nm ? groups : nm;
  const double t_split = waves(tiles1 * g_eff, cta_cap) * (double)((nm + g_eff - 1) / g_eff) / nm;
  const double t_pair = waves(tiles2 * nm, pairs_avail) * 2.0 / (kModPairGain * nm);
  const bool split_ok = a.tri == 0 && (tiles1 <= 8 || (2 * tiles1 < sms && k >= 2048));
  char choice = 's';  // single
  if (force && (force[0] == 'p' || force[0] == 's')) {
    choice = strcmp(force, "split") == 0 ? 'x' : force[0];
  } else if (split_ok && t_split <= t_pair && t_split <= t_one) {
    choice = 'x';
  } else if (t_pair < t_one) {
    choice = 'p';
  }
  if (choice == 'x' && a.tri != 0) choice = 's';
  if (choice == 'p' && cta_cap < 2) choice = 's';
  const bool pair = choice == 'p';
  const uint32_t brows = pair ? 128u : (uint32_t)kBM;  // rows of A (and of op(B)^T) one CTA stages
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, (uint64_t)nmod_ws};
  const uint64_t pA[2] = {(uint64_t)ws.kp * 2, (uint64_t)m * ws.kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, brows, 1u};
  int rc = encode_tmap(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, (uint64_t)nmod_ws};
  const uint64_t pB[2] = {(uint64_t)ws.kp * 2, (uint64_t)n * ws.kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, brows, 1u};
  rc = encode_tmap(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  a.nkb = (int)((k + kBK - 1) / kBK);
  const int tbm = pair ? k2BM : kBM, tbn = pair ? k2BN : kBN;
  a.tiles_m = (int)((m + tbm - 1) / tbm);
  const int64_t tiles = count(tbm, tbn);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  cudaError_t e;
  if (choice == 'x') {
    a.groups = (int)groups;
    a.group_m = 1;
    const int64_t units = tiles * groups;
    const int grid = (int)(units < sms ? units : sms);
    e = cudaFuncSetAttribute(k_mod_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm split)");
    k_mod_gemm<true><<<grid, kThreads, Smem::kAlloc, stream>>>(a, tmA, tmB);
  } else if (pair) {
    // (tile, modulus) units, at most nmod_ws per tile; pairs left without one return at once
    const int64_t units = tiles * nmod_ws;
    if (units >= ((int64_t)1 << 31)) return set_error(GBD_ERR_LIMIT, "too many output tiles");
    const int64_t pairs = units < pairs_avail ? units : pairs_avail;
    // GBD_EMU_GROUP_M sets the rows of tiles per raster group (tuning); by default about the
    // square root of the pairs' concurrent tiles
    const char* gm_env = getenv("GBD_EMU_GROUP_M");
    const int gm_set = gm_env ? atoi(gm_env) : 0;
    a.group_m = gm_set > 0 ? (gm_set < a.tiles_m ? gm_set : a.tiles_m) : group_rows((int)pairs, k2BM, k2BN, a.tiles_m);
    // one exact FP32 chunk per modulus (k <= 1024): its own instance, so that the int32 path of
    // deeper products keeps its registers
    auto kern = a.nkb <= kChunkBlocks ? k_mod_gemm_pair<false, 1> : k_mod_gemm_pair<false, 0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm pair)");
    kern<<<(unsigned)(2 * pairs), k2Threads, Smem2::kAlloc, stream>>>(a, tmA, tmB, nullptr, 0, nullptr);
  } else {
    const int grid = (int)(tiles < cta_cap ? tiles : cta_cap);
    a.group_m = group_rows(grid, kBM, kBN, a.tiles_m);
    e = cudaFuncSetAttribute(k_mod_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm)");
    k_mod_gemm<false><<<grid, kThreads, Smem::kAlloc, stream>>>(a, tmA, tmB);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "modular gemm launch");
}

}  // namespace
}  // namespace emu
}  // namespace gbd

namespace gbd {
namespace emu {

// gbd_dgemm_emu_mod, and the triangular-output form of DSYRK (tri = 1 lower, 2 upper; m = n,
// alpha != 0, k > 0): only the elements of C on that triangle are read and written
int dgemm_emu_mod_impl(char transa, char transb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int bits,
                       double tol, void* workspace, size_t workspace_bytes, gbd_emu_info* info, void* stream,
                       int tri) {
  int rc = check_dgemm_args(transa, transb, m, n, k, lda, ldb, ldc);
  if (rc) return rc;
  if (info) {
    const int rp = info->record_phases;
    memset(info, 0, sizeof(*info));
    info->record_phases = rp;
  }
  if (bits < -1 || bits > 62)
    return set_error(GBD_ERR_ARG, "dgemm_emu_mod: bits must be -1 or 0 (automatic) or 1..62");
  if (m == 0 || n == 0) return GBD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (tri && (m != n || alpha == 0.0 || k == 0))
    return set_error(GBD_ERR_ARG, "dgemm_emu_mod: a triangular output needs m = n, alpha != 0 and k > 0");
  if (alpha == 0.0 || k == 0) return scale_c(m, n, beta, C, ldc, s);
  const int64_t lim = (int64_t)1 << 31;
  if (m >= lim || n >= lim || k >= lim)
    return set_error(GBD_ERR_LIMIT, "dgemm_emu_mod: m, n and k below 2^31 are supported");
  int sms = 0;
  if ((rc = current_device(nullptr, &sms))) return rc;
  const ModProducts prods = moduli_products();
  int nmod_ws = kMaxModuli;
  if (bits > 0) {
    nmod_ws = moduli_for_products(bits, k, prods);
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
  const bool timing = info && info->record_phases;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  struct EventGuard {
    cudaEvent_t* e;
    ~EventGuard() {
      for (int i = 0; i < 4; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  cudaError_t e;
  if (timing) {
    for (int i = 0; i < 4; ++i)
      if ((e = cudaEventCreate(&ev[i])) != cudaSuccess) return cuda_fail(e, "dgemm_emu_mod: cudaEventCreate");
    if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu_mod: cudaEventRecord");
  }
  const int ta = (transa == 'N' || transa == 'n') ? 0 : 1, tb = (transb == 'N' || transb == 'n') ? 0 : 1;
  const bool automatic = bits <= 0;

  // exponents (and, in automatic mode, the magnitude statistics) of both sides
  PrepPair pp;
  memset(&pp, 0, sizeof(pp));
  PrepJob& ja = pp.j[0];
  PrepJob& jb = pp.j[1];
  ja.X = A; ja.ld = lda; ja.R = m; ja.K = k; ja.rows_contig = ta == 0;
  ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = automatic ? ws.muA : nullptr; ja.D = ws.DA; ja.kp = ws.kp;
  jb.X = B; jb.ld = ldb; jb.R = n; jb.K = k; jb.rows_contig = tb != 0;
  jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = automatic ? ws.muB : nullptr; jb.D = ws.DB; jb.kp = ws.kp;
  ja.emin = automatic ? ws.eminA : nullptr;
  jb.emin = automatic ? ws.eminB : nullptr;
  ja.st = ws.st[0];
  jb.st = ws.st[1];
  int64_t exp_blocks = 0, split_blocks = 0;
  prep_pair_blocks(pp, exp_blocks, split_blocks);
  const int prec = cert_prec_default();
  if (automatic) {
    // one pass over the operands: exponents, flags, magnitude and square sums, exactness widths,
    // and the FP8 magnitude planes (in the residue planes' place, which are written after the
    // plan); then the certification product with the reduction of the bound's ratios
    if ((e = cudaMemsetAsync(ws.cert, 0, sizeof(unsigned int) * kCertWords, s)) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu_mod: clearing the certification words");
    if ((rc = launch_statplane_pair(pp, split_blocks, ws.cert + kCertTexA, ws.cert + kCertNormA, s))) return rc;
    if (prec == kCertBF16 && (rc = launch_magplane_pair(pp, prec, ws.cert + kCertTexA, split_blocks, s))) return rc;
    if ((rc = launch_cert(m, n, k, prec, ws.DA, ws.DB, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB, ws.eminA,
                          ws.eminB, ws.cert, nullptr, 0, sms, s)))
      return rc;
  } else if ((rc = launch_exponents_pair(pp, exp_blocks, nullptr, 0, s))) {
    return rc;
  }
  // the plan: t and n, on the device; after FP8 planes, a plan that finds no feasible t is made
  // again from a BF16 certification (its kernels return at once when the first plan is feasible)
  const double target = tol > 0.0 ? tol : 2.0 * (double)k * kUnitRoundoff;
  const bool retry = automatic && prec == kCertFP8;
  k_mod_plan<<<1, 32, 0, s>>>(ws.cert, k, target, automatic ? 0 : bits, prods, ws.plan, device_error_word(),
                              (bits == -1 && !retry) ? 1 : 0, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "plan launch");
  if (retry) {
    if ((rc = launch_magplane_pair(pp, kCertBF16, ws.cert + kCertRetry + kCertTexA, split_blocks, s, ws.plan)))
      return rc;
    if ((rc = launch_cert(m, n, k, kCertBF16, ws.DA, ws.DB, ws.muA, ws.muB, ws.badA, ws.badB, ws.sigA, ws.sigB,
                          ws.eminA, ws.eminB, ws.cert + kCertRetry, nullptr, 0, sms, s, ws.plan)))
      return rc;
    k_mod_plan<<<1, 32, 0, s>>>(ws.cert, k, target, 0, prods, ws.plan, device_error_word(), bits == -1 ? 1 : 0, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "plan launch");
  }
  ModPlan host_plan;
  memset(&host_plan, 0, sizeof(host_plan));
  if (bits == 0) {  // read the plan back: an unreachable target is refused before C is touched
    if ((e = cudaMemcpyAsync(&host_plan, ws.plan, sizeof(host_plan), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu_mod: reading the plan");
    if (!host_plan.feasible)
      return set_error(GBD_ERR_LIMIT,
                       "dgemm_emu_mod: the accuracy target cannot be certified within %d moduli at k = %lld (%s; "
                       "gbd_dgemm_emu covers every target)",
                       kMaxModuli, (long long)k,
                       host_plan.want > 62 ? "no bit count up to 62 meets it" : "too many bits");
  }

  // residues of both sides (the first n of the kMaxModuli, t bits, from the plan)
  ModSplit ms;
  mod_split_params(ms);
  ms.plan = ws.plan;
  if ((rc = launch_residue_pair(pp, ms, split_blocks, s))) return rc;
  k_mod_colscale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ws.sigB, ws.badB, n, alpha, ws.plan, ws.cs);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "column scale launch");

  // products modulo each modulus, parked; then the reconstruction of C
  ModArgs a;
  mod_constants(a);
  a.tri = tri;
  a.m = m;
  a.n = n;
  a.plan = ws.plan;
  a.park = ws.park;
  a.park_mods = ws.park_mods;
  a.nbn = ws.nbn;
  a.err = device_error_word();
  if (timing && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu_mod: cudaEventRecord");
  if ((rc = launch_mod_gemm(m, n, k, nmod_ws, bits, a, ws, sms, s))) return rc;
  if (timing && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu_mod: cudaEventRecord");
  CrtJob job;
  memset(&job, 0, sizeof(job));
  job.park = ws.park;
  job.plan = ws.plan;
  job.C = C;
  job.sigA = ws.sigA;
  job.badA = ws.badA;
  job.cs = ws.cs;
  job.m = m;
  job.n = n;
  job.ldc = ldc;
  job.beta = beta;
  job.park_mods = ws.park_mods;
  job.nbm = ws.nbm;
  job.nbn = ws.nbn;
  job.tri = tri;
  if ((rc = launch_mod_crt(job, nullptr, nullptr, 0, (int64_t)ws.nbm * ws.nbn, sms, s))) return rc;
  if (timing) {
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    if ((e = cudaEventRecord(ev[3], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[3])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t0, ev[0], ev[1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t1, ev[1], ev[2])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t2, ev[2], ev[3])) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu_mod: phase timing");
    info->prep_ms = t0;
    info->gemm_ms = t1;
    info->recon_ms = t2;
  }
  if (info) {
    if (bits > 0) {
      host_plan.t = bits;
      host_plan.n = nmod_ws;
    } else if (bits == -1) {  // the device-side choice: read it back (this synchronises `stream`)
      if ((e = cudaMemcpyAsync(&host_plan, ws.plan, sizeof(host_plan), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "dgemm_emu_mod: reading the plan");
    }
    info->path = GBD_PATH_MODULAR;
    info->slices = host_plan.n;
    info->digit_bits = host_plan.t;
    info->products = host_plan.n;
    info->exact = host_plan.exact;
    info->rho = host_plan.rho;
    info->gamma = host_plan.gamma;
    info->bound = host_plan.bound;
  }
  return GBD_OK;
}

// ---- grouped modular problems ----
namespace {
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// GBD_EMU_KERNEL=single keeps every grouped modular problem on the one-SM kernel (tests and tuning)
bool mod_grouped_pairs_enabled() {
  const char* force = getenv("GBD_EMU_KERNEL");
  return !(force && strcmp(force, "single") == 0);
}
// A problem whose products run on CTA pairs: at least 256 on every side, so that a 256 x 256 tile
// pads little, and a k that keeps the tensor pipe busy while the epilogue drains a unit
bool mod_grouped_pair_problem(const gbd_problem& p) { return p.m >= 256 && p.n >= 256 && p.k >= 256; }
}  // namespace

size_t mod_grouped_layout(const gbd_problem* probs, const int* which, int count, void* base, ModGrouped* g, int* rc) {
  *rc = GBD_OK;
  char* b = static_cast<char*>(base);
  size_t off = 0;
  const size_t o_jobs = off; off = up256(off + sizeof(PrepJob) * 2 * (size_t)count);
  const size_t o_cert = off; off = up256(off + sizeof(CertTableEntry) * 2 * (size_t)count);  // FP8, BF16 retry
  const size_t o_plj = off; off = up256(off + sizeof(ModPlanJob) * (size_t)count);
  const size_t o_col = off; off = up256(off + sizeof(ColJob) * (size_t)count);
  const size_t o_tab = off; off = up256(off + sizeof(ModTableEntry) * (size_t)count);
  const size_t o_crt = off; off = up256(off + sizeof(CrtJob) * (size_t)count);
  const size_t o_words = off; off = up256(off + sizeof(unsigned int) * kCertWords * (size_t)(count + 1));
  std::vector<size_t> o_ws(count);
  std::vector<int> nmod_ws(count);
  for (int q = 0; q < count; ++q) {
    const gbd_problem& p = probs[which[q]];
    int nm = kMaxModuli;
    if (p.slices > 0) {
      nm = moduli_for(p.slices, p.k);
      if (nm == 0) {
        *rc = set_error(GBD_ERR_LIMIT, "grouped problem %d: %d bits need more than %d moduli at k = %lld", which[q],
                        p.slices, kMaxModuli, (long long)p.k);
        nm = kMaxModuli;
      }
    }
    nmod_ws[q] = nm;
    o_ws[q] = off;
    off = up256(off + mod_layout(p.m, p.n, p.k, nm, nullptr, nullptr));
  }
  if (!base || !g || *rc) return off;

  g->count = count;
  g->index.assign(which, which + count);
  g->jobs_dev = reinterpret_cast<PrepJob*>(b + o_jobs);
  g->cert_dev = reinterpret_cast<CertTableEntry*>(b + o_cert);
  g->planjobs_dev = reinterpret_cast<ModPlanJob*>(b + o_plj);
  g->coljobs_dev = reinterpret_cast<ColJob*>(b + o_col);
  g->table_dev = reinterpret_cast<ModTableEntry*>(b + o_tab);
  g->words_dev = reinterpret_cast<unsigned int*>(b + o_words);
  g->flags_dev = g->words_dev + (size_t)kCertWords * count;
  g->crt_dev = reinterpret_cast<CrtJob*>(b + o_crt);
  g->jobs.assign(2 * (size_t)count, PrepJob{});
  g->cert.assign(2 * (size_t)count, CertTableEntry{});
  g->planjobs.assign(count, ModPlanJob{});
  g->coljobs.assign(count, ColJob{});
  g->plans.assign(count, nullptr);
  std::vector<ModWorkspace> ws(count);
  g->exp_blocks = 0;
  g->split_blocks = 0;
  int64_t cert_tiles = 0;
  for (int q = 0; q < count; ++q) {
    const gbd_problem& p = probs[which[q]];
    mod_layout(p.m, p.n, p.k, nmod_ws[q], b + o_ws[q], &ws[q]);
    const ModWorkspace& w = ws[q];
    unsigned int* words = g->words_dev + (size_t)kCertWords * q;
    PrepJob& ja = g->jobs[2 * q];
    PrepJob& jb = g->jobs[2 * q + 1];
    // op(A) rows: A[p*lda + i] when 'N' (rows contiguous); op(B)^T rows: B[p*ldb + j] when 'T'
    ja.X = p.A; ja.ld = p.lda; ja.R = p.m; ja.K = p.k; ja.rows_contig = trans_code(p.transa) == 0;
    ja.sig = w.sigA; ja.bad = w.badA; ja.mu = w.muA; ja.D = w.DA; ja.kp = w.kp;
    ja.tex = words + kCertTexA; ja.plan = w.plan; ja.emin = w.eminA; ja.norm = words + kCertNormA; ja.st = w.st[0];
    jb.X = p.B; jb.ld = p.ldb; jb.R = p.n; jb.K = p.k; jb.rows_contig = trans_code(p.transb) != 0;
    jb.sig = w.sigB; jb.bad = w.badB; jb.mu = w.muB; jb.D = w.DB; jb.kp = w.kp;
    jb.tex = words + kCertTexB; jb.plan = w.plan; jb.emin = w.eminB; jb.norm = words + kCertNormB; jb.st = w.st[1];
    prep_job_blocks(ja, g->exp_blocks, g->split_blocks);
    prep_job_blocks(jb, g->exp_blocks, g->split_blocks);
    CertTableEntry& ce = g->cert[q];
    if ((*rc = make_cert_entry(p.m, p.n, p.k, cert_prec_default(), w.DA, w.DB, w.muA, w.muB, w.badA, w.badB, w.sigA, w.sigB,
                               w.eminA, w.eminB, words, nullptr, &ce)))
      return off;
    CertTableEntry& cr = g->cert[count + q];  // the BF16 retry, for a plan that found no feasible t
    if ((*rc = make_cert_entry(p.m, p.n, p.k, kCertBF16, w.DA, w.DB, w.muA, w.muB, w.badA, w.badB, w.sigA, w.sigB,
                               w.eminA, w.eminB, words + kCertRetry, w.plan, &cr)))
      return off;
    ce.tile_begin = cr.tile_begin = cert_tiles;
    cert_tiles += ce.a.num_tiles;
    ModPlanJob& pj = g->planjobs[q];
    pj.words = words;
    pj.plan = w.plan;
    pj.k = p.k;
    pj.tol = p.tol > 0.0 ? p.tol : 2.0 * (double)p.k * kUnitRoundoff;
    pj.fixed_t = p.slices > 0 ? p.slices : 0;
    ColJob& cj = g->coljobs[q];
    cj.sigB = w.sigB;
    cj.badB = w.badB;
    cj.cs = w.cs;
    cj.plan = w.plan;
    cj.alpha = p.alpha;
    cj.n = p.n;
    g->plans[q] = w.plan;
  }
  g->cert_tiles = (int)cert_tiles;
  // the product table: first the problems for the two-SM kernel, then those for the one-SM
  // kernel, each part with the deepest problems' tiles first (longest tiles first over the SMs)
  std::vector<int> order(count);
  for (int q = 0; q < count; ++q) order[q] = q;
  const bool pairs_on = mod_grouped_pairs_enabled();
  auto on_pair = [&](int q) {
    const gbd_problem& p = probs[which[q]];
    return pairs_on && p.tile != 128 && mod_grouped_pair_problem(p);  // tile 128: single SMs only
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const bool px = on_pair(x), py = on_pair(y);
    if (px != py) return px;
    return probs[which[x]].k > probs[which[y]].k;
  });
  g->table.assign(count, ModTableEntry{});
  g->crt.assign(count, CrtJob{});
  g->pair_count = 0;
  int64_t mt = 0, pt = 0, blocks = 0;
  for (int r = 0; r < count; ++r) {
    const int q = order[r];
    const gbd_problem& p = probs[which[q]];
    const bool pair = on_pair(q);
    if (pair) g->pair_count = r + 1;
    const ModWorkspace& w = ws[q];
    ModTableEntry& e = g->table[r];
    const uint64_t dA[3] = {(uint64_t)p.k, (uint64_t)p.m, (uint64_t)nmod_ws[q]};
    const uint64_t pA[2] = {(uint64_t)w.kp * 2, (uint64_t)p.m * w.kp * 2};
    const uint32_t bA[3] = {(uint32_t)kBK, (uint32_t)kBM, 1u};
    if ((*rc = encode_tmap(&e.tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, w.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B)))
      return off;
    const uint64_t dB[3] = {(uint64_t)p.k, (uint64_t)p.n, (uint64_t)nmod_ws[q]};
    const uint64_t pB[2] = {(uint64_t)w.kp * 2, (uint64_t)p.n * w.kp * 2};
    const uint32_t bB[3] = {(uint32_t)kBK, (uint32_t)kBN, 1u};
    if ((*rc = encode_tmap(&e.tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, w.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B)))
      return off;
    e.m = p.m;
    e.n = p.n;
    e.plan = w.plan;
    e.park = w.park;
    e.park_mods = w.park_mods;
    e.nbn = w.nbn;
    e.nkb = (int)((p.k + kBK - 1) / kBK);
    const int tbm = pair ? k2BM : kBM, tbn = pair ? k2BN : kBN;  // the maps' boxes (128 rows) serve both
    e.tiles_m = (int)((p.m + tbm - 1) / tbm);
    e.num_tiles = e.tiles_m * (int)((p.n + tbn - 1) / tbn);
    e.group_m = e.tiles_m;  // within one problem the tiles walk down the rows
    int64_t& tiles = pair ? pt : mt;
    e.tile_begin = tiles;
    tiles += e.num_tiles;
    CrtJob& cj = g->crt[r];
    cj.park = w.park;
    cj.plan = w.plan;
    cj.C = p.C;
    cj.sigA = w.sigA;
    cj.badA = w.badA;
    cj.cs = w.cs;
    cj.m = p.m;
    cj.n = p.n;
    cj.ldc = p.ldc;
    cj.beta = p.beta;
    cj.blk_begin = blocks;
    cj.park_mods = w.park_mods;
    cj.nbm = w.nbm;
    cj.nbn = w.nbn;
    cj.tri = 0;
    cj.skip_infeasible = 1;
    blocks += (int64_t)w.nbm * w.nbn;
  }
  g->mod_tiles = (int)mt;
  g->pair_tiles = (int)pt;
  g->crt_blocks = blocks;
  if (mt > ((int64_t)1 << 30) || pt * kMaxModuli >= ((int64_t)1 << 31) || cert_tiles > ((int64_t)1 << 30))
    *rc = set_error(GBD_ERR_LIMIT, "grouped: too many tiles");
  return off;
}

int mod_grouped_run(const ModGrouped& g, int sms, cudaStream_t s) {
  if (g.count == 0) return GBD_OK;
  cudaError_t e;
  int rc;
  const int njobs = (int)g.jobs.size();
  if ((e = cudaMemsetAsync(g.words_dev, 0, sizeof(unsigned int) * kCertWords * (size_t)(g.count + 1), s)) !=
      cudaSuccess)
    return cuda_fail(e, "grouped modular: clearing the certification words");
  // one pass over every side: statistics and FP8 magnitude planes (as the single call)
  int64_t max_rows = 0;
  for (const PrepJob& j : g.jobs) max_rows = j.R > max_rows ? j.R : max_rows;
  if ((rc = launch_statplane_batched(g.jobs_dev, g.jobs.data(), njobs, g.split_blocks, max_rows, s))) return rc;
  // the certification: magnitude planes, their products, the plans (the same precision as the
  // single call's, so that a problem gets the same plan alone and in a batch)
  const int prec = cert_prec_default();
  const bool retry = prec == kCertFP8;
  if (prec == kCertBF16 && (rc = launch_magplane_batched(g.jobs_dev, g.jobs.data(), njobs, g.split_blocks, s, prec))) return rc;
  if ((rc = launch_cert_grouped(g.cert_dev, g.count, g.cert_tiles, prec, sms, s))) return rc;
  const ModProducts prods = moduli_products();
  k_mod_plan_batched<<<(g.count + 127) / 128, 128, 0, s>>>(g.planjobs_dev, g.count, prods, 0, g.flags_dev,
                                                           retry ? 0 : 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped plan launch");
  if (retry) {
    // the BF16 retry of every problem whose plan found no feasible t; the launches return at once
    // when no problem needs it, and skip the problems whose plan is feasible
    if ((rc = launch_magplane_batched(g.jobs_dev, g.jobs.data(), njobs, g.split_blocks, s, kCertBF16, g.flags_dev))) return rc;
    if ((rc = launch_cert_grouped(g.cert_dev + g.count, g.count, g.cert_tiles, kCertBF16, sms, s, g.flags_dev)))
      return rc;
    k_mod_plan_batched<<<(g.count + 127) / 128, 128, 0, s>>>(g.planjobs_dev, g.count, prods, 1, g.flags_dev, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped plan launch");
  }
  // residues and column scales with each problem's plan
  ModSplit ms;
  mod_split_params(ms);
  if ((rc = launch_residue_batched(g.jobs_dev, g.jobs.data(), njobs, ms, g.split_blocks, s))) return rc;
  k_mod_colscale_batched<<<g.count, 256, 0, s>>>(g.coljobs_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped column scale launch");
  // the products of every feasible problem: the large problems' (256 x 256 tile, modulus) units
  // on CTA pairs, then the other problems' tiles on single SMs, each a persistent launch
  ModArgs a;
  mod_constants(a);
  a.plan = g.plans[0];  // read at kernel start; the tiles use their own problems' plans
  a.err = device_error_word();
  a.tiles_m = 1;
  a.group_m = 1;
  a.nkb = 1;
  a.groups = 1;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  if (g.pair_tiles > 0) {
    a.num_tiles = g.pair_tiles;
    const int64_t pairs_avail = sms / 2 > 0 ? sms / 2 : 1;
    const int64_t units = (int64_t)g.pair_tiles * kMaxModuli;  // at most; the plans' largest count bounds them
    const int64_t pairs = units < pairs_avail ? units : pairs_avail;
    e = cudaFuncSetAttribute(k_mod_gemm_pair<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped modular gemm pair)");
    k_mod_gemm_pair<true, 2><<<(unsigned)(2 * pairs), k2Threads, Smem2::kAlloc, s>>>(a, dummy, dummy, g.table_dev,
                                                                                  g.pair_count, g.flags_dev + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped modular gemm pair launch");
  }
  if (g.mod_tiles <= 0) return GBD_OK;
  a.num_tiles = g.mod_tiles;
  const int grid = g.mod_tiles < sms ? g.mod_tiles : sms;
  e = cudaFuncSetAttribute(k_mod_gemm<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped modular gemm)");
  k_mod_gemm<false, true><<<grid, kThreads, Smem::kAlloc, s>>>(a, dummy, dummy, g.table_dev + g.pair_count,
                                                               g.count - g.pair_count);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped modular gemm launch");
  // the reconstruction of every feasible problem
  CrtJob none;
  memset(&none, 0, sizeof(none));
  return launch_mod_crt(none, g.crt_dev, g.crt.data(), g.count, g.crt_blocks, sms, s);
}

}  // namespace emu
}  // namespace gbd

namespace gbd {

int dgemm_emu_mod_tri(char transa, char transb, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int upper, double tol,
                      void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  return emu::dgemm_emu_mod_impl(transa, transb, n, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, tol, workspace,
                                 workspace_bytes, nullptr, stream, upper ? 2 : 1);
}

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
  return gbd::emu::dgemm_emu_mod_impl(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, bits, tol,
                                      workspace, workspace_bytes, info, stream, 0);
}

}  // extern "C"
