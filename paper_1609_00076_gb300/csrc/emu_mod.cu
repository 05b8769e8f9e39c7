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
// parked residue bytes: per CTA two slots (the tile being multiplied and the one being
// reconstructed) of [modulus][column / 4][128 rows][4 columns] bytes, sized for the widest tile:
// a thread moves four columns in one 32-bit word and a warp 128 contiguous bytes
constexpr int kSlotCols = 256;
constexpr int64_t kLStride = (int64_t)kSlotCols * 128;
constexpr int64_t kSlotBytes = (int64_t)kMaxModuli * kLStride;
constexpr int kMaxModCtas = 256;
// few-tile problems split each 128 x 128 tile's moduli over several CTAs (at most this many tiles)
constexpr int kSplitMaxTiles = 64;
constexpr int64_t kTileSlotBytes = (int64_t)kMaxModuli * (128 / 4) * 128 * 4;  // one tile's parked bytes

// the reconstruction constants of the first n moduli (M = p_0 ... p_(n-1))
struct CrtSet {
  int c[kMaxModuli];            // (M/p_l)^-1 mod p_l
  uint32_t mpl[kMaxModuli][4];  // M/p_l in 32-bit limbs, least significant first
  uint64_t M_lo, M_hi, half_lo, half_hi;  // M and floor(M/2)
};

struct ModArgs {
  int64_t m, n, ldc;
  int nkb;
  int tiles_m, num_tiles, group_m;
  int tile_end;  // the two-SM form computes tiles [0, tile_end) of its num_tiles
  int tri;       // 0: all of C; 1: only its lower triangle (i >= j), 2: its upper one (m = n): the
                 // tiles are those that meet the triangle, and elements outside it are neither
                 // read nor written
  // a one-SM launch over the tail of a two-SM raster (tail_from >= 0): its tile u is quadrant
  // u % 4 of the 256 x 256 tile tail_from + u / 4 of that raster (tail_tiles_m, tail_group_m,
  // tail_num as tiles_m, group_m and num_tiles of the two-SM launch)
  int tail_from, tail_tiles_m, tail_group_m, tail_num;
  int p[kMaxModuli];         // moduli
  uint32_t bar[kMaxModuli];  // floor(2^32 / p_l), for Barrett reduction
  uint32_t rq[kMaxModuli];   // ceil(2^24 / p_l)
  CrtSet set[kMaxModuli];    // set[n - 1]: the constants for the first n moduli
  const ModPlan* plan;       // the call's n (and whether the target was reachable)
  double beta;
  double* C;
  const int* sigA;
  const int* badA;
  const double* cs;  // [n] alpha 2^(tau_j - 2t); NaN for a column with a non-finite entry
  uint8_t* scr;      // [CTA][2][kMaxModuli][kSlotCols / 4][128][4] parked u_l
  // split over moduli (one-SM form, few tiles): each tile's moduli in `groups` work units
  int groups;
  uint8_t* tslot;            // [tile][kMaxModuli][kBN / 4][128][4] parked u_l of every unit of the tile
  unsigned int* tile_done;   // [tile] finished units (zero at launch)
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
  if (p.tail_from < 0) {
    raster_coords(p.tri, tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
    return;
  }
  int tm2, tn2;
  raster_coords(p.tri, p.tail_from + tile / 4, p.tail_tiles_m, p.tail_group_m, p.tail_num, tm2, tn2);
  tm = 2 * tm2 + (tile & 1);
  tn = 2 * tn2 + ((tile >> 1) & 1);
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

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 make_u128(uint64_t hi, uint64_t lo) { return ((u128)hi << 64) | lo; }

// C' from its parked bytes u_l = (C' mod p_l) c_l mod p_l: sum_l u_l (M/p_l) = (C' mod M) + q M
// with q = floor(sum_l u_l / p_l).  Returns the representative of (-M/2, M/2] in two's
// complement 128 bits.
__device__ __forceinline__ u128 crt_combine(const uint32_t (&u)[kMaxModuli], const ModArgs& p, const CrtSet& cs,
                                            int nmod) {
  uint64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // limb sums, each below 16 * 255 * 2^32 < 2^44
  uint32_t qfix = 0;                         // sum_l u_l ceil(2^24/p_l) < 2^29
#pragma unroll
  for (int l = 0; l < kMaxModuli; ++l) {
    if (l < nmod) {
      a0 += (uint64_t)u[l] * cs.mpl[l][0];
      a1 += (uint64_t)u[l] * cs.mpl[l][1];
      a2 += (uint64_t)u[l] * cs.mpl[l][2];
      a3 += (uint64_t)u[l] * cs.mpl[l][3];
      qfix += u[l] * p.rq[l];
    }
  }
  const u128 s = (u128)a0 + ((u128)a1 << 32) + ((u128)a2 << 64) + ((u128)a3 << 96);  // modulo 2^128
  // qfix / 2^24 exceeds sum_l u_l/p_l by less than 16 * 255 / 2^24, so its floor is q or q + 1
  const u128 M = make_u128(cs.M_hi, cs.M_lo);
  u128 cu = s - (u128)(qfix >> 24) * M;
  if ((uint64_t)(cu >> 127)) cu += M;  // the estimate was one too large
  else if (cu >= M) cu -= M;
  const u128 half = make_u128(cs.half_hi, cs.half_lo);
  return cu > half ? cu - M : cu;
}

// fl(v) 2^sig for a two's complement 128-bit v: fl rounds to nearest (ties to even); the
// scaling rounds again only where the result leaves the normal range (as ldexp).  The common
// case builds the double from integers.
__device__ __forceinline__ double scaled_double(u128 v, int sig) {
  const bool neg = (uint64_t)(v >> 127) != 0;
  const u128 a = neg ? (u128)0 - v : v;
  const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
  if ((hi | lo) == 0ull) return 0.0;
  const int nbits = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  uint64_t mant = lo;
  int e = 0;
  if (nbits > 53) {
    const int shift = nbits - 53;
    mant = (uint64_t)(a >> shift);
    const u128 rem = a & (((u128)1 << shift) - 1), hf = (u128)1 << (shift - 1);
    e = shift;
    if (rem > hf || (rem == hf && (mant & 1ull))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++e;
      }
    }
  }
  // |v| rounded = mant 2^e with mant < 2^53
  const int L = 64 - __clzll((long long)mant);
  const int E = e + sig + L - 1;  // exponent of the scaled value
  if (E >= -1022 && E <= 1023) {
    const uint64_t bits = ((uint64_t)(E + 1023) << 52) | ((mant << (53 - L)) & 0xFFFFFFFFFFFFFull) |
                          (neg ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
  }
  const double y = ldexp(ldexp((double)mant, e), sig);  // the first ldexp is exact
  return neg ? -y : y;
}

// The epilogue of both product kernels.  Each thread owns one TMEM lane (a row of the CTA's
// 128) and COLS columns of the TBN-wide tile.  Per modulus: drain the chunks into int32 sums,
// park u_l; at each modulus boundary (sums dead), reconstruct a few groups of four columns of
// the previous tile from its parked bytes and write them to C.  All loads of a group are
// issued before its arithmetic, so a group waits for memory once.  nan_out: the plan found the
// target unreachable; every result is NaN.
// TABLE: the tiles belong to the problems of a grouped launch (table entries in tile order); each
// tile takes its problem's sizes, C, scales and moduli count from its entry, and a tile whose
// problem's plan is infeasible is skipped (another kernel computes that problem).
template <int EPI_WARPS, int TBN, bool PAIR, bool TABLE = false>
__device__ __forceinline__ void mod_epilogue(const ModArgs& p, int nmod, bool nan_out, uint32_t tmem_base,
                                             uint64_t* acc_full, uint64_t* acc_empty, int warp, int lane, int tile0,
                                             int tile_step, int tbm, int row_off,
                                             const ModTableEntry* table = nullptr, int count = 0) {
  const CrtSet* cset = &p.set[nmod - 1];
  constexpr int COLS = TBN / (EPI_WARPS / 4);
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
  uint8_t* const scr_cta = p.scr + (int64_t)blockIdx.x * 2 * kSlotBytes + (int64_t)(col0 / 4) * 512 + row * 4;
  constexpr int kGroups = COLS / 4;
  int per_boundary = (kGroups + nmod - 1) / nmod;  // groups of four columns

  // the pending reconstruction: this thread's row and columns of the previous tile
  bool pd_active = false, pd_bad = false;
  int pd_done = 0, pd_slot = 0, pd_sig = 0, pd_cols = 0, pd_first = 0;  // columns [pd_first, pd_cols) are written
  double* pd_c = nullptr;
  const double* pd_cs = nullptr;
  // grouped: the pending tile's problem (its moduli, beta and leading dimension)
  int pd_nmod = nmod;
  const CrtSet* pd_cset = cset;
  double pd_beta = p.beta;
  int64_t pd_ldc = p.ldc;
  auto advance = [&](int ngroups) {
    const int g1 = min(pd_done + ngroups, kGroups);
    const uint8_t* ub = scr_cta + (int64_t)pd_slot * kSlotBytes;
    for (int g = pd_done; g < g1; ++g) {
      const int c0 = 4 * g;
      if (c0 >= pd_cols) break;
      if (c0 + 4 <= pd_first) continue;
      const int nm = TABLE ? pd_nmod : nmod;
      const double beta = TABLE ? pd_beta : p.beta;
      const int64_t ldc = TABLE ? pd_ldc : p.ldc;
      uint32_t w4[kMaxModuli];  // the bytes of columns c0..c0+3, one word per modulus
#pragma unroll
      for (int l = 0; l < kMaxModuli; ++l)
        w4[l] = l < nm ? *reinterpret_cast<const uint32_t*>(ub + l * kLStride + g * 512) : 0u;
      double c0v[4], csv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool in = c0 + q < pd_cols && c0 + q >= pd_first;
        c0v[q] = (in && beta != 0.0) ? pd_c[(int64_t)(c0 + q) * ldc] : 0.0;
        csv[q] = in ? pd_cs[c0 + q] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (c0 + q >= pd_cols) break;
        if (c0 + q < pd_first) continue;
        uint32_t u[kMaxModuli];
#pragma unroll
        for (int l = 0; l < kMaxModuli; ++l) u[l] = (w4[l] >> (8 * q)) & 0xFFu;
        const double w0 = beta != 0.0 ? beta * c0v[q] : 0.0;
        double w;
        if (nan_out || pd_bad || csv[q] != csv[q]) w = __longlong_as_double(0x7FF8000000000000ll);
        else w = fma(csv[q], scaled_double(crt_combine(u, p, TABLE ? *pd_cset : *cset, nm), pd_sig), w0);
        pd_c[(int64_t)(c0 + q) * ldc] = w;
      }
    }
    pd_done = g1;
    if (pd_done >= kGroups) pd_active = false;
  };

  uint32_t chunk = 0;
  int acc[COLS];
  int tcount = 0;
  const int tile_end = PAIR ? p.tile_end : p.num_tiles;
  int cur = 0;  // grouped: the table entry of the current tile (a CTA's tiles increase)
  for (int tile = tile0; tile < tile_end; tile += tile_step) {
    int tm, tn, nkb = p.nkb;
    const ModTableEntry* e = nullptr;
    if (TABLE) {
      while (cur + 1 < count && table[cur + 1].tile_begin <= tile) ++cur;
      e = &table[cur];
      const ModPlan* pl = e->plan;
      if (!pl->feasible) continue;  // computed by the FP64 kernel instead
      nmod = pl->n;
      nkb = e->nkb;
      cset = &p.set[nmod - 1];
      per_boundary = (kGroups + nmod - 1) / nmod;
      tile_coords(tile - (int)e->tile_begin, e->tiles_m, e->group_m, e->num_tiles, tm, tn);
    } else if (PAIR) {
      raster_coords(p.tri, tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
    } else {
      tile128_coords(p, tile, tm, tn);
    }
    const int64_t i = (int64_t)tm * tbm + row_off + row;
    const int64_t jc0 = (int64_t)tn * TBN + col0;
    const int slot = tcount & 1;
    ++tcount;
    uint8_t* const ub = scr_cta + (int64_t)slot * kSlotBytes;
    for (int l = 0; l < nmod; ++l) {
      const uint32_t pm = (uint32_t)p.p[l], bm = p.bar[l];
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
        tc_fence_before();
        if (PAIR) mbar_arrive_remote(empty_remote[buf]);
        else mbar_arrive(&acc_empty[buf]);
        if (++nch == kReduceChunks) {  // keep the running sums below 2^30 in magnitude
          nch = 0;
#pragma unroll
          for (int c = 0; c < COLS; ++c) acc[c] = mod_nonneg(acc[c], pm, bm);
        }
      }
      const uint32_t cl = (uint32_t)cset->c[l];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        uint32_t w = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          w |= mod_barrett((uint32_t)mod_nonneg(acc[4 * g + b], pm, bm) * cl, pm, bm) << (8 * b);
        *reinterpret_cast<uint32_t*>(ub + l * kLStride + g * 512) = w;
      }
      if (pd_active) advance(l + 1 == nmod ? kGroups : per_boundary);
    }
    // this tile's residues are complete: it becomes the pending reconstruction
    const int64_t pm = TABLE ? e->m : p.m, pn = TABLE ? e->n : p.n;
    const bool row_ok = i < pm;
    pd_active = true;
    pd_done = 0;
    pd_slot = slot;
    pd_cols = row_ok && jc0 < pn ? (int)min((int64_t)COLS, pn - jc0) : 0;
    pd_first = 0;
    if (!TABLE && p.tri == 1) pd_cols = (int)max((int64_t)0, min((int64_t)pd_cols, i - jc0 + 1));  // j <= i
    else if (!TABLE && p.tri == 2) pd_first = (int)max((int64_t)0, i - jc0);                      // j >= i
    pd_sig = 0;
    pd_bad = false;
    const int* sigA = TABLE ? e->sigA : p.sigA;
    const int* badA = TABLE ? e->badA : p.badA;
    if (row_ok) {
      const int sg = sigA[i];
      pd_sig = sg == kExpEmpty ? 0 : sg;
      pd_bad = badA[i] != 0;
    }
    if (TABLE) {
      pd_nmod = nmod;
      pd_cset = cset;
      pd_beta = e->beta;
      pd_ldc = e->ldc;
      pd_c = e->C + jc0 * e->ldc + i;  // dereferenced only for the pd_cols columns inside C
      pd_cs = e->cs + jc0;
    } else {
      pd_c = p.C + jc0 * p.ldc + i;
      pd_cs = p.cs + jc0;
    }
  }
  if (pd_active) advance(kGroups);
}

// The epilogue of the split form (one-SM kernel, 128 x 128 tiles, few of them): the moduli
// of a tile are spread over `groups` work units on different CTAs.  Each unit drains its
// moduli and parks their bytes in the tile's global slot; after a barrier of the epilogue
// warps one thread publishes the unit (fence, then a counter per tile); the CTA that
// finishes the tile's last unit rebuilds the whole tile from the slot, immediately.
template <int EPI_WARPS, int TBN>
__device__ __forceinline__ void mod_epilogue_split(const ModArgs& p, int nmod, bool nan_out, uint32_t tmem_base,
                                                   uint64_t* acc_full, uint64_t* acc_empty, int* last_flag, int warp,
                                                   int lane) {
  constexpr int COLS = TBN / (EPI_WARPS / 4);
  constexpr int kGroups = COLS / 4;
  constexpr int64_t kTileStride = (int64_t)TBN / 4 * 128 * 4;  // one modulus of one tile
  const CrtSet& cset = p.set[nmod - 1];
  const int ew = warp - 2;
  const int quad = warp & 3;
  const int part = ew >> 2;
  const int row = quad * 32 + lane;
  const int col0 = part * COLS;
  const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
  const int groups = min(p.groups, nmod);
  const int units = p.num_tiles * groups;
  uint32_t chunk = 0;
  int acc[COLS];
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int tile = u / groups;
    int l0, l1;
    unit_range(u % groups, groups, nmod, l0, l1);
    uint8_t* const ub = p.tslot + (int64_t)tile * kMaxModuli * kTileStride + (int64_t)(col0 / 4) * 512 + row * 4;
    for (int l = l0; l < l1; ++l) {
      const uint32_t pm = (uint32_t)p.p[l], bm = p.bar[l];
#pragma unroll
      for (int c = 0; c < COLS; ++c) acc[c] = 0;
      int nch = 0;
      for (int i0 = 0; i0 < p.nkb; i0 += kChunkBlocks, ++chunk) {
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
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
        if (++nch == kReduceChunks) {
          nch = 0;
#pragma unroll
          for (int c = 0; c < COLS; ++c) acc[c] = mod_nonneg(acc[c], pm, bm);
        }
      }
      const uint32_t cl = (uint32_t)cset.c[l];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        uint32_t w = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          w |= mod_barrett((uint32_t)mod_nonneg(acc[4 * g + b], pm, bm) * cl, pm, bm) << (8 * b);
        *reinterpret_cast<uint32_t*>(ub + l * kTileStride + g * 512) = w;
      }
    }
    // publish the unit; the last of the tile's units rebuilds it
    epi_barrier<EPI_WARPS>();
    if (warp == 2 && lane == 0) {
      __threadfence();
      const unsigned int prev = atomicAdd(p.tile_done + tile, 1u);
      *last_flag = prev + 1u == (unsigned int)groups;
    }
    epi_barrier<EPI_WARPS>();
    if (!*last_flag) continue;
    __threadfence();  // the other units' bytes, published before their counts
    int tm, tn;
    tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
    const int64_t i = (int64_t)tm * 128 + row;
    const int64_t jc0 = (int64_t)tn * TBN + col0;
    if (i >= p.m || jc0 >= p.n) continue;
    const int cols = (int)min((int64_t)COLS, p.n - jc0);
    const int sg = p.sigA[i];
    const int sig = sg == kExpEmpty ? 0 : sg;
    const bool bad = p.badA[i] != 0;
    double* crow = p.C + jc0 * p.ldc + i;
    for (int g = 0; g * 4 < cols; ++g) {
      uint32_t w4[kMaxModuli];
#pragma unroll
      for (int l = 0; l < kMaxModuli; ++l)
        w4[l] = l < nmod ? __ldcg(reinterpret_cast<const unsigned int*>(ub + l * kTileStride + g * 512)) : 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 4 * g + q;
        if (c >= cols) break;
        uint32_t uu[kMaxModuli];
#pragma unroll
        for (int l = 0; l < kMaxModuli; ++l) uu[l] = (w4[l] >> (8 * q)) & 0xFFu;
        const double csv = p.cs[jc0 + c];
        const double w0 = p.beta != 0.0 ? p.beta * crow[(int64_t)c * p.ldc] : 0.0;
        double w;
        if (nan_out || bad || csv != csv) w = __longlong_as_double(0x7FF8000000000000ll);
        else w = fma(csv, scaled_double(crt_combine(uu, p, cset, nmod), sig), w0);
        crow[(int64_t)c * p.ldc] = w;
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
  static constexpr int kBytes = kOffTmemSlot + 16;
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
  int* last_flag = reinterpret_cast<int*>(smem + L::kOffTmemSlot + 8);
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
  const ModPlan plan = *p.plan;  // written by k_mod_plan earlier on the stream (grouped: the first problem's)
  const int nmod = plan.n;
  // work units: tiles, or (tile, group of moduli) with at most nmod groups per tile
  const int groups = SPLIT ? min(p.groups, nmod) : 1;
  const int units = p.num_tiles * groups;
  // grouped: the moduli count and k-blocks of unit u's problem (0 moduli: skipped), its maps
  auto table_unit = [&](int u, int& cur, int& tm, int& tn, int& nm, int& nkb, const CUtensorMap*& ma,
                        const CUtensorMap*& mb) {
    while (cur + 1 < count && table[cur + 1].tile_begin <= u) ++cur;
    const ModTableEntry& e = table[cur];
    const ModPlan* pl = e.plan;
    nm = pl->feasible ? pl->n : 0;
    nkb = e.nkb;
    tile_coords(u - (int)e.tile_begin, e.tiles_m, e.group_m, e.num_tiles, tm, tn);
    ma = &e.tmA;
    mb = &e.tmB;
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
  } else if (SPLIT) {
    mod_epilogue_split<kEpiWarps, kBN>(p, nmod, plan.feasible == 0, tmem_base, acc_full, acc_empty, last_flag, warp,
                                       lane);
  } else {
    mod_epilogue<kEpiWarps, kBN, false, TABLE>(p, nmod, !TABLE && plan.feasible == 0, tmem_base, acc_full, acc_empty,
                                               warp, lane, blockIdx.x, gridDim.x, kBM, 0, table, count);
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
static_assert(k2BN <= kSlotCols && kBN <= kSlotCols, "parked bytes of a tile fit one slot");

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
    k_mod_gemm_pair(const __grid_constant__ ModArgs p, const __grid_constant__ CUtensorMap tmA,
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
  const ModPlan plan = *p.plan;  // written by k_mod_plan earlier on the stream
  const int nmod = plan.n;

  if (warp == 0) {
    // ------------------------------ TMA producer (both CTAs) ------------------------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      const uint32_t pair_bytes = (uint32_t)(2 * (L::kABytes + L::kBBytes));
      for (int tile = pair_id; tile < p.tile_end; tile += num_pairs) {
        int tm, tn;
        raster_coords(p.tri, tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
        const int m0 = tm * k2BM + (int)rank * 128;
        const int nb0 = tn * k2BN + (int)rank * 128;
        for (int l = 0; l < nmod; ++l)
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
      for (int tile = pair_id; tile < p.tile_end; tile += num_pairs)
        for (int l = 0; l < nmod; ++l)
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
    mod_epilogue<k2EpiWarps, k2BN, true>(p, nmod, plan.feasible == 0, tmem_base, acc_full, acc_empty, warp, lane,
                                         pair_id, num_pairs, k2BM, (int)rank * 128);
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
  uint8_t* scr;  // [scr_ctas][2][kSlotBytes]
  int scr_ctas;
  uint8_t* tslot;            // [tiles][kTileSlotBytes] when the split form may run, else null
  unsigned int* tile_done;   // [tiles]
  int64_t kp;
};

// scratch = false (a problem of a grouped launch): no park slots, no split-form slots; the
// launch has its own
size_t mod_layout(int64_t m, int64_t n, int64_t k, int nmod, void* base, ModWorkspace* ws, bool scratch = true) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t kp = (k + 7) / 8 * 8;
  // one CTA per 128 x 128 tile (one-SM form) or two per 256 x 256 tile (two-SM form), at most kMaxModCtas
  const int64_t tiles1 = ((m + 127) / 128) * ((n + 127) / 128);
  const int64_t tiles2 = ((m + 255) / 256) * ((n + 255) / 256);
  int64_t ctas = tiles1 > 2 * tiles2 ? tiles1 : 2 * tiles2;
  if (ctas > kMaxModCtas) ctas = kMaxModCtas;
  if (!scratch) ctas = 0;
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
  const size_t o_scr = off; off = up(off + 2 * (size_t)kSlotBytes * (size_t)ctas);
  const int64_t split_tiles = (scratch && tiles1 <= kSplitMaxTiles) ? tiles1 : 0;
  const size_t o_tslot = off; off = up(off + (size_t)kTileSlotBytes * (size_t)split_tiles);
  const size_t o_tdone = off; off = up(off + sizeof(unsigned int) * (size_t)split_tiles);
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
    ws->scr = reinterpret_cast<uint8_t*>(b + o_scr);
    ws->scr_ctas = (int)ctas;
    ws->tslot = split_tiles ? reinterpret_cast<uint8_t*>(b + o_tslot) : nullptr;
    ws->tile_done = split_tiles ? reinterpret_cast<unsigned int*>(b + o_tdone) : nullptr;
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

int64_t inverse_mod(int64_t a, int64_t p) {  // a^-1 mod p, gcd(a, p) = 1
  int64_t t = 0, nt = 1, r = p, nr = ((a % p) + p) % p;
  while (nr) {
    const int64_t q = r / nr;
    int64_t x = t - q * nt; t = nt; nt = x;
    x = r - q * nr; r = nr; nr = x;
  }
  return t < 0 ? t + p : t;
}

// the moduli, their Barrett constants and the reconstruction constants of every n = 1..kMaxModuli;
// the rest of `a` zeroed
void mod_constants(ModArgs& a, const ModProducts& prods) {
  memset(&a, 0, sizeof(a));
  for (int l = 0; l < kMaxModuli; ++l) {
    a.p[l] = kModuli[l];
    a.bar[l] = (uint32_t)((1ull << 32) / (uint64_t)kModuli[l]);
    a.rq[l] = ((1u << 24) + (uint32_t)kModuli[l] - 1u) / (uint32_t)kModuli[l];
  }
  for (int nn = 1; nn <= kMaxModuli; ++nn) {
    CrtSet& cs = a.set[nn - 1];
    const hu128 M = ((hu128)prods.hi[nn - 1] << 64) | prods.lo[nn - 1];
    for (int l = 0; l < nn; ++l) {
      const hu128 Mp = M / (hu128)kModuli[l];
      cs.c[l] = (int)inverse_mod((int64_t)(Mp % (hu128)kModuli[l]), kModuli[l]);
      for (int w = 0; w < 4; ++w) cs.mpl[l][w] = (uint32_t)(Mp >> (32 * w));
    }
    cs.M_lo = (uint64_t)M; cs.M_hi = (uint64_t)(M >> 64);
    const hu128 half = M / 2;
    cs.half_lo = (uint64_t)half; cs.half_hi = (uint64_t)(half >> 64);
  }
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

// the product kernel of one call; `a` carries everything but the tile geometry; the residue
// planes hold up to nmod_ws moduli (the plan's n is at most that)
int launch_mod_gemm(int64_t m, int64_t n, int64_t k, int nmod_ws, ModArgs& a, const ModWorkspace& ws, int sms,
                    cudaStream_t stream) {
  // GBD_EMU_KERNEL=pair|single|split overrides the choice (tests and tuning).  Otherwise the
  // expected time in units of one 128 x 128 tile on one SM: whole waves of tiles over the SMs
  // (or SM pairs), a 256 x 256 tile being four units on two SMs at kModPairGain, a last wave
  // that leaves pairs idle going to one-SM CTAs when its quarters fit one wave; and the one-SM
  // form splits the moduli of each tile over several CTAs for at most 8 tiles, or for fewer
  // tiles than half the SMs with a deep inner dimension (k >= 2048); measured at 256^3 (4
  // tiles) 0.145 against 0.169 ms, 256^2 x 4096 0.25 against 0.47 ms, but 512^3 (16 tiles) 0.22
  // against 0.20 ms and 1024^3 (64 tiles) 0.34 against 0.30 ms.
  const char* force = getenv("GBD_EMU_KERNEL");
  const bool force_split = force && strcmp(force, "split") == 0;
  if (force_split) force = nullptr;
  const int cta_cap = sms < ws.scr_ctas ? sms : ws.scr_ctas;
  // a triangular output (m = n) covers the tiles that meet its triangle
  auto count = [&](int64_t bm, int64_t bn) {
    const int64_t tm = (m + bm - 1) / bm, tn = (n + bn - 1) / bn;
    return a.tri ? tm * (tm + 1) / 2 : tm * tn;
  };
  const int64_t tiles1 = count(kBM, kBN);
  const int64_t tiles2 = count(k2BM, k2BN);
  const int64_t pairs_avail = cta_cap / 2 > 0 ? cta_cap / 2 : 1;
  const int64_t pairs = tiles2 < pairs_avail ? tiles2 : pairs_avail;
  const int64_t waves2 = (tiles2 + pairs - 1) / pairs;
  const int64_t last = tiles2 - (waves2 - 1) * pairs;  // tiles of the last two-SM wave
  const char* tail_env = getenv("GBD_EMU_TAIL");       // GBD_EMU_TAIL=0 keeps the last wave on the pairs
  const bool tail = waves2 > 1 && last < pairs && 4 * last <= cta_cap && !(tail_env && tail_env[0] == '0');
  const double t_one = (double)((tiles1 + cta_cap - 1) / cta_cap);
  const double t_pair = tail ? (double)(waves2 - 1) * 2.0 / kModPairGain + 1.0 : (double)waves2 * 2.0 / kModPairGain;
  const bool pair = (force ? force[0] == 'p' : t_pair < t_one) && cta_cap >= 2;
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
  a.tile_end = (int)tiles;
  a.tail_from = -1;
  a.tail_tiles_m = a.tail_group_m = a.tail_num = 0;
  cudaError_t e;
  const bool split = !pair && ws.tslot != nullptr && a.tri == 0 &&
                     (force_split || (!force && (tiles <= 8 || (2 * tiles < sms && k >= 2048))));
  if (split) {
    int groups = (int)((sms + tiles - 1) / tiles);  // the kernel keeps at most nmod of them
    if (groups > kMaxModuli) groups = kMaxModuli;
    a.groups = groups;
    a.tslot = ws.tslot;
    a.tile_done = ws.tile_done;
    a.group_m = 1;
    const int64_t units = tiles * groups;
    const int grid = (int)(units < sms ? units : sms);
    if ((e = cudaMemsetAsync(ws.tile_done, 0, sizeof(unsigned int) * (size_t)tiles, stream)) != cudaSuccess)
      return cuda_fail(e, "modular gemm: clearing the tile counters");
    e = cudaFuncSetAttribute(k_mod_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm split)");
    k_mod_gemm<true><<<grid, kThreads, Smem::kAlloc, stream>>>(a, tmA, tmB);
  } else if (pair) {
    a.group_m = group_rows((int)pairs, k2BM, k2BN, a.tiles_m);
    // a last wave that would leave SM pairs idle goes to one-SM CTAs instead, as four 128 x 128
    // tiles per 256 x 256 tile, when they fill at most one wave of SMs: it then takes about
    // kModPairGain / 2 of a two-SM wave
    if (tail) a.tile_end = (int)(tiles - last);
    e = cudaFuncSetAttribute(k_mod_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem2::kAlloc);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm pair)");
    k_mod_gemm_pair<<<(unsigned)(2 * pairs), k2Threads, Smem2::kAlloc, stream>>>(a, tmA, tmB);
    if (tail) {
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "modular gemm pair launch");
      ModArgs b = a;
      b.tail_from = a.tile_end;
      b.tail_tiles_m = a.tiles_m;
      b.tail_group_m = a.group_m;
      b.tail_num = a.num_tiles;
      b.tiles_m = 0;
      b.group_m = 1;
      b.num_tiles = b.tile_end = (int)(4 * last);
      e = cudaFuncSetAttribute(k_mod_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(modular gemm)");
      k_mod_gemm<false><<<(unsigned)(4 * last), kThreads, Smem::kAlloc, stream>>>(b, tmA, tmB);
    }
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
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  struct EventGuard {
    cudaEvent_t* e;
    ~EventGuard() {
      for (int i = 0; i < 3; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  cudaError_t e;
  if (timing) {
    for (int i = 0; i < 3; ++i)
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

  // products modulo each modulus and the reconstruction; the constants of every n ride along
  ModArgs a;
  mod_constants(a, prods);
  a.tri = tri;
  a.m = m; a.n = n; a.ldc = ldc;
  a.plan = ws.plan;
  a.beta = beta;
  a.C = C;
  a.sigA = ws.sigA; a.badA = ws.badA;
  a.cs = ws.cs;
  a.scr = ws.scr;
  a.err = device_error_word();
  if (timing && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return cuda_fail(e, "dgemm_emu_mod: cudaEventRecord");
  if ((rc = launch_mod_gemm(m, n, k, nmod_ws, a, ws, sms, s))) return rc;
  if (timing) {
    float t0 = 0.f, t1 = 0.f;
    if ((e = cudaEventRecord(ev[2], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[2])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t0, ev[0], ev[1])) != cudaSuccess ||
        (e = cudaEventElapsedTime(&t1, ev[1], ev[2])) != cudaSuccess)
      return cuda_fail(e, "dgemm_emu_mod: phase timing");
    info->prep_ms = t0;
    info->gemm_ms = t1;
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
constexpr int kGroupedModCtas = 160;  // park slots of the grouped product launch (one CTA per SM)
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

size_t mod_grouped_layout(const gbd_problem* probs, const int* which, int count, void* base, ModGrouped* g, int* rc) {
  *rc = GBD_OK;
  char* b = static_cast<char*>(base);
  size_t off = 0;
  int64_t tiles = 0;
  for (int q = 0; q < count; ++q) {
    const gbd_problem& p = probs[which[q]];
    tiles += ((p.m + kBM - 1) / kBM) * ((p.n + kBN - 1) / kBN);
  }
  const int ctas = (int)(tiles < kGroupedModCtas ? (tiles > 0 ? tiles : 1) : kGroupedModCtas);
  const size_t o_jobs = off; off = up256(off + sizeof(PrepJob) * 2 * (size_t)count);
  const size_t o_cert = off; off = up256(off + sizeof(CertTableEntry) * 2 * (size_t)count);  // FP8, BF16 retry
  const size_t o_plj = off; off = up256(off + sizeof(ModPlanJob) * (size_t)count);
  const size_t o_col = off; off = up256(off + sizeof(ColJob) * (size_t)count);
  const size_t o_tab = off; off = up256(off + sizeof(ModTableEntry) * (size_t)count);
  const size_t o_words = off; off = up256(off + sizeof(unsigned int) * kCertWords * (size_t)(count + 1));
  const size_t o_scr = off; off = up256(off + 2 * (size_t)kSlotBytes * (size_t)ctas);
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
    off = up256(off + mod_layout(p.m, p.n, p.k, nm, nullptr, nullptr, false));
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
  g->scr = reinterpret_cast<uint8_t*>(b + o_scr);
  g->scr_ctas = ctas;
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
    mod_layout(p.m, p.n, p.k, nmod_ws[q], b + o_ws[q], &ws[q], false);
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
  // the product table: the deepest problems' tiles first (longest tiles first over the SMs)
  std::vector<int> order(count);
  for (int q = 0; q < count; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return probs[which[x]].k > probs[which[y]].k; });
  g->table.assign(count, ModTableEntry{});
  int64_t mt = 0;
  for (int r = 0; r < count; ++r) {
    const int q = order[r];
    const gbd_problem& p = probs[which[q]];
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
    e.m = p.m; e.n = p.n; e.ldc = p.ldc;
    e.beta = p.beta;
    e.C = p.C;
    e.sigA = w.sigA; e.badA = w.badA;
    e.cs = w.cs;
    e.plan = w.plan;
    e.nkb = (int)((p.k + kBK - 1) / kBK);
    e.tiles_m = (int)((p.m + kBM - 1) / kBM);
    e.num_tiles = e.tiles_m * (int)((p.n + kBN - 1) / kBN);
    e.group_m = e.tiles_m;  // within one problem the tiles walk down the rows
    e.tile_begin = mt;
    mt += e.num_tiles;
  }
  g->mod_tiles = (int)mt;
  if (mt > ((int64_t)1 << 30) || cert_tiles > ((int64_t)1 << 30)) *rc = set_error(GBD_ERR_LIMIT, "grouped: too many tiles");
  return off;
}

int mod_grouped_upload(const ModGrouped& g, cudaStream_t s) {
  if (g.count == 0) return GBD_OK;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(g.jobs_dev, g.jobs.data(), sizeof(PrepJob) * g.jobs.size(), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(g.cert_dev, g.cert.data(), sizeof(CertTableEntry) * g.cert.size(), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(g.planjobs_dev, g.planjobs.data(), sizeof(ModPlanJob) * g.planjobs.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(g.coljobs_dev, g.coljobs.data(), sizeof(ColJob) * g.coljobs.size(), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(g.table_dev, g.table.data(), sizeof(ModTableEntry) * g.table.size(),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "grouped modular: table copies");
  return GBD_OK;
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
  if ((rc = launch_statplane_batched(g.jobs_dev, njobs, g.split_blocks, max_rows, s))) return rc;
  // the certification: magnitude planes, their products, the plans (the same precision as the
  // single call's, so that a problem gets the same plan alone and in a batch)
  const int prec = cert_prec_default();
  const bool retry = prec == kCertFP8;
  if (prec == kCertBF16 && (rc = launch_magplane_batched(g.jobs_dev, njobs, g.split_blocks, s, prec))) return rc;
  if ((rc = launch_cert_grouped(g.cert_dev, g.count, g.cert_tiles, prec, sms, s))) return rc;
  const ModProducts prods = moduli_products();
  k_mod_plan_batched<<<(g.count + 127) / 128, 128, 0, s>>>(g.planjobs_dev, g.count, prods, 0, g.flags_dev,
                                                           retry ? 0 : 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped plan launch");
  if (retry) {
    // the BF16 retry of every problem whose plan found no feasible t; the launches return at once
    // when no problem needs it, and skip the problems whose plan is feasible
    if ((rc = launch_magplane_batched(g.jobs_dev, njobs, g.split_blocks, s, kCertBF16, g.flags_dev))) return rc;
    if ((rc = launch_cert_grouped(g.cert_dev + g.count, g.count, g.cert_tiles, kCertBF16, sms, s, g.flags_dev)))
      return rc;
    k_mod_plan_batched<<<(g.count + 127) / 128, 128, 0, s>>>(g.planjobs_dev, g.count, prods, 1, g.flags_dev, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped plan launch");
  }
  // residues and column scales with each problem's plan
  ModSplit ms;
  mod_split_params(ms);
  if ((rc = launch_residue_batched(g.jobs_dev, njobs, ms, g.split_blocks, s))) return rc;
  k_mod_colscale_batched<<<g.count, 256, 0, s>>>(g.coljobs_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped column scale launch");
  // the products of every feasible problem in one persistent launch
  if (g.mod_tiles <= 0) return GBD_OK;
  ModArgs a;
  mod_constants(a, moduli_products());
  a.plan = g.plans[0];  // read at kernel start; the tiles use their own problems' plans
  a.scr = g.scr;
  a.err = device_error_word();
  a.num_tiles = g.mod_tiles;
  a.tile_end = g.mod_tiles;
  a.tail_from = -1;
  a.tiles_m = 1;
  a.group_m = 1;
  a.nkb = 1;
  a.groups = 1;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  int grid = g.mod_tiles < sms ? g.mod_tiles : sms;
  if (grid > g.scr_ctas) grid = g.scr_ctas;
  e = cudaFuncSetAttribute(k_mod_gemm<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped modular gemm)");
  k_mod_gemm<false, true><<<grid, kThreads, Smem::kAlloc, s>>>(a, dummy, dummy, g.table_dev, g.count);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "grouped modular gemm launch");
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
