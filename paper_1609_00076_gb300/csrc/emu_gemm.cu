// emu_gemm.cu -- steps 3 and 4 of the split emulation on the 5th-generation
// tensor cores: the digit-slice products with tcgen05.mma (BF16 x BF16 -> FP32 in
// Tensor Memory), exact integer level sums, and the FP64 update of C.
//
// Persistent, warp-specialised kernel; one 128 x BN output tile at a time per CTA:
//   warp 0      TMA producer: for each (segment, level g, k-block, pair t) loads the
//               128 x 64 tile of digit slice t of op(A) and the BN x 64 tile of slice
//               g-t of op(B)^T (128-byte swizzle) into a kStages-deep ring;
//   warp 1      MMA issuer: 4 x tcgen05.mma (M=128, N=BN, K=16) per k-block into one
//               of two TMEM accumulators; a chunk of kChunkBlocks k-blocks (1024 k) is
//               accumulated from zero, so every FP32 partial sum is an integer below
//               2^24 and exact;
//   warps 2..9  epilogue: drain each finished chunk from TMEM (tcgen05.ld) and add it
//               exactly into 32-bit integer registers (cvt.rni.s32.f32 of an exact
//               integer), so the MMA runs on while a chunk is drained.  A finished
//               level's sums are parked in scratch; at the end of a group of up to
//               kGroupLevels levels (smallest level h) they are combined exactly into
//               Y = sum_g P_g 2^(b (h - g)) in 64-bit integers and
//               C := fma(alpha 2^(tau_j - h b), Y 2^sigma_i, C), one FP64 fma per
//               element and group, coalesced down the columns of C.
// All waits are bounded (2 s); a wait that gives up sets the device error word and
// the kernel runs to its end without hanging.
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

constexpr int kBM = 128;
constexpr int kStages = 6;
constexpr int kMaxGroups = (kMaxSlices + kGroupLevels - 1) / kGroupLevels;  // level groups per segment
constexpr int kEpiWarps = 8;                     // two-SM kernel: 2 x 4 warps over 128 lanes x 256 columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kEpiWarps1 = 16;                   // one-SM kernel: 4 x 4 warps over 128 lanes x 128 columns
constexpr int kThreads1 = 64 + 32 * kEpiWarps1;
constexpr int kTmemCols = 512;

template <int BN>
struct SmemLayout {
  static constexpr int kABytes = kBM * kBK * 2;  // 16 KiB
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + kStages * kABytes;
  static constexpr int kOffBar = kOffB + kStages * kBBytes;
  static constexpr int kNumBars = 2 * kStages + 5;  // full, empty, acc_full[2], acc_empty[2], done
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kOffScale = (kOffTmemSlot + 16 + 15) / 16 * 16;
  static constexpr int kBytes = kOffScale + kMaxGroups * BN * 8 + 16;  // colscale per level group, a flag
  static constexpr int kAlloc = kBytes + 1024;  // slack to align the base to 1024 bytes
  static_assert(kAlloc <= 227 * 1024, "shared memory of one CTA");
};

struct Args {
  int64_t m, n, k;
  int slices;
  int nkb;      // k-blocks of kBK
  int tiles_m;  // row tiles
  int num_tiles;
  int group_m;  // rasterisation: consecutive tiles walk group_m row tiles, then the next column
  double alpha, beta;
  double* C;
  int64_t ldc;
  const int* sigA;
  const int* sigB;
  const int* badA;
  const int* badB;
  double* scratch;     // two-SM kernel: one 128 x 256 FP64 slot per CTA (running sums)
  int32_t* scratch_p;  // two-SM kernel: kParkSlots 128 x 256 int32 slots per CTA (parked level sums)
  unsigned int* err;
  // one-SM kernel, split inner dimension: each k segment of a tile is cut into `splits`
  // sub-ranges, one work item each; the items add their exact group sums into ysum
  // [tile][segment][group][128 x 128] (column-major) and the tile's last item applies them
  int splits;               // 1: a CTA takes whole tiles
  int nsegs, ngroups;       // k segments per tile, level groups per segment
  unsigned long long* ysum;  // zeroed before the launch
  unsigned int* tile_done;   // items finished per tile, zeroed before the launch
};

// named barrier 1 over the epilogue warps only (the two-SM kernel's by default)
template <int WARPS = kEpiWarps>
__device__ __forceinline__ void epi_bar_sync() {
  epi_barrier<WARPS>();
}

// x * 2^e for the rare results outside the normal range, out of line so that its code
// takes no registers in the unrolled epilogue loops
__device__ __noinline__ double ldexp_rare(double x, int e) { return ldexp(x, e); }

// Y * 2^sigma as a double, exactly (Y is an integer with |Y| < 2^53)
__device__ __forceinline__ double scaled_i64(int64_t Y, int sigma) {
  if (Y == 0) return 0.0;
  const uint64_t a = Y < 0 ? 0ull - (uint64_t)Y : (uint64_t)Y;
  const int msb = 63 - __clzll((long long)a);
  const int ef = 1023 + msb + sigma;
  if (ef <= 0 || ef >= 2047) return ldexp_rare((double)Y, sigma);  // outside the normal range
  const uint64_t mant = (a << (52 - msb)) & 0xFFFFFFFFFFFFFull;
  const uint64_t bits = ((uint64_t)(Y < 0) << 63) | ((uint64_t)ef << 52) | mant;
  return __longlong_as_double((long long)bits);
}

// Parked sums P_l (l = h - g, level g of the group whose smallest level is h) combined
// exactly: Y = sum_l P_l 2^(b l); levels the group does not have are zero.
__device__ __forceinline__ int64_t combine_levels(const int32_t (&P)[kGroupLevels]) {
  int64_t Y = P[kGroupLevels - 1];
#pragma unroll
  for (int l = kGroupLevels - 2; l >= 0; --l) Y = Y * (1 << kDigitBits) + P[l];
  return Y;
}

// largest level of the group whose smallest level is h (levels h, h-1, ..., down to 2)
__device__ __forceinline__ int group_high(int h) { return max(2, h - kGroupLevels + 1); }

// number of MMA chunks of level-segment (g, seg0..seg0+segn)
__device__ __forceinline__ int chunks_of(int g, int segn) {
  return ((g - 1) * segn + kChunkBlocks - 1) / kChunkBlocks;
}

// One output tile's view of its problem.  The single-problem launch reads the
// problem's fields from the kernel arguments, the grouped launch from the tile's
// table entry in global memory (JF below); only the entry's address is kept, so the
// fields are not held in registers across the tile.
struct Job {
  const EmuTableEntry* e;  // grouped launch: this tile's problem
  int m0, n0;
  int s, nkb;
};
#define JF(field) (TABLE ? j.e->field : p.field)

template <int BM, int BN, bool TABLE>
__device__ __forceinline__ void get_job(const Args& p, const EmuTableEntry* table, int count, int tile, int& cur,
                                        Job& j) {
  int tm, tn;
  if (!TABLE) {
    tile_coords(tile, p.tiles_m, p.group_m, p.num_tiles, tm, tn);
    j.e = nullptr;
    j.s = p.slices; j.nkb = p.nkb;
  } else {
    // last entry whose first tile is <= tile; a CTA's tiles increase, so cur only moves forward
    while (cur + 1 < count && table[cur + 1].tile_begin <= tile) ++cur;
    const EmuTableEntry& e = table[cur];
    tile_coords((int)(tile - e.tile_begin), e.tiles_m, e.group_m, e.num_tiles, tm, tn);
    j.e = &e;
    j.s = p.slices;  // one launch per slice count: a launch constant keeps the loop control uniform
    j.nkb = e.nkb;
  }
  j.m0 = tm * BM;
  j.n0 = tn * BN;
}

// Work item of the one-SM kernel: a whole tile, or with a split inner dimension one
// sub-range of one k segment of a tile (the items of a tile are consecutive).
template <bool TABLE>
__device__ __forceinline__ void item_coords(const Args& p, int item, int& tile, int& seg, int& sub) {
  if (!TABLE && p.splits > 1) {
    const int per = p.nsegs * p.splits;
    tile = item / per;
    const int r = item - tile * per;
    seg = r / p.splits;
    sub = r - seg * p.splits;
  } else {
    tile = item;
    seg = 0;
    sub = 0;
  }
}
// k-block range [kb0, kb1) of an item (the whole inner dimension without a split)
template <bool TABLE>
__device__ __forceinline__ void item_range(const Args& p, int nkb, int seg, int sub, int& kb0, int& kb1) {
  if (!TABLE && p.splits > 1) {
    const int s0 = seg * kSegBlocks;
    const int len = min(kSegBlocks, nkb - s0);
    kb0 = s0 + (int)((int64_t)sub * len / p.splits);
    kb1 = s0 + (int)((int64_t)(sub + 1) * len / p.splits);
  } else {
    kb0 = 0;
    kb1 = nkb;
  }
}

template <int BN, bool TABLE>
__global__ void __launch_bounds__(kThreads1, 1)
    k_slice_gemm(const Args p, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const EmuTableEntry* __restrict__ table, int count, int total_tiles) {
  using L = SmemLayout<BN>;
  // TMEM: two FP32 accumulators of BN columns, then the low and high words of the group sum Y
  static_assert(4 * BN <= kTmemCols, "accumulators and group sums must fit in TMEM");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = bars + 2 * kStages + 2;
  uint64_t* done = bars + 2 * kStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmemSlot);
  double* colscale = reinterpret_cast<double*>(smem + L::kOffScale);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool split = !TABLE && p.splits > 1;
  const int nitems = TABLE ? total_tiles : (split ? p.num_tiles * p.nsegs * p.splits : p.num_tiles);

  if (warp == 0 && lane == 0) {
    if (!TABLE) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
    }
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 32 * kEpiWarps1);
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
      int cur = 0;
      for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        int tile, seg, sub, kb0, kb1;
        item_coords<TABLE>(p, item, tile, seg, sub);
        Job j;
        get_job<kBM, BN, TABLE>(p, table, count, tile, cur, j);
        item_range<TABLE>(p, j.nkb, seg, sub, kb0, kb1);
        const CUtensorMap* mapA = TABLE ? &j.e->tmA : &tmA;
        const CUtensorMap* mapB = TABLE ? &j.e->tmB : &tmB;
        if (TABLE) {  // maps written into global memory before the launch: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapA) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapB) : "memory");
        }
        const int m0 = j.m0, n0 = j.n0;
        for (int seg0 = kb0; seg0 < kb1; seg0 += kSegBlocks) {
          const int segn = min(kSegBlocks, kb1 - seg0);
          for (int h = j.s + 1; h >= 2; h -= kGroupLevels)
            for (int g = h; g >= group_high(h); --g)
              for (int kb = seg0; kb < seg0 + segn; ++kb)  // k-major: tiles in flight share a narrow k window in L2
                for (int t = 1; t <= g - 1; ++t) {
                  mbar_wait(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
                  mbar_arrive_expect_tx(&full[stage], bytes);
                  tma_load_3d(smem + L::kOffA + stage * L::kABytes, mapA, &full[stage], kb * kBK, m0, t - 1);
                  tma_load_3d(smem + L::kOffB + stage * L::kBBytes, mapB, &full[stage], kb * kBK, n0, g - t - 1);
                  if (++stage == kStages) { stage = 0; phase ^= 1u; }
                }
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------ MMA issuer --------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      uint32_t stage = 0, phase = 0, chunk = 0;
      const uint32_t a_base = smem_u32(smem + L::kOffA), b_base = smem_u32(smem + L::kOffB);
      int cur = 0;
      for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        int tile, seg, sub, kb0, kb1;
        item_coords<TABLE>(p, item, tile, seg, sub);
        Job j;
        get_job<kBM, BN, TABLE>(p, table, count, tile, cur, j);
        item_range<TABLE>(p, j.nkb, seg, sub, kb0, kb1);
        for (int seg0 = kb0; seg0 < kb1; seg0 += kSegBlocks)
          for (int h = j.s + 1; h >= 2; h -= kGroupLevels)
          for (int g = h; g >= group_high(h); --g) {
            const int segn = min(kSegBlocks, kb1 - seg0);
            const int items = (g - 1) * segn;
            for (int i0 = 0; i0 < items; i0 += kChunkBlocks, ++chunk) {
              const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
              mbar_wait(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
              tc_fence_after();
              const uint32_t dtm = tmem_base + buf * BN;
              const int i1 = min(items, i0 + kChunkBlocks);
              for (int it = i0; it < i1; ++it) {
                mbar_wait(&full[stage], phase, p.err, kErrWaitTma);
                tc_fence_after();
                const uint64_t da = smem_desc_sw128(a_base + stage * L::kABytes);
                const uint64_t db = smem_desc_sw128(b_base + stage * L::kBBytes);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)  // K = 16 per MMA: +32 bytes = +2 in the descriptor
                  umma_bf16(dtm, da + 2 * kk, db + 2 * kk, idesc, (it > i0 || kk > 0) ? 1u : 0u);
                umma_commit(&empty[stage]);  // frees the stage when these MMAs have read it
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
              }
              umma_commit(&acc_full[buf]);  // chunk complete in TMEM
            }
          }
      }
      umma_commit(done);
      mbar_wait(done, 0, p.err, kErrWaitMma);  // every MMA of this CTA has finished
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue ----------------------------------
    // The exact group sum Y lives in TMEM next to the accumulators, as two 32-bit words
    // per element: each finished level is folded into it, and the group's last level
    // turns it into the FP64 update of C.  The MMA runs one chunk ahead meanwhile.
    constexpr int kParts = kEpiWarps1 / 4;  // warps that share one quarter of the TMEM lanes
    constexpr int kCols = BN / kParts;      // columns per thread
    const int ew = warp - 2;
    const int quad = warp & 3;     // TMEM lanes 32*quad .. +31 are reachable from this warp
    const int part = ew >> 2;      // which part of the tile's columns
    const int row = quad * 32 + lane;
    const int col0 = part * kCols;
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    const uint32_t y_lo = trow + 2 * BN + col0, y_hi = trow + 3 * BN + col0;
    uint32_t chunk = 0;
    uint32_t acc[kCols];
    int* last_flag = reinterpret_cast<int*>(colscale + kMaxGroups * BN);
    int cur = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      int tile, seg, sub, kb0, kb1;
      item_coords<TABLE>(p, item, tile, seg, sub);
      Job j;
      get_job<kBM, BN, TABLE>(p, table, count, tile, cur, j);
      item_range<TABLE>(p, j.nkb, seg, sub, kb0, kb1);
      const int64_t m0 = j.m0, n0 = j.n0;
      const int64_t i = m0 + row;
      const bool row_ok = i < JF(m);
      int sig_i = 0;
      bool bad_i = false;
      if (row_ok) {
        sig_i = JF(sigA)[i];
        if (sig_i == kExpEmpty) sig_i = 0;
        bad_i = JF(badA)[i] != 0;
      }
      double* crow = JF(C) + (n0 + col0) * JF(ldc) + i;
      const int64_t cols_left = JF(n) - n0 - col0;  // columns of this thread's part inside C
      // split items: this thread's elements of the tile's group sums for the item's segment
      unsigned long long* ysum_seg =
          split ? p.ysum + ((int64_t)tile * p.nsegs + seg) * p.ngroups * (kBM * BN) + (int64_t)col0 * kBM + row
                : nullptr;
      bool first = true;
      for (int seg0 = kb0; seg0 < kb1; seg0 += kSegBlocks) {
        const int segn = min(kSegBlocks, kb1 - seg0);
        for (int h = j.s + 1; h >= 2; h -= kGroupLevels) {
          const int glo = group_high(h);
          for (int g = h; g >= glo; --g) {
            const int nch = chunks_of(g, segn);
            const int l = h - g;  // Y holds sum_l P_l 2^(b l)
#pragma unroll
            for (int c = 0; c < kCols; ++c) acc[c] = 0u;
            for (int ci = 0; ci < nch; ++ci, ++chunk) {
              const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
              mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
              tc_fence_after();
              const uint32_t taddr = trow + buf * BN + col0;
#pragma unroll
              for (int q = 0; q < kCols / 16; ++q) {
                uint32_t v[16];
                tmem_ld_16(taddr + q * 16, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) acc[q * 16 + jj] += (uint32_t)__float2int_rn(__uint_as_float(v[jj]));
              }
              tc_fence_before();
              mbar_arrive(&acc_empty[buf]);
            }
            if (g != glo) {
              // fold this level into Y (the loads are unconditional: no branch around warp-wide TMEM access)
#pragma unroll
              for (int q = 0; q < kCols / 8; ++q) {
                uint32_t lo[8], hi[8];
                tmem_ld_8(y_lo + q * 8, lo);
                tmem_ld_8(y_hi + q * 8, hi);
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                  const int64_t add = (int64_t)(int32_t)acc[q * 8 + jj] * ((int64_t)1 << (kDigitBits * l));
                  const int64_t y = (l > 0 ? (int64_t)(((uint64_t)hi[jj] << 32) | lo[jj]) : 0) + add;
                  lo[jj] = (uint32_t)y;
                  hi[jj] = (uint32_t)((uint64_t)y >> 32);
                }
                tmem_st_8(y_lo + q * 8, lo);
                tmem_st_8(y_hi + q * 8, hi);
              }
              tmem_wait_st();
              continue;
            }
            if (split) {
              // group end of a split item: add this sub-range's exact group sums into the tile's
              // (64-bit integer additions: the total does not depend on the order of the items)
              unsigned long long* yg = ysum_seg + (int64_t)((j.s + 1 - h) / kGroupLevels) * (kBM * BN);
#pragma unroll
              for (int q = 0; q < kCols / 8; ++q) {
                uint32_t lo[8], hi[8];
                tmem_ld_8(y_lo + q * 8, lo);
                tmem_ld_8(y_hi + q * 8, hi);
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                  const int64_t add = (int64_t)(int32_t)acc[q * 8 + jj] * ((int64_t)1 << (kDigitBits * l));
                  const int64_t y = (l > 0 ? (int64_t)(((uint64_t)hi[jj] << 32) | lo[jj]) : 0) + add;
                  atomicAdd(yg + (int64_t)(q * 8 + jj) * kBM, (unsigned long long)y);
                }
              }
              continue;
            }
            // group end: C := fma(alpha 2^(tau_j - h b), Y 2^sigma_i, C)
            epi_bar_sync<kEpiWarps1>();  // the previous group's readers of colscale are done
            {
              const int idx = ew * 32 + lane;
              if (idx < BN) {
                const int64_t jc = n0 + idx;
                double cs = 0.0;
                if (jc < JF(n)) {
                  int tau = JF(sigB)[jc];
                  if (tau == kExpEmpty) tau = 0;
                  cs = JF(badB)[jc] ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(JF(alpha), tau - h * kDigitBits);
                }
                colscale[idx] = cs;
              }
            }
            epi_bar_sync<kEpiWarps1>();
            const double beta = JF(beta);
            const int64_t ldc = JF(ldc);
            const bool read_c = !(first && beta == 0.0);
#pragma unroll
            for (int q = 0; q < kCols / 8; ++q) {
              double w[8];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {  // all 8 loads in flight before any use
                const int c = q * 8 + jj;
                w[jj] = (read_c && row_ok && c < cols_left) ? crow[(int64_t)c * ldc] : 0.0;
              }
              uint32_t lo[8], hi[8];
              tmem_ld_8(y_lo + q * 8, lo);
              tmem_ld_8(y_hi + q * 8, hi);
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int c = q * 8 + jj;
                const int64_t add = (int64_t)(int32_t)acc[c] * ((int64_t)1 << (kDigitBits * l));
                const int64_t y = (l > 0 ? (int64_t)(((uint64_t)hi[jj] << 32) | lo[jj]) : 0) + add;
                const double wp = first ? (beta == 0.0 ? 0.0 : beta * w[jj]) : w[jj];
                const double x = bad_i ? __longlong_as_double(0x7FF8000000000000ll) : scaled_i64(y, sig_i);
                if (row_ok && c < cols_left) crow[(int64_t)c * ldc] = fma(colscale[col0 + c], x, wp);
              }
            }
            first = false;
          }
        }
      }
      if (!split) continue;
      // ---- split item done: the tile's last item applies the summed groups to C ----
      __threadfence();  // this item's additions are visible before it is counted
      epi_bar_sync<kEpiWarps1>();
      if (ew == 0 && lane == 0)
        *last_flag = atomicAdd(p.tile_done + tile, 1u) == (unsigned)(p.nsegs * p.splits - 1) ? 1 : 0;
      epi_bar_sync<kEpiWarps1>();
      if (!*last_flag) continue;
      __threadfence();
      {
        const int idx = ew * 32 + lane;  // colscale of every group: alpha 2^(tau_j - 7h)
        if (idx < BN) {
          const int64_t jc = n0 + idx;
          int tau = 0;
          bool badc = false;
          if (jc < p.n) {
            tau = p.sigB[jc] == kExpEmpty ? 0 : p.sigB[jc];
            badc = p.badB[jc] != 0;
          }
          for (int gi = 0; gi < p.ngroups; ++gi) {
            const int h = j.s + 1 - gi * kGroupLevels;
            colscale[gi * BN + idx] = jc >= p.n ? 0.0
                                      : badc   ? __longlong_as_double(0x7FF8000000000000ll)
                                               : ldexp(p.alpha, tau - h * kDigitBits);
          }
        }
      }
      epi_bar_sync<kEpiWarps1>();
      // W := beta*C0, then W := fma(alpha 2^(tau_j - 7h), Y 2^sigma_i, W) for every segment and
      // group in order, as an unsplit tile does
      const unsigned long long* ytile = p.ysum + (int64_t)tile * p.nsegs * p.ngroups * (kBM * BN) +
                                        (int64_t)col0 * kBM + row;
#pragma unroll 1
      for (int q = 0; q < kCols / 8; ++q) {
        double w[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int c = q * 8 + jj;
          w[jj] = (p.beta != 0.0 && row_ok && c < cols_left) ? p.beta * crow[(int64_t)c * p.ldc] : 0.0;
        }
        for (int sg = 0; sg < p.nsegs; ++sg)
          for (int gi = 0; gi < p.ngroups; ++gi) {
            const unsigned long long* yg = ytile + (int64_t)(sg * p.ngroups + gi) * (kBM * BN) + (int64_t)q * 8 * kBM;
            int64_t y[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) y[jj] = (int64_t)__ldcg(yg + (int64_t)jj * kBM);
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const double x = bad_i ? __longlong_as_double(0x7FF8000000000000ll) : scaled_i64(y[jj], sig_i);
              w[jj] = fma(colscale[gi * BN + col0 + q * 8 + jj], x, w[jj]);
            }
          }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int c = q * 8 + jj;
          if (row_ok && c < cols_left) crow[(int64_t)c * p.ldc] = w[jj];
        }
      }
      epi_bar_sync<kEpiWarps1>();  // colscale and the flag are rewritten by the next item
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

// =====================================================================================
// Two-SM variant (tcgen05 cta_group::2): a CTA pair computes a 256 x 256 tile, each
// SM holding 128 rows x 256 columns in its TMEM (two accumulators of 256 columns).
// Each CTA loads its own 128 rows of the A slice and 128 of the 256 rows of the B
// slice; the leader's MMA reads both CTAs' shared memory.  Between level
// groups the FP64 running sum of each CTA's 128 x 256 block lives in a private
// scratch slot of the workspace, laid out so that every warp access is 256
// contiguous bytes and each warp sweeps 32 KiB in order; C itself is read once
// (beta*C0) and written once per tile.
// =====================================================================================
constexpr int k2Stages = 6;
constexpr int k2BM = 256;  // pair tile rows (128 per CTA)
constexpr int k2BN = 256;  // pair tile columns (128 rows of op(B)^T loaded per CTA)
constexpr int k2ColsPerThread = 128;

struct Smem2 {
  static constexpr int kABytes = 128 * kBK * 2;  // 16 KiB
  static constexpr int kBBytes = 128 * kBK * 2;  // 16 KiB
  static constexpr int kOffA = 0;
  static constexpr int kOffB = kOffA + k2Stages * kABytes;
  static constexpr int kOffBar = kOffB + k2Stages * kBBytes;
  static constexpr int kNumBars = 2 * k2Stages + 5;
  static constexpr int kOffTmemSlot = kOffBar + kNumBars * 8;
  static constexpr int kOffScale = (kOffTmemSlot + 16 + 15) / 16 * 16;
  static constexpr int kBytes = kOffScale + 2 * k2BN * 8;  // two colscale buffers
  static constexpr int kAlloc = kBytes + 1024;
};

template <bool TABLE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_slice_gemm_pair(const Args p, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const EmuTableEntry* __restrict__ table, int count, int total_tiles) {
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
  double* colscale = reinterpret_cast<double*>(smem + L::kOffScale);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int s = p.slices;  // one launch per slice count, also for a table of problems
  const int num_pairs = gridDim.x / 2, pair_id = blockIdx.x / 2;
  const int ntiles = TABLE ? total_tiles : p.num_tiles;

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
      mbar_init(&acc_empty[i], 2 * 32 * kEpiWarps);  // every epilogue thread of both CTAs
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(kTmemCols)
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
      int cur = 0;
      for (int tile = pair_id; tile < ntiles; tile += num_pairs) {
        Job j;
        get_job<k2BM, k2BN, TABLE>(p, table, count, tile, cur, j);
        const CUtensorMap* mapA = TABLE ? &j.e->tmA : &tmA;
        const CUtensorMap* mapB = TABLE ? &j.e->tmB : &tmB;
        if (TABLE) {  // maps written into global memory before the launch: acquire them for the TMA unit
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapA) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mapB) : "memory");
        }
        const int m0 = j.m0 + (int)rank * 128;
        const int nb0 = j.n0 + (int)rank * 128;
        for (int seg0 = 0; seg0 < j.nkb; seg0 += kSegBlocks) {
          const int segn = min(kSegBlocks, j.nkb - seg0);
          for (int h = s + 1; h >= 2; h -= kGroupLevels)
            for (int g = h; g >= group_high(h); --g)
              for (int kb = seg0; kb < seg0 + segn; ++kb)  // k-major: tiles in flight share a narrow k window in L2
                for (int t = 1; t <= g - 1; ++t) {
                  mbar_wait_cluster(&empty[stage], phase ^ 1u, p.err, kErrWaitSlot);
                  if (leader) mbar_arrive_expect_tx(&full[stage], pair_bytes);
                  const uint32_t fbar = map_to_rank(smem_u32(&full[stage]), 0);
                  tma_load_3d_pair(smem + L::kOffA + stage * L::kABytes, mapA, fbar, kb * kBK, m0, t - 1);
                  tma_load_3d_pair(smem + L::kOffB + stage * L::kBBytes, mapB, fbar, kb * kBK, nb0, g - t - 1);
                  if (++stage == k2Stages) { stage = 0; phase ^= 1u; }
                }
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
      int cur = 0;
      for (int tile = pair_id; tile < ntiles; tile += num_pairs) {
        Job j;
        get_job<k2BM, k2BN, TABLE>(p, table, count, tile, cur, j);
        for (int seg0 = 0; seg0 < j.nkb; seg0 += kSegBlocks)
          for (int h = s + 1; h >= 2; h -= kGroupLevels)
          for (int g = h; g >= group_high(h); --g) {
            const int segn = min(kSegBlocks, j.nkb - seg0);
            const int items = (g - 1) * segn;
            for (int i0 = 0; i0 < items; i0 += kChunkBlocks, ++chunk) {
              const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
              mbar_wait_cluster(&acc_empty[buf], cph ^ 1u, p.err, kErrWaitEpi);
              tc_fence_after();
              const uint32_t dtm = tmem_base + buf * k2BN;
              const int i1 = min(items, i0 + kChunkBlocks);
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
      }
      umma_commit_pair(done);
      mbar_wait_cluster(done, 0, p.err, kErrWaitMma);
    }
    __syncwarp();
  } else {
    // ------------------------------ epilogue (both CTAs) ------------------------------
    // Each finished level's integer sums are parked in scratch; the FP64 update of a
    // finished group of levels is deferred and folded into the running sums a few
    // columns at a time while the next group's chunks are drained, so the MMA never
    // waits for it.  Two sets of park slots hold the group being drained and the
    // pending one.
    constexpr int kStep = 4;  // columns per step of the pending update
    constexpr int64_t kSlot = (int64_t)128 * k2BN;  // one parked level of the CTA's block
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int half = ew >> 2;
    const int row = quad * 32 + lane;
    const int col0 = half * k2ColsPerThread;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    // this thread's column sweep in the CTA's scratch slots: 256 (or 128) contiguous bytes per warp per column
    const int64_t within = (int64_t)((half * 4 + quad) * k2ColsPerThread) * 32 + lane;
    double* scrW = p.scratch + (int64_t)blockIdx.x * kSlot + within;
    int32_t* scrP = p.scratch_p + (int64_t)blockIdx.x * (kParkSlots * kSlot) + within;
    uint32_t chunk = 0;
    uint32_t acc[k2ColsPerThread];
    uint32_t empty_remote[2];
    empty_remote[0] = map_to_rank(smem_u32(&acc_empty[0]), 0);
    empty_remote[1] = map_to_rank(smem_u32(&acc_empty[1]), 0);
    // the pending update
    bool pd_active = false, pd_first = false, pd_last = false, pd_bad = false, pd_row_ok = false;
    int pd_done = 0, pd_sig = 0, pd_buf = 0, pd_set = 0, pd_nlev = 0, cs_next = 0, park_set = 0;
    double pd_beta = 0.0;
    double* pd_crow = nullptr;
    int64_t pd_ldc = 0, pd_cols_left = 0;  // columns of the pending tile inside C (n - n0 - col0, clamped)
    // kStep columns per step: all their loads are issued before any is used
    auto advance = [&](int ncols) {
      const int c1 = min(pd_done + ncols, k2ColsPerThread);
      const double* cs = colscale + pd_buf * k2BN + col0;
      const int32_t* pk = scrP + (int64_t)pd_set * kGroupLevels * kSlot;
      for (int c = pd_done; c < c1; c += kStep) {
        double w[kStep];
        int32_t P[kStep][kGroupLevels];
#pragma unroll
        for (int u = 0; u < kStep; ++u) {
          const bool in = c + u < c1;
          const bool col_ok = in && pd_row_ok && c + u < pd_cols_left;
          if (pd_first) w[u] = (pd_beta != 0.0 && col_ok) ? pd_crow[(int64_t)(c + u) * pd_ldc] : 0.0;
          else w[u] = in ? scrW[(c + u) * 32] : 0.0;
#pragma unroll
          for (int l = 0; l < kGroupLevels; ++l) P[u][l] = (in && l < pd_nlev) ? pk[l * kSlot + (c + u) * 32] : 0;
        }
#pragma unroll
        for (int u = 0; u < kStep; ++u) {
          if (c + u >= c1) continue;
          const bool col_ok = pd_row_ok && c + u < pd_cols_left;
          const double wp = pd_first ? (pd_beta != 0.0 && col_ok ? pd_beta * w[u] : 0.0) : w[u];
          const double x =
              pd_bad ? __longlong_as_double(0x7FF8000000000000ll) : scaled_i64(combine_levels(P[u]), pd_sig);
          const double r = fma(cs[c + u], x, wp);
          if (pd_last) {
            if (col_ok) pd_crow[(int64_t)(c + u) * pd_ldc] = r;
          } else {
            scrW[(c + u) * 32] = r;
          }
        }
      }
      pd_done = c1;
      if (pd_done >= k2ColsPerThread) pd_active = false;
    };
    int cur = 0;
    for (int tile = pair_id; tile < ntiles; tile += num_pairs) {
      Job j;
      get_job<k2BM, k2BN, TABLE>(p, table, count, tile, cur, j);
      const int64_t m0 = (int64_t)j.m0 + rank * 128;
      const int64_t n0 = j.n0;
      const int64_t i = m0 + row;
      const bool row_ok = i < JF(m);
      int sig_i = 0;
      bool bad_i = false;
      if (row_ok) {
        sig_i = JF(sigA)[i];
        if (sig_i == kExpEmpty) sig_i = 0;
        bad_i = JF(badA)[i] != 0;
      }
      bool first = true;
      for (int seg0 = 0; seg0 < j.nkb; seg0 += kSegBlocks) {
        const int segn = min(kSegBlocks, j.nkb - seg0);
        for (int h = s + 1; h >= 2; h -= kGroupLevels) {
          const int glo = group_high(h);
          const bool last = (glo == 2) && (seg0 + kSegBlocks >= j.nkb);
          int gch = 0;  // chunks of this group: the pending update is spread over them
          for (int g = h; g >= glo; --g) gch += chunks_of(g, segn);
          const int portion = ((k2ColsPerThread + gch - 1) / gch + kStep - 1) / kStep * kStep;
          for (int g = h; g >= glo; --g) {
            const int nch = chunks_of(g, segn);
#pragma unroll
            for (int c = 0; c < k2ColsPerThread; ++c) acc[c] = 0u;
            for (int ci = 0; ci < nch; ++ci, ++chunk) {
              const uint32_t buf = chunk & 1u, cph = (chunk >> 1) & 1u;
              mbar_wait(&acc_full[buf], cph, p.err, kErrWaitMma);
              tc_fence_after();
              const uint32_t taddr = tmem_base + lane_base + buf * k2BN + col0;
#pragma unroll
              for (int q = 0; q < k2ColsPerThread / 16; ++q) {
                uint32_t v[16];
                tmem_ld_16(taddr + q * 16, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[q * 16 + j] += (uint32_t)__float2int_rn(__uint_as_float(v[j]));
              }
              tc_fence_before();
              mbar_arrive_remote(empty_remote[buf]);
              if (pd_active) advance(portion);
            }
            int32_t* dst = scrP + (int64_t)(park_set * kGroupLevels + (h - g)) * kSlot;
#pragma unroll
            for (int c = 0; c < k2ColsPerThread; ++c) dst[c * 32] = (int32_t)acc[c];
          }
          // group end: finish the previous pending update, then make this group pending
          if (pd_active) advance(k2ColsPerThread);
          epi_bar_sync();  // nobody reads the colscale buffer about to be rewritten
          {
            const int idx = ew * 32 + lane;
            if (idx < k2BN) {
              const int64_t jc = n0 + idx;
              double cs = 0.0;
              if (jc < JF(n)) {
                int tau = JF(sigB)[jc];
                if (tau == kExpEmpty) tau = 0;
                cs = JF(badB)[jc] ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(JF(alpha), tau - h * kDigitBits);
              }
              colscale[cs_next * k2BN + idx] = cs;
            }
          }
          epi_bar_sync();
          pd_active = true;
          pd_done = 0;
          pd_first = first;
          pd_last = last;
          pd_bad = bad_i;
          pd_row_ok = row_ok;
          pd_sig = sig_i;
          pd_buf = cs_next;
          pd_set = park_set;
          pd_nlev = h - glo + 1;
          pd_beta = JF(beta);
          pd_ldc = JF(ldc);
          pd_crow = JF(C) + (n0 + col0) * pd_ldc + i;
          pd_cols_left = JF(n) - n0 - col0;
          cs_next ^= 1;
          park_set ^= 1;
          first = false;
        }
      }
    }
    if (pd_active) advance(k2ColsPerThread);  // the last group of the last tile
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA leaves while the pair still uses its shared memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "n"(kTmemCols)
                 : "memory");
  }
}

int launch_pair(const GemmParams& gp, const Workspace& ws, int sms, cudaStream_t stream) {
  using L = Smem2;
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const uint64_t dA[3] = {(uint64_t)gp.k, (uint64_t)gp.m, (uint64_t)gp.slices};
  const uint64_t pA[2] = {(uint64_t)ws.kp * 2, (uint64_t)gp.m * ws.kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, 128u, 1u};
  int rc = encode_tmap(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)gp.k, (uint64_t)gp.n, (uint64_t)gp.slices};
  const uint64_t pB[2] = {(uint64_t)ws.kp * 2, (uint64_t)gp.n * ws.kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, 128u, 1u};
  rc = encode_tmap(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;

  Args a;
  memset(&a, 0, sizeof(a));
  a.m = gp.m; a.n = gp.n; a.k = gp.k;
  a.slices = gp.slices;
  a.nkb = (int)((gp.k + kBK - 1) / kBK);
  a.tiles_m = (int)((gp.m + k2BM - 1) / k2BM);
  const int64_t tiles = (int64_t)a.tiles_m * ((gp.n + k2BN - 1) / k2BN);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  int64_t pairs = tiles < sms / 2 ? tiles : sms / 2;
  if (pairs > ws.scratch_ctas / 2) pairs = ws.scratch_ctas / 2;
  if (pairs < 1) return set_error(GBD_ERR_WORKSPACE, "no scratch slot for the two-SM kernel");
  a.group_m = group_rows((int)pairs, k2BM, k2BN, a.tiles_m);
  a.alpha = gp.alpha; a.beta = gp.beta;
  a.C = gp.C; a.ldc = gp.ldc;
  a.sigA = gp.sigA; a.sigB = gp.sigB; a.badA = gp.badA; a.badB = gp.badB;
  a.scratch = ws.scratch;
  a.scratch_p = ws.scratch_p;
  a.err = device_error_word();

  cudaError_t e =
      cudaFuncSetAttribute(k_slice_gemm_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(slice gemm pair)");
  k_slice_gemm_pair<false><<<(unsigned)(2 * pairs), kThreads, L::kAlloc, stream>>>(a, tmA, tmB, nullptr, 0, 0);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "slice gemm pair launch");
}

template <int BN>
int launch_bn(const GemmParams& gp, const Workspace& ws, int sms, cudaStream_t stream) {
  using L = SmemLayout<BN>;
  CUtensorMap tmA, tmB;
  memset(&tmA, 0, sizeof(tmA));
  memset(&tmB, 0, sizeof(tmB));
  const uint64_t dA[3] = {(uint64_t)gp.k, (uint64_t)gp.m, (uint64_t)gp.slices};
  const uint64_t pA[2] = {(uint64_t)ws.kp * 2, (uint64_t)gp.m * ws.kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, (uint32_t)kBM, 1};
  int rc = encode_tmap(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)gp.k, (uint64_t)gp.n, (uint64_t)gp.slices};
  const uint64_t pB[2] = {(uint64_t)ws.kp * 2, (uint64_t)gp.n * ws.kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, (uint32_t)BN, 1};
  rc = encode_tmap(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;

  Args a;
  memset(&a, 0, sizeof(a));
  a.m = gp.m; a.n = gp.n; a.k = gp.k;
  a.slices = gp.slices;
  a.nkb = (int)((gp.k + kBK - 1) / kBK);
  a.tiles_m = (int)((gp.m + kBM - 1) / kBM);
  const int64_t tiles = (int64_t)a.tiles_m * ((gp.n + BN - 1) / BN);
  if (tiles > (int64_t)1 << 30) return set_error(GBD_ERR_LIMIT, "too many output tiles");
  a.num_tiles = (int)tiles;
  int grid = (int)(tiles < sms ? tiles : sms);
  a.group_m = group_rows(grid, kBM, BN, a.tiles_m);
  a.alpha = gp.alpha; a.beta = gp.beta;
  a.C = gp.C; a.ldc = gp.ldc;
  a.sigA = gp.sigA; a.sigB = gp.sigB; a.badA = gp.badA; a.badB = gp.badB;
  a.scratch = nullptr;
  a.scratch_p = nullptr;
  a.err = device_error_word();
  // split inner dimension for few tiles (the workspace holds the sums; see split_count)
  a.splits = ws.splits;
  a.nsegs = (a.nkb + kSegBlocks - 1) / kSegBlocks;
  a.ngroups = (gp.slices + kGroupLevels - 1) / kGroupLevels;
  a.ysum = ws.ysum;
  a.tile_done = ws.tile_done;
  if (a.splits > 1) {
    const int64_t items = tiles * a.nsegs * a.splits;
    grid = (int)(items < sms ? items : sms);
  }

  auto kern = k_slice_gemm<BN, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(slice gemm)");
  kern<<<grid, kThreads1, L::kAlloc, stream>>>(a, tmA, tmB, nullptr, 0, 0);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "slice gemm launch");
}

}  // namespace

int encode_slice_maps(const Workspace& ws, int64_t m, int64_t n, int64_t k, int slices, EmuTableEntry* e) {
  const uint64_t dA[3] = {(uint64_t)k, (uint64_t)m, (uint64_t)slices};
  const uint64_t pA[2] = {(uint64_t)ws.kp * 2, (uint64_t)m * ws.kp * 2};
  const uint32_t bA[3] = {(uint32_t)kBK, (uint32_t)kBM, 1u};
  int rc = encode_tmap(&e->tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DA, dA, pA, bA, CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  const uint64_t dB[3] = {(uint64_t)k, (uint64_t)n, (uint64_t)slices};
  const uint64_t pB[2] = {(uint64_t)ws.kp * 2, (uint64_t)n * ws.kp * 2};
  const uint32_t bB[3] = {(uint32_t)kBK, (uint32_t)kGroupedBN, 1u};
  return encode_tmap(&e->tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws.DB, dB, pB, bB, CU_TENSOR_MAP_SWIZZLE_128B);
}

int launch_slice_gemm_grouped(const EmuTableEntry* table_dev, int count, int total_tiles, int slices,
                              cudaStream_t stream) {
  using L = SmemLayout<kGroupedBN>;
  if (count <= 0 || total_tiles <= 0) return GBD_OK;
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  Args a;
  memset(&a, 0, sizeof(a));
  a.err = device_error_word();
  a.slices = slices;
  auto kern = k_slice_gemm<kGroupedBN, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped slice gemm)");
  const int grid = total_tiles < sms ? total_tiles : sms;
  kern<<<grid, kThreads1, L::kAlloc, stream>>>(a, dummy, dummy, table_dev, count, total_tiles);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "grouped slice gemm launch");
}

int launch_slice_gemm_grouped_pair(const EmuTableEntry* table_dev, int count, int total_tiles, int slices,
                                   double* scratch, int32_t* scratch_p, int max_ctas, cudaStream_t stream) {
  using L = Smem2;
  if (count <= 0 || total_tiles <= 0) return GBD_OK;
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof(dummy));
  Args a;
  memset(&a, 0, sizeof(a));
  a.err = device_error_word();
  a.slices = slices;
  a.scratch = scratch;
  a.scratch_p = scratch_p;
  int pairs = total_tiles < sms / 2 ? total_tiles : sms / 2;
  if (pairs > max_ctas / 2) pairs = max_ctas / 2;
  if (pairs < 1) return set_error(GBD_ERR_WORKSPACE, "no scratch slot for the grouped two-SM kernel");
  cudaError_t e =
      cudaFuncSetAttribute(k_slice_gemm_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kAlloc);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped slice gemm pair)");
  k_slice_gemm_pair<true><<<(unsigned)(2 * pairs), kThreads, L::kAlloc, stream>>>(a, dummy, dummy, table_dev, count,
                                                                                  total_tiles);
  e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, "grouped slice gemm pair launch");
}

// Throughput per SM of the two-SM 256 x 256 kernel relative to the one-SM 128 x 128 kernel, as
// a function of k, measured on GB300 with every SM busy (2048 x 2048 outputs, 8 slices).  The
// two-SM kernel moves half the operand bytes per flop but pays for its deferred FP64 update
// per tile, which only a deep inner dimension amortises.
double pair_gain(int64_t k) {
  static const double lk[] = {7, 8, 9, 10, 11, 12, 13};                    // log2 k
  static const double gain[] = {0.42, 0.51, 0.69, 0.98, 1.29, 1.56, 1.80};  // 8192: from the 8192^3 runs
  const double x = log2((double)(k > 1 ? k : 1));
  if (x <= lk[0]) return gain[0];
  for (int i = 1; i < 7; ++i)
    if (x <= lk[i]) return gain[i - 1] + (gain[i] - gain[i - 1]) * (x - lk[i - 1]) / (lk[i] - lk[i - 1]);
  return gain[6];
}

int launch_slice_gemm(const GemmParams& gp, const Workspace& ws, cudaStream_t stream) {
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  if (gp.m == 0 || gp.n == 0) return GBD_OK;
  // GBD_EMU_KERNEL=pair|single overrides the choice below (tests and tuning)
  const char* force = getenv("GBD_EMU_KERNEL");
  if (force && force[0] == 'p') return launch_pair(gp, ws, sms, stream);
  const bool single = force && force[0] == 's';
  // Expected time of each kernel in units of one 128 x 128 tile on one SM: whole waves of tiles
  // over the SMs (or SM pairs), a 256 x 256 tile being four units on two SMs at pair_gain(k).
  const int64_t tiles = ((gp.m + kBM - 1) / kBM) * ((gp.n + kBM - 1) / kBM);
  const int64_t pair_tiles = ((gp.m + k2BM - 1) / k2BM) * ((gp.n + k2BN - 1) / k2BN);
  const int64_t pairs = sms / 2 > 0 ? sms / 2 : 1;
  const double t_one = (double)((tiles + sms - 1) / sms);
  const double t_pair = (double)((pair_tiles + pairs - 1) / pairs) * 2.0 / pair_gain(gp.k);
  if (!single && t_pair < t_one) return launch_pair(gp, ws, sms, stream);
  return launch_bn<128>(gp, ws, sms, stream);
}

}  // namespace emu
}  // namespace gbd
