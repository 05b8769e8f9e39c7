// native_tile.cuh -- one output tile of the native FP64-MMA DGEMM, shared by the
// single-problem kernel (native.cu) and the persistent grouped kernel (grouped.cu).
//
// C := alpha*op(A)*op(B) + beta*C  (BLAS dgemm, paper Section 1.2), column-major
// with leading dimensions (Section 2.1).  FP64 arithmetic runs on a low-rate unit
// on GB300 (about 1.05 TFLOP/s for both mma.sync f64 and DFMA), so the tile is
// bound by the FP64 pipe; the staging and epilogue only have to stay out of its way.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace gbd {

struct NativeArgs {
  int64_t m, n, k;
  double alpha, beta;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  unsigned int* err;
  int vec_c;  // C and ldc allow 16-byte stores at even rows
};

constexpr int kNativeThreads = 128;
constexpr int kNativeBK = 16;
constexpr int kNativeStages = 4;

template <int BM, int BN>
constexpr size_t native_smem_bytes() {
  return (size_t)kNativeStages * (BM * kNativeBK + kNativeBK * BN) * sizeof(double) + kNativeStages * sizeof(uint64_t);
}

// One part of a tile whose inner dimension is split (grouped problems with a small output
// and a deep k): the part's k-blocks [kb0, kb1), its slot of BM x BN doubles in `part` (the
// tile's `parts` slots in part order) and the tile's arrival counter.  The last part to
// arrive adds the slots in part order, so the sum is the same whatever order the parts run in,
// applies the epilogue and clears the counter for the next run.
struct KSplit {
  int kb0, kb1;
  int parts, index;
  double* part;
  unsigned int* done;
};

// One BM x BN tile of C at (m0, n0): staged mainloop and fused epilogue.  Shared by
// the single-problem kernel and the persistent grouped kernel (grouped.cu), so a
// problem gets the same bits alone and inside a batch.
template <bool TA, bool TB, int BM, int BN, bool USE_TMA>
__device__ __forceinline__ void native_tile(const NativeArgs& p, const CUtensorMap* tmA_p,
                                            const CUtensorMap* tmB_p, int64_t m0, int64_t n0,
                                            unsigned char* smem_raw, const KSplit* ks = nullptr) {
  constexpr int A_EL = BM * kNativeBK, B_EL = kNativeBK * BN;
  constexpr int WM = BM / 2, WN = BN / 2, MI = WM / 16, NI = WN / 8;
  static_assert(MI >= 1 && NI >= 1, "warp tile too small");
  double* sA = reinterpret_cast<double*>(smem_raw);  // [kNativeStages][A_EL]
  double* sB = sA + kNativeStages * A_EL;                  // [kNativeStages][B_EL]
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kNativeStages * B_EL);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  // the k-blocks of this tile (all of them, or one part's)
  const int kbase = ks ? ks->kb0 : 0;
  const int nkb = ks ? ks->kb1 - ks->kb0 : (int)((p.k + kNativeBK - 1) / kNativeBK);
  const int wm0 = (warp >> 1) * WM, wn0 = (warp & 1) * WN;

  __syncthreads();  // the shared memory of a previous tile is no longer in use
  if (USE_TMA && tid == 0) {
    tma_prefetch_desc(tmA_p);
    tma_prefetch_desc(tmB_p);
    for (int s = 0; s < kNativeStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // stage kb of the tile's k loop into ring slot kb % kNativeStages
  auto issue = [&](int kb) {
    const int s = kb % kNativeStages;
    const int64_t k0 = (int64_t)(kbase + kb) * kNativeBK;
    if (USE_TMA) {
      if (tid == 0 && kb < nkb) {
        mbar_arrive_expect_tx(&full[s], (uint32_t)((A_EL + B_EL) * sizeof(double)));
        if (!TA) tma_load_2d(sA + s * A_EL, tmA_p, &full[s], (int)m0, (int)k0);
        else tma_load_2d(sA + s * A_EL, tmA_p, &full[s], (int)k0, (int)m0);
        if (!TB) tma_load_2d(sB + s * B_EL, tmB_p, &full[s], (int)k0, (int)n0);
        else tma_load_2d(sB + s * B_EL, tmB_p, &full[s], (int)n0, (int)k0);
      }
    } else {
      if (kb < nkb) {
        double* a_s = sA + s * A_EL;
        double* b_s = sB + s * B_EL;
        for (int idx = tid; idx < A_EL; idx += kNativeThreads) {
          int i, pk;
          if (!TA) { i = idx % BM; pk = idx / BM; }  // smem [BK][BM]
          else { pk = idx % kNativeBK; i = idx / kNativeBK; }    // smem [BM][BK]
          const int64_t gi = m0 + i, gp = k0 + pk;
          const bool ok = gi < p.m && gp < p.k;
          const double* src = ok ? (TA ? p.A + gi * p.lda + gp : p.A + gp * p.lda + gi) : p.A;
          cp_async_8(a_s + idx, src, ok);
        }
        for (int idx = tid; idx < B_EL; idx += kNativeThreads) {
          int j, pk;
          if (!TB) { pk = idx % kNativeBK; j = idx / kNativeBK; }  // smem [BN][BK]
          else { j = idx % BN; pk = idx / BN; }        // smem [BK][BN]
          const int64_t gj = n0 + j, gp = k0 + pk;
          const bool ok = gj < p.n && gp < p.k;
          const double* src = ok ? (TB ? p.B + gp * p.ldb + gj : p.B + gj * p.ldb + gp) : p.B;
          cp_async_8(b_s + idx, src, ok);
        }
      }
      cp_async_commit();  // one group per stage, empty past the end, keeps the count uniform
    }
  };

  double acc[MI][NI][4];
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.0;

  for (int kb = 0; kb < kNativeStages - 1; ++kb) issue(kb);

  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb % kNativeStages;
    if (USE_TMA) mbar_wait(&full[s], (uint32_t)((kb / kNativeStages) & 1), p.err, kErrWaitTma);
    else cp_async_wait<kNativeStages - 2>();
    __syncthreads();  // tile kb visible to all; slot (kb-1) % kNativeStages no longer read
    issue(kb + kNativeStages - 1);

    const double* a_s = sA + s * A_EL;
    const double* b_s = sB + s * B_EL;
#pragma unroll
    for (int kk = 0; kk < kNativeBK; kk += 16) {
      double af[MI][8], bf[NI][4];
#pragma unroll
      for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = wm0 + mi * 16 + g + 8 * (q & 1);
          const int pk = kk + t + 4 * (q >> 1);
          af[mi][q] = TA ? a_s[i * kNativeBK + pk] : a_s[pk * BM + i];
        }
#pragma unroll
      for (int ni = 0; ni < NI; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = wn0 + ni * 8 + g;
          const int pk = kk + t + 4 * q;
          bf[ni][q] = TB ? b_s[pk * BN + j] : b_s[j * kNativeBK + pk];
        }
#pragma unroll
      for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < NI; ++ni) dmma_16x8x16(acc[mi][ni], af[mi], bf[ni]);
    }
  }

  // ---- fused epilogue through shared memory, column by column ----
  __syncthreads();  // every load was consumed; the ring is free
  constexpr int LDS = BM + 2;
  double* sC = reinterpret_cast<double*>(smem_raw);  // [BN][LDS], column-major tile
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni) {
      const int r = wm0 + mi * 16 + g, c = wn0 + ni * 8 + 2 * t;
      sC[c * LDS + r] = acc[mi][ni][0];
      sC[(c + 1) * LDS + r] = acc[mi][ni][1];
      sC[c * LDS + r + 8] = acc[mi][ni][2];
      sC[(c + 1) * LDS + r + 8] = acc[mi][ni][3];
    }
  __syncthreads();
  if (ks) {
    // this part's sums into its slot; the last part to arrive adds all slots in part order
    __shared__ unsigned int s_last;
    double* mine = ks->part + (int64_t)ks->index * BM * BN;
    for (int idx = tid; idx < BM * BN; idx += kNativeThreads) mine[idx] = sC[(idx / BM) * LDS + idx % BM];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(ks->done, 1u) == (unsigned)(ks->parts - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int idx = tid; idx < BM * BN; idx += kNativeThreads) {
      double v = __ldcg(ks->part + idx);
      for (int q = 1; q < ks->parts; ++q) v += __ldcg(ks->part + (int64_t)q * BM * BN + idx);
      sC[(idx / BM) * LDS + idx % BM] = v;
    }
    if (tid == 0) *ks->done = 0u;  // ready for the next run of the plan
    __syncthreads();
  }
  const double alpha = p.alpha, beta = p.beta;
  for (int jj = warp; jj < BN; jj += kNativeThreads / 32) {
    const int64_t j = n0 + jj;
    if (j >= p.n) break;
    double* ccol = p.C + j * p.ldc;
    for (int ii = 2 * lane; ii < BM; ii += 64) {
      const int64_t i = m0 + ii;
      if (i >= p.m) break;
      const double v0 = sC[jj * LDS + ii], v1 = sC[jj * LDS + ii + 1];
      if (p.vec_c && i + 1 < p.m) {
        double2* dst = reinterpret_cast<double2*>(ccol + i);
        double2 out;
        if (beta == 0.0) {
          out.x = alpha * v0;
          out.y = alpha * v1;
        } else {
          const double2 c0 = *dst;
          out.x = fma(alpha, v0, beta * c0.x);
          out.y = fma(alpha, v1, beta * c0.y);
        }
        *dst = out;
      } else {
        ccol[i] = (beta == 0.0) ? alpha * v0 : fma(alpha, v0, beta * ccol[i]);
        if (i + 1 < p.m) ccol[i + 1] = (beta == 0.0) ? alpha * v1 : fma(alpha, v1, beta * ccol[i + 1]);
      }
    }
  }
}


}  // namespace gbd
