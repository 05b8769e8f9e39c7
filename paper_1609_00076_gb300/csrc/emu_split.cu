// emu_split.cu -- steps 1 and 2 of the split emulation: row/column exponents and
// the digit slices, with integer bit operations only (FP64 arithmetic is a
// low-rate unit on GB300; none is used here).
//
// These kernels are bound by HBM: each reads the operand once (8 bytes per
// element) and the split writes s BF16 digits (2s bytes per element).
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include <cstdint>

#include "emu.cuh"

namespace gbd {
namespace emu {
namespace {

// frexp exponent e of a finite non-zero double (x = f 2^e, 0.5 <= |f| < 1), from its bits
__device__ __forceinline__ int exponent_of(uint64_t bits) {
  const uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
  if (E) return (int)E - 1022;
  const uint64_t frac = bits & 0xFFFFFFFFFFFFFull;  // subnormal: frac * 2^-1074
  return (64 - __clzll((long long)frac)) - 1074;
}

__device__ __forceinline__ bool is_nonfinite(uint64_t bits) {
  return ((bits >> 52) & 0x7FFu) == 0x7FFu;
}
__device__ __forceinline__ bool is_zero(uint64_t bits) { return (bits << 1) == 0; }

template <bool ROWS_CONTIG>
__device__ __forceinline__ uint64_t load_bits(const double* X, int64_t ld, int64_t r, int64_t p) {
  const double* a = ROWS_CONTIG ? X + p * ld + r : X + r * ld + p;
  return (uint64_t)__double_as_longlong(__ldg(a));
}

constexpr int kRedChunk = 1024;  // k elements per block of the reductions

// sigma_r = max over non-zero finite entries of the frexp exponent; bad_r |= any Inf/NaN.
// Block (bx, by) covers 32 rows (ROWS_CONTIG) or 8 rows x 1024 k.
// direct: this block is the only one covering its rows (K <= kRedChunk), so the results are
// stored, with no initialisation of sig and bad needed; otherwise they are merged atomically.
template <bool ROWS_CONTIG>
__device__ __forceinline__ void exponents_body(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                                               int* __restrict__ sig, int* __restrict__ bad, int64_t bx, int64_t by,
                                               int (*s_max)[33], int (*s_bad)[33], bool direct = false) {
  const int64_t p_begin = by * kRedChunk;
  const int64_t p_end = p_begin + kRedChunk < K ? p_begin + kRedChunk : K;
  if (ROWS_CONTIG) {
    // 32 consecutive rows per warp (coalesced), 8 warps split the k range
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r = bx * 32 + tx;
    int mx = kExpEmpty, bd = 0;
    if (r < R)
#pragma unroll 4
      for (int64_t p = p_begin + ty; p < p_end; p += 8) {
        const uint64_t b = load_bits<true>(X, ld, r, p);
        if (is_nonfinite(b)) bd = 1;
        else if (!is_zero(b)) mx = max(mx, exponent_of(b));
      }
    s_max[ty][tx] = mx;
    s_bad[ty][tx] = bd;
    __syncthreads();
    if (ty == 0 && r < R) {
      for (int q = 1; q < 8; ++q) {
        mx = max(mx, s_max[q][tx]);
        bd |= s_bad[q][tx];
      }
      if (direct) {
        sig[r] = mx;
        bad[r] = bd;
      } else {
        if (mx != kExpEmpty) atomicMax(sig + r, mx);
        if (bd) atomicOr(bad + r, 1);
      }
    }
  } else {
    // one row per warp, lanes along the contiguous k direction
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r = bx * 8 + w;
    if (r >= R) return;
    int mx = kExpEmpty, bd = 0;
#pragma unroll 4
    for (int64_t p = p_begin + lane; p < p_end; p += 32) {
      const uint64_t b = load_bits<false>(X, ld, r, p);
      if (is_nonfinite(b)) bd = 1;
      else if (!is_zero(b)) mx = max(mx, exponent_of(b));
    }
    for (int o = 16; o; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bd |= __shfl_xor_sync(0xffffffffu, bd, o);
    }
    if (lane == 0) {
      if (direct) {
        sig[r] = mx;
        bad[r] = bd;
      } else {
        if (mx != kExpEmpty) atomicMax(sig + r, mx);
        if (bd) atomicOr(bad + r, 1);
      }
    }
  }
}

// |x| * 2^-sigma as a float, the mantissa truncated (so within a factor 1 - 2^-23 of the value,
// below it); 0 for a non-finite x and where the result is below 2^-126
__device__ __forceinline__ float scaled_magnitude(uint64_t bits, int sigma) {
  const int E = (int)((bits >> 52) & 0x7FFu);
  if (E == 0x7FF) return 0.0f;
  uint64_t frac = bits & 0xFFFFFFFFFFFFFull;  // |x| = 1.frac 2^ex
  int ex;
  if (E) {
    ex = E - 1023;
  } else {  // subnormal: frac 2^-1074, normalised here
    if (!frac) return 0.0f;
    const int nb = 64 - __clzll((long long)frac);
    ex = nb - 1 - 1074;
    frac = (frac << (53 - nb)) & 0xFFFFFFFFFFFFFull;
  }
  const int fe = ex - sigma + 127;
  if (fe <= 0) return 0.0f;
  if (fe >= 255) return 3.0e38f;
  const uint32_t fb = ((uint32_t)fe << 23) | (uint32_t)(frac >> 29);
  return __uint_as_float(fb);
}

// A block's partial magnitude sum (< 2^31) in 32.32 fixed point.  Partial sums are formed in
// a fixed order inside a block and added across blocks as integers, so the total does not
// depend on the order in which blocks run.
__device__ __forceinline__ unsigned long long magnitude_fixed(float partial) {
  return __float2ull_rz(partial * 4294967296.0f);
}

template <bool ROWS_CONTIG>
__device__ __forceinline__ void magnitudes_body(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                                                const int* __restrict__ sig, unsigned long long* __restrict__ mu,
                                                int64_t bx, int64_t by, float (*s_sum)[33], bool direct = false) {
  const int64_t p_begin = by * kRedChunk;
  const int64_t p_end = p_begin + kRedChunk < K ? p_begin + kRedChunk : K;
  if (ROWS_CONTIG) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r = bx * 32 + tx;
    float acc = 0.0f;
    if (r < R) {
      const int sg = sig[r] == kExpEmpty ? 0 : sig[r];
      for (int64_t p = p_begin + ty; p < p_end; p += 8) acc += scaled_magnitude(load_bits<true>(X, ld, r, p), sg);
    }
    s_sum[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && r < R) {
      for (int q = 1; q < 8; ++q) acc += s_sum[q][tx];
      if (direct) mu[r] = magnitude_fixed(acc);
      else atomicAdd(mu + r, magnitude_fixed(acc));
    }
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r = bx * 8 + w;
    if (r >= R) return;
    const int sg = sig[r] == kExpEmpty ? 0 : sig[r];
    float acc = 0.0f;
    for (int64_t p = p_begin + lane; p < p_end; p += 32) acc += scaled_magnitude(load_bits<false>(X, ld, r, p), sg);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (direct) mu[r] = magnitude_fixed(acc);
      else atomicAdd(mu + r, magnitude_fixed(acc));
    }
  }
}

// a magnitude sum back from 32.32 fixed point
__device__ __forceinline__ float magnitude_value(unsigned long long q) { return (float)((double)q * 0x1p-32); }

__device__ __forceinline__ void min_stats_body(const unsigned long long* __restrict__ muA, int64_t m,
                                               const unsigned long long* __restrict__ muB, int64_t n,
                                               const int* __restrict__ badA,
                                               const int* __restrict__ badB, float* __restrict__ stats,
                                               float (*s_min)[256], int (*s_bad)[256]) {
  float mn[2] = {3.0e38f, 3.0e38f};
  int bd[2] = {0, 0};
  for (int64_t i = threadIdx.x; i < m; i += 256) {
    if (muA[i] > 0ull) mn[0] = fminf(mn[0], magnitude_value(muA[i]));
    bd[0] |= badA[i];
  }
  for (int64_t j = threadIdx.x; j < n; j += 256) {
    if (muB[j] > 0ull) mn[1] = fminf(mn[1], magnitude_value(muB[j]));
    bd[1] |= badB[j];
  }
  for (int q = 0; q < 2; ++q) {
    s_min[q][threadIdx.x] = mn[q];
    s_bad[q][threadIdx.x] = bd[q];
  }
  __syncthreads();
  for (int stride = 128; stride; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int q = 0; q < 2; ++q) {
        s_min[q][threadIdx.x] = fminf(s_min[q][threadIdx.x], s_min[q][threadIdx.x + stride]);
        s_bad[q][threadIdx.x] |= s_bad[q][threadIdx.x + stride];
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[0] = s_min[0][0];
    stats[1] = s_min[1][0];
    stats[2] = (float)s_bad[0][0];
    stats[3] = (float)s_bad[1][0];
  }
}

__global__ void __launch_bounds__(256) k_min_stats(const unsigned long long* __restrict__ muA, int64_t m,
                                                   const unsigned long long* __restrict__ muB, int64_t n,
                                                   const int* __restrict__ badA, const int* __restrict__ badB,
                                                   float* __restrict__ stats) {
  __shared__ float s_min[2][256];
  __shared__ int s_bad[2][256];
  min_stats_body(muA, m, muB, n, badA, badB, stats, s_min, s_bad);
}

// s digits of kDigitBits bits of |x| 2^-sigma, truncated toward zero, with the sign of x:
// Q = floor(|x| 2^(s*b - sigma)) and digit t is bits [(s-t)b, (s-t+1)b) of Q.
__device__ __forceinline__ uint64_t scaled_fixed(uint64_t bits, int sigma, int sb) {
  const uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
  if (E == 0x7FFu) return 0;  // non-finite: the row is flagged, its digits are zero
  uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
  int e2;  // x = mant * 2^e2
  if (E) {
    mant |= 1ull << 52;
    e2 = (int)E - 1075;
  } else {
    e2 = -1074;
  }
  const int sh = e2 - sigma + sb;
  if (sh >= 0) return sh >= 64 ? 0 : (mant << sh);  // |x| < 2^sigma keeps this below 2^sb
  return (-sh >= 64) ? 0 : (mant >> (-sh));
}

__device__ __forceinline__ uint32_t bf16_of_digit(int d) {
  return __float_as_uint((float)d) >> 16;  // |d| <= 127: exact in BF16
}

constexpr int kTile = 64;
constexpr int kPerThread = 8;       // k elements per thread: one 16-byte store per slice
constexpr int kSplitThreads = 512;  // 64 rows x 8 groups of 8 k per 64 x 64 tile

// digits of the 8 values x[0..7] (bits) of row r at k positions pbase..pbase+7, written to
// every slice; 16-byte vector stores when all 8 are inside k (kp % 8 == 0, pbase % 8 == 0)
__device__ __forceinline__ void write_digits(const uint64_t (&x)[kPerThread], int sg, int slices, int64_t R,
                                             int64_t K, int64_t r, int64_t pbase, uint16_t* __restrict__ D,
                                             int64_t kp) {
  const int sb = slices * kDigitBits;
  uint64_t q[kPerThread];
  uint32_t neg = 0;
#pragma unroll
  for (int v = 0; v < kPerThread; ++v) {
    q[v] = scaled_fixed(x[v], sg, sb);
    neg |= (uint32_t)(x[v] >> 63) << v;
  }
  const bool full = pbase + kPerThread <= K;
  for (int t = 0; t < slices; ++t) {
    const int shift = (slices - 1 - t) * kDigitBits;
    uint32_t packed[kPerThread / 2];
#pragma unroll
    for (int v = 0; v < kPerThread; v += 2) {
      int d0 = (int)((q[v] >> shift) & 0x7Fu), d1 = (int)((q[v + 1] >> shift) & 0x7Fu);
      if ((neg >> v) & 1u) d0 = -d0;
      if ((neg >> (v + 1)) & 1u) d1 = -d1;
      packed[v / 2] = bf16_of_digit(d0) | (bf16_of_digit(d1) << 16);
    }
    uint16_t* row = D + ((int64_t)t * R + r) * kp + pbase;
    if (full) {
      *reinterpret_cast<uint4*>(row) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    } else {
      for (int v = 0; v < kPerThread && pbase + v < K; ++v)
        row[v] = (uint16_t)((packed[v / 2] >> (16 * (v & 1))) & 0xFFFFu);
    }
  }
}

// Block (bx, by) writes the digits of the 64 x 64 (row, k) tile at (by*64, bx*64).
// k contiguous in memory: each thread reads its 8 values directly (vector loads when
// 16-byte aligned), a warp sweeps 2 KiB of one row.  Rows contiguous: the tile is
// transposed through shared memory.
// the digits of the split emulation (writer of split_body)
struct DigitWriter {
  int slices;
  int64_t R, K;
  uint16_t* D;
  int64_t kp;
  __device__ __forceinline__ void operator()(const uint64_t (&x)[kPerThread], int sg, int64_t r,
                                             int64_t pbase) const {
    write_digits(x, sg, slices, R, K, r, pbase, D, kp);
  }
};

// rint(x 2^(t - sigma)) of a double given by its bits, ties to even, from integer operations
// (|x| < 2^sigma keeps the result within 2^t); 0 for a non-finite x (its row is flagged)
__device__ __forceinline__ int64_t rounded_scaled(uint64_t bits, int sigma, int t) {
  const uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
  if (E == 0x7FFu) return 0;
  uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
  int e2;  // |x| = mant * 2^e2
  if (E) {
    mant |= 1ull << 52;
    e2 = (int)E - 1075;
  } else {
    e2 = -1074;
  }
  const int sh = e2 - sigma + t;
  uint64_t q;
  if (sh >= 0) {
    q = mant << sh;
  } else if (-sh >= 64) {
    q = 0;  // below a quarter of a unit
  } else {
    const int s = -sh;
    q = mant >> s;
    const uint64_t rem = mant & ((1ull << s) - 1ull), half = 1ull << (s - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (bits >> 63) ? -(int64_t)q : (int64_t)q;
}

// the residues of the modular emulation (writer of split_body): for each modulus p, a residue
// of A' = rint(x 2^(t - sigma)) of magnitude at most 128 (exact in BF16).  The bytes of |A'|
// weighted by 256^d mod p sum, with the start value wbias = 0x4B000000 + c (c = -2^23 mod p),
// to the FP32 bits of x = 2^23 + s' with s' < 2^20 + p, so x = |A'| (mod p).  One fma gives
// q = rint(x * fl(1/p)), within 1/p of x/p, so r = x - p q (exact in one fma) has |r| <= p/2 + 1,
// that is |r| <= 128 for every modulus; the sign of A' is then set on the BF16 pair.
struct ResidueWriter {
  const ModSplit* mp;  // in the kernel's parameter space
  int n, t;            // from the call's plan
  int64_t R, K;
  uint16_t* D;
  int64_t kp;
  __device__ __forceinline__ void operator()(const uint64_t (&x)[kPerThread], int sg, int64_t r,
                                             int64_t pbase) const {
    uint32_t lo[kPerThread], hi[kPerThread];  // the bytes of |A'| (0..3, 4..7)
    uint32_t sgn[kPerThread / 2];             // sign bits 15 and 31 of each BF16 pair
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) {
      const int64_t q = rounded_scaled(x[v], sg, t);
      const uint64_t a = q < 0 ? 0ull - (uint64_t)q : (uint64_t)q;
      lo[v] = (uint32_t)a;
      hi[v] = (uint32_t)(a >> 32);
      if (v & 1) sgn[v / 2] |= q < 0 ? 0x80000000u : 0u;
      else sgn[v / 2] = q < 0 ? 0x00008000u : 0u;
    }
    const bool full = pbase + kPerThread <= K;
    for (int i = 0; i < n; ++i) {
      const float pf = mp->pf[i], inv = mp->inv[i];
      const uint32_t wl = mp->wlo[i], wh = mp->whi[i], wb = mp->wbias[i];  // 256^d mod p, one byte per d
      uint32_t bits[kPerThread];
#pragma unroll
      for (int v = 0; v < kPerThread; ++v) {
        const float xf = __uint_as_float(__dp4a(lo[v], wl, __dp4a(hi[v], wh, wb)));  // 2^23 + s'
        const float qf = fmaf(xf, inv, 12582912.0f) - 12582912.0f;                 // rint(x/p), to 1/p
        bits[v] = __float_as_uint(fmaf(-pf, qf, xf));                               // r, exact
      }
      uint32_t packed[kPerThread / 2];  // BF16 pairs: the upper halves of the FP32 bits (exact here)
#pragma unroll
      for (int v = 0; v < kPerThread; v += 2) packed[v / 2] = __byte_perm(bits[v], bits[v + 1], 0x7632) ^ sgn[v / 2];
      uint16_t* row = D + ((int64_t)i * R + r) * kp + pbase;
      if (full) {
        *reinterpret_cast<uint4*>(row) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
      } else {
        for (int v = 0; v < kPerThread && pbase + v < K; ++v)
          row[v] = (uint16_t)((packed[v / 2] >> (16 * (v & 1))) & 0xFFFFu);
      }
    }
  }
};

// The magnitude plane of the certified precision choice (writer of split_body): for each entry
// v = RZ(max(|x| 2^-sigma, w) 2^S) when x is finite and non-zero, else 0, in BF16 (w = 2^(-63-S)) or
// in FP8 E5M2 (S = 15, w = 2^-29: the smallest normal E5M2 value, so no subnormal is formed).
// Rounding toward zero keeps v below |x| 2^(S-sigma) except where the floor raises it; the floor
// makes the product of two non-zero entries an FP32 normal (at least 2^-126, BF16, or 2^-28,
// FP8), so a product of the planes is zero exactly where every term of |A||B| has a zero factor.
// With |x| < 2^sigma, v < 2^S.  Also the exactness width: the largest sigma - lambda(x) over the
// side, x = odd 2^lambda(x), so that every x 2^(t - sigma) is an integer once t reaches it (capped
// at 255).  Rows hold kp BF16 values or kp FP8 bytes (16-byte pitches either way).
template <bool FP8>
struct MagWriter {
  int S;
  int64_t R, K;
  void* D;
  int64_t kp;
  unsigned int* s_tex;  // the block's exactness width (shared-memory maximum; the kernel flushes it)
  int* s_emin;          // [kTile] the block's rows: smallest frexp exponent of a non-zero entry (shared
                        // minimum; the kernel flushes it), or null
  __device__ __forceinline__ void operator()(const uint64_t (&x)[kPerThread], int sg, int64_t r,
                                             int64_t pbase) const {
    constexpr int kMant = FP8 ? 2 : 7;     // stored fraction bits
    constexpr int kBias = FP8 ? 15 : 127;  // exponent bias
    constexpr int kFloor = FP8 ? -14 : -63;  // exponent of the floor in plane units
    const int base = S - sg - 1023;          // a normal x: exponent of |x| 2^(S - sigma) = E + base
    uint32_t h[kPerThread];
    int w = 0, em = kEminNone;
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) {
      const uint32_t hi = (uint32_t)(x[v] >> 32), lo = (uint32_t)x[v];
      const int E = (int)((hi >> 20) & 0x7FFu);
      if (E == 0x7FF || ((hi << 1) | lo) == 0u) {
        h[v] = 0u;
        continue;
      }
      if (E != 0) {  // normal: the 53-bit significand 1.f, its top fraction bits in hi
        const int eb = E + base;
        h[v] = eb < kFloor ? (uint32_t)(kFloor + kBias) << kMant
                           : ((uint32_t)(eb + kBias) << kMant) | ((hi >> (20 - kMant)) & ((1u << kMant) - 1u));
        // trailing zeros of the significand (the implicit bit bounds them by 52)
        const int tz = lo ? __ffs((int)lo) - 1 : 31 + __ffs((int)((hi & 0xFFFFFu) | 0x100000u));
        w = max(w, min(255, sg - (E - 1075 + tz)));
        em = min(em, E - 1022);
      } else {  // subnormal: |x| = f 2^-1074
        const uint64_t mant = x[v] & 0xFFFFFFFFFFFFFull;
        const int nb = 64 - __clzll((long long)mant);  // bit length, 1..52
        const int eb = nb - 1 - 1074 - sg + S;
        if (eb < kFloor) {
          h[v] = (uint32_t)(kFloor + kBias) << kMant;
        } else {
          const uint32_t mf = (uint32_t)((nb >= kMant + 1 ? (mant >> (nb - kMant - 1)) : (mant << (kMant + 1 - nb))) &
                                         ((1u << kMant) - 1u));
          h[v] = ((uint32_t)(eb + kBias) << kMant) | mf;
        }
        w = max(w, min(255, sg - (-1074 + __ffsll((long long)mant) - 1)));
        em = min(em, nb - 1074);
      }
    }
    const bool full = pbase + kPerThread <= K;
    if (FP8) {
      uint8_t* row = static_cast<uint8_t*>(D) + r * kp + pbase;
      if (full) {
        *reinterpret_cast<uint2*>(row) = make_uint2(h[0] | (h[1] << 8) | (h[2] << 16) | (h[3] << 24),
                                                    h[4] | (h[5] << 8) | (h[6] << 16) | (h[7] << 24));
      } else {
        for (int v = 0; v < kPerThread && pbase + v < K; ++v) row[v] = (uint8_t)h[v];
      }
    } else {
      uint16_t* row = static_cast<uint16_t*>(D) + r * kp + pbase;
      if (full) {
        *reinterpret_cast<uint4*>(row) =
            make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
      } else {
        for (int v = 0; v < kPerThread && pbase + v < K; ++v) row[v] = (uint16_t)h[v];
      }
    }
    // the row's minimum into shared memory; the width reduced over the lanes here together (one
    // mask for all of them), one shared maximum per warp
    if (s_emin && em != kEminNone) atomicMin(s_emin + (r & (kTile - 1)), em);
    const unsigned act = __activemask();
    const unsigned wm = __reduce_max_sync(act, (unsigned)w);
    if ((int)(threadIdx.x & 31) == __ffs((int)act) - 1 && wm) atomicMax(s_tex, wm);
  }
};

// the block's shared width and row minima start empty (before the block's split_body)
__device__ __forceinline__ void mag_shared_init(unsigned int* s_tex, int* s_emin) {
  if (threadIdx.x == 0) *s_tex = 0u;
  if (threadIdx.x < kTile) s_emin[threadIdx.x] = kEminNone;
}
// after a barrier: the block's width into *tex (atomic maximum) and its row minima into emin (rows
// r0 .. r0 + kTile of a side with R rows); then empty again
__device__ __forceinline__ void mag_shared_flush(unsigned int* s_tex, int* s_emin, unsigned int* tex, int* emin,
                                                 int64_t r0, int64_t R) {
  if (threadIdx.x == 0 && *s_tex) {
    atomicMax(tex, *s_tex);
    *s_tex = 0u;
  }
  if (threadIdx.x < kTile) {
    const int v = s_emin[threadIdx.x];
    if (emin && v != kEminNone && r0 + threadIdx.x < R) atomicMin(emin + r0 + threadIdx.x, v);
    s_emin[threadIdx.x] = kEminNone;
  }
}

template <bool ROWS_CONTIG, class Writer>
__device__ __forceinline__ void split_body(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                                           const int* __restrict__ sig, int64_t bx, int64_t by,
                                           uint64_t (*tile)[kTile + 1], const Writer& write) {
  const int64_t p0 = bx * kTile, r0 = by * kTile;
  const int tid = threadIdx.x;
  const int rr = tid >> 3, pp0 = (tid & 7) * kPerThread;
  const int64_t r = r0 + rr, pbase = p0 + pp0;
  uint64_t x[kPerThread];
  if (ROWS_CONTIG) {
    // column pi of a tile row is stored at (pi & ~7) | ((pi ^ (pi >> 3)) & 7): the eight
    // threads that read the same v of eight consecutive groups then hit eight banks
#pragma unroll
    for (int it = 0; it < kTile * kTile / kSplitThreads; ++it) {
      const int idx = tid + it * kSplitThreads;
      const int ri = idx % kTile, pi = idx / kTile;  // coalesced along rows
      const int64_t rg = r0 + ri, pg = p0 + pi;
      tile[ri][(pi & ~7) | ((pi ^ (pi >> 3)) & 7)] = (rg < R && pg < K) ? load_bits<true>(X, ld, rg, pg) : 0ull;
    }
    __syncthreads();
    if (r >= R || pbase >= K) return;  // no barrier follows in here (the grid-stride callers hold theirs)
    const int grp = pp0 >> 3;
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) x[v] = tile[rr][pp0 + (v ^ grp)];
  } else {
    if (r >= R || pbase >= K) return;
    const double* src = X + r * ld + pbase;
    if (pbase + kPerThread <= K && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
      const longlong2* s2 = reinterpret_cast<const longlong2*>(src);
#pragma unroll
      for (int v = 0; v < kPerThread / 2; ++v) {
        const longlong2 w = __ldg(s2 + v);
        x[2 * v] = (uint64_t)w.x;
        x[2 * v + 1] = (uint64_t)w.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < kPerThread; ++v)
        x[v] = (pbase + v < K) ? (uint64_t)__double_as_longlong(__ldg(src + v)) : 0ull;
    }
  }
  const int sg = sig[r] == kExpEmpty ? 0 : sig[r];
  write(x, sg, r, pbase);
}

// ---- batched forms over a job table (one operand side of one problem per job) ----
// the job of block b: the last whose first block is at most b (begins from the kernel parameters
// when they hold every job, else from the table)
__device__ __forceinline__ int find_job(const JobBegins& jb, const PrepJob* __restrict__ jobs, int njobs, int64_t b,
                                        bool split) {
  int lo = 0, hi = njobs - 1;
  if (jb.n == njobs) {
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jb.b[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((split ? jobs[mid].split_begin : jobs[mid].exp_begin) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_prep_init_batched(const PrepJob* __restrict__ jobs) {
  const PrepJob& j = jobs[blockIdx.x];
  for (int64_t r = threadIdx.x; r < j.R; r += blockDim.x) {
    j.sig[r] = kExpEmpty;
    j.bad[r] = 0;
    if (j.mu) j.mu[r] = 0ull;
    if (j.emin) j.emin[r] = kEminNone;
  }
}

__global__ void __launch_bounds__(256) k_exponents_batched(const PrepJob* __restrict__ jobs, int njobs,
                                                           const __grid_constant__ JobBegins jb) {
  __shared__ int s_max[8][33];
  __shared__ int s_bad[8][33];
  const int ji = find_job(jb, jobs, njobs, blockIdx.x, false);
  const PrepJob& j = jobs[ji];
  const int64_t local = (int64_t)blockIdx.x - j.exp_begin;
  const int64_t bx = local % j.exp_gx, by = local / j.exp_gx;
  if (j.rows_contig) exponents_body<true>(j.X, j.ld, j.R, j.K, j.sig, j.bad, bx, by, s_max, s_bad);
  else exponents_body<false>(j.X, j.ld, j.R, j.K, j.sig, j.bad, bx, by, s_max, s_bad);
}

__global__ void __launch_bounds__(kSplitThreads) k_split_batched(const PrepJob* __restrict__ jobs, int njobs,
                                                                 const __grid_constant__ JobBegins jb) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = find_job(jb, jobs, njobs, blockIdx.x, true);
  const PrepJob& j = jobs[ji];
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  const DigitWriter w{j.slices, j.R, j.K, j.D, j.kp};
  if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
  else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
}

// grouped modular problems: magnitude planes (FP8) and residues over a job table
// FP8 planes (the certification), or BF16 planes for its retry: then only the jobs whose problem's
// plan found no feasible precision, with the widths into the retry's words
// RETRY: a grid-stride loop over the blocks that starts only when `run_if` is non-zero (some
// problem's first plan found no feasible t), and skips the jobs whose plan is feasible
template <bool FP8, bool RETRY>
__global__ void __launch_bounds__(kSplitThreads, 3) k_magplane_batched(const PrepJob* __restrict__ jobs, int njobs,
                                                                    int64_t nblocks,
                                                                    const unsigned int* __restrict__ run_if,
                                                                    const __grid_constant__ JobBegins jb) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  __shared__ unsigned int s_tex;
  __shared__ int s_emin[kTile];
  if (RETRY && *run_if == 0u) return;
  mag_shared_init(&s_tex, s_emin);
  __syncthreads();
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int ji = find_job(jb, jobs, njobs, b, true);
    const PrepJob& j = jobs[ji];
    const bool live = !RETRY || !j.plan->feasible;  // uniform over the block
    const int64_t local = b - j.split_begin;
    const int64_t bx = local % j.split_gx, by = local / j.split_gx;
    if (live) {
      int S = 15;  // the E5M2 plane scale; BF16: the largest with K 2^(2S) < 2^124
      if (!FP8) {
        int kb = 0;
        while (((int64_t)1 << kb) < j.K) ++kb;
        S = (124 - kb) / 2;
      }
      const int64_t pitch = FP8 ? (j.K + 15) / 16 * 16 : (j.K + 7) / 8 * 8;
      const MagWriter<FP8> w{S, j.R, j.K, j.D, pitch, &s_tex, j.emin ? s_emin : nullptr};
      if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
      else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
    }
    __syncthreads();  // the block's width and row minima are complete (and the tile free)
    mag_shared_flush(&s_tex, s_emin, RETRY ? j.tex + kCertRetry : j.tex, j.emin, by * kTile, j.R);
    if (!RETRY) break;  // one block per grid index
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSplitThreads, 3) k_residue_batched(const PrepJob* __restrict__ jobs, int njobs,
                                                                   const __grid_constant__ ModSplit mp,
                                                                   const __grid_constant__ JobBegins jb) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = find_job(jb, jobs, njobs, blockIdx.x, true);
  const PrepJob& j = jobs[ji];
  const ModPlan pl = *j.plan;
  if (!pl.feasible) return;  // the problem is computed by the FP64 kernel
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  const ResidueWriter w{&mp, pl.n, pl.t, j.R, j.K, j.D, j.kp};
  if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
  else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
}

// ---- both operand sides of one problem in one launch (single calls) ----
// job 0 is op(A), job 1 op(B)^T; their blocks are numbered by prep_job_blocks.  The jobs are
// kernel arguments, so no job table has to be copied to the device.
__global__ void __launch_bounds__(256) k_prep_init_pair(const __grid_constant__ PrepPair pp) {
  const PrepJob& j = pp.j[blockIdx.y];
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < j.R; r += (int64_t)gridDim.x * blockDim.x) {
    j.sig[r] = kExpEmpty;
    j.bad[r] = 0;
    if (j.mu) j.mu[r] = 0ull;
  }
}

__global__ void __launch_bounds__(256) k_exponents_pair(const __grid_constant__ PrepPair pp, bool direct,
                                                        uint4* __restrict__ zero, int64_t zero_vecs) {
  __shared__ int s_max[8][33];
  __shared__ int s_bad[8][33];
  // clears the slice kernel's accumulation area on the way (16-byte stores over the grid)
  for (int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; z < zero_vecs; z += (int64_t)gridDim.x * blockDim.x)
    zero[z] = make_uint4(0u, 0u, 0u, 0u);
  const int ji = (int64_t)blockIdx.x >= pp.j[1].exp_begin ? 1 : 0;
  const PrepJob& j = pp.j[ji];
  const int64_t local = (int64_t)blockIdx.x - j.exp_begin;
  const int64_t bx = local % j.exp_gx, by = local / j.exp_gx;
  if (j.rows_contig) exponents_body<true>(j.X, j.ld, j.R, j.K, j.sig, j.bad, bx, by, s_max, s_bad, direct);
  else exponents_body<false>(j.X, j.ld, j.R, j.K, j.sig, j.bad, bx, by, s_max, s_bad, direct);
}

__global__ void __launch_bounds__(256) k_magnitudes_pair(const __grid_constant__ PrepPair pp, bool direct) {
  __shared__ float s_sum[8][33];
  const int ji = (int64_t)blockIdx.x >= pp.j[1].exp_begin ? 1 : 0;
  const PrepJob& j = pp.j[ji];
  const int64_t local = (int64_t)blockIdx.x - j.exp_begin;
  const int64_t bx = local % j.exp_gx, by = local / j.exp_gx;
  if (j.rows_contig) magnitudes_body<true>(j.X, j.ld, j.R, j.K, j.sig, j.mu, bx, by, s_sum, direct);
  else magnitudes_body<false>(j.X, j.ld, j.R, j.K, j.sig, j.mu, bx, by, s_sum, direct);
}

// ---- statistics and FP8 magnitude planes in one pass (the modular emulation's automatic mode) ----
// 2^d for d <= 0 as a float (0 below 2^-126)
__device__ __forceinline__ float pow2f_nonpos(int d) { return d < -126 ? 0.0f : __int_as_float((127 + d) << 23); }

// One 64 x 64 tile of one side (rows r0 + 0..63, k p0 + 0..63), eight threads per row, each with
// eight consecutive entries (split_body's layout; no thread leaves early, so the eight threads of
// a row can reduce together).  For each row of the tile: its largest exponent E_t, the FP8 E5M2
// magnitude-plane bytes of its entries relative to E_t (MagWriter's bytes with E_t in place of
// sigma; the row merge moves them to sigma), and the tile's partial statistics, written by
// the row's first thread at [r][bx]: E_t, a non-finite flag, the magnitude and square sums
// relative to E_t (FP32, in a fixed order), the smallest frexp exponent of a non-zero entry and
// the smallest exponent of a lowest set bit.
template <bool ROWS_CONTIG>
__device__ __forceinline__ void statplane_tile(const double* __restrict__ X, int64_t ld, int64_t R, int64_t K,
                                               uint8_t* __restrict__ D, int64_t kp, const StatSide& st, int64_t bx,
                                               int64_t by, uint64_t (*tile)[kTile + 1]) {
  constexpr int S = 15, kMant = 2, kBias = 15, kFloor = -14;  // E5M2, as MagWriter<true>
  const int64_t p0 = bx * kTile, r0 = by * kTile;
  const int tid = threadIdx.x;
  const int rr = tid >> 3, pp0 = (tid & 7) * kPerThread;
  const int64_t r = r0 + rr, pbase = p0 + pp0;
  const bool row_in = r < R;
  uint64_t x[kPerThread];
  if (ROWS_CONTIG) {
    // column pi of a tile row is stored at (pi & ~7) | ((pi ^ (pi >> 3)) & 7) (as split_body)
#pragma unroll
    for (int it = 0; it < kTile * kTile / kSplitThreads; ++it) {
      const int idx = tid + it * kSplitThreads;
      const int ri = idx % kTile, pi = idx / kTile;  // coalesced along rows
      const int64_t rg = r0 + ri, pg = p0 + pi;
      tile[ri][(pi & ~7) | ((pi ^ (pi >> 3)) & 7)] = (rg < R && pg < K) ? load_bits<true>(X, ld, rg, pg) : 0ull;
    }
    __syncthreads();
    const int grp = pp0 >> 3;
#pragma unroll
    for (int v = 0; v < kPerThread; ++v) x[v] = tile[rr][pp0 + (v ^ grp)];
  } else {
    const double* src = X + (row_in ? r : 0) * ld + pbase;
    if (row_in && pbase + kPerThread <= K && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
      const longlong2* s2 = reinterpret_cast<const longlong2*>(src);
#pragma unroll
      for (int v = 0; v < kPerThread / 2; ++v) {
        const longlong2 w = __ldg(s2 + v);
        x[2 * v] = (uint64_t)w.x;
        x[2 * v + 1] = (uint64_t)w.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < kPerThread; ++v)
        x[v] = (row_in && pbase + v < K) ? (uint64_t)__double_as_longlong(__ldg(src + v)) : 0ull;
    }
  }
  // the row's largest exponent over the tile (its eight threads: lanes 8q .. 8q + 7 of the warp)
  int emax = kExpEmpty, bad = 0;
#pragma unroll
  for (int v = 0; v < kPerThread; ++v) {
    if (is_nonfinite(x[v])) bad = 1;
    else if (!is_zero(x[v])) emax = max(emax, exponent_of(x[v]));
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int sg = emax == kExpEmpty ? 0 : emax;
  const int base = S - sg - 1023;  // a normal x: exponent of |x| 2^(S - E_t) = E + base
  uint32_t h[kPerThread];
  float acc = 0.0f, sq = 0.0f;
  int em = kEminNone, low = kEminNone;
#pragma unroll
  for (int v = 0; v < kPerThread; ++v) {
    const uint32_t hi = (uint32_t)(x[v] >> 32), lo = (uint32_t)x[v];
    const int E = (int)((hi >> 20) & 0x7FFu);
    if (E == 0x7FF || ((hi << 1) | lo) == 0u) {
      h[v] = 0u;
      continue;
    }
    if (E != 0) {  // normal: the 53-bit significand 1.f, its top fraction bits in hi
      const int eb = E + base;
      h[v] = eb < kFloor ? (uint32_t)(kFloor + kBias) << kMant
                         : ((uint32_t)(eb + kBias) << kMant) | ((hi >> (20 - kMant)) & ((1u << kMant) - 1u));
      const int tz = lo ? __ffs((int)lo) - 1 : 31 + __ffs((int)((hi & 0xFFFFFu) | 0x100000u));
      low = min(low, E - 1075 + tz);
      em = min(em, E - 1022);
      // |x| 2^-E_t as a float, its mantissa truncated (as scaled_magnitude; below 2^-126: 0)
      const int fe = E - sg - 896;  // <= 126: |x| < 2^E_t
      const float vf = fe > 0 ? __uint_as_float(((uint32_t)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29)) : 0.0f;
      acc += vf;
      sq = fmaf(vf, vf, sq);
    } else {  // subnormal: |x| = f 2^-1074
      const uint64_t mant = x[v] & 0xFFFFFFFFFFFFFull;
      const int nb = 64 - __clzll((long long)mant);
      const int eb = nb - 1 - 1074 - sg + S;
      if (eb < kFloor) {
        h[v] = (uint32_t)(kFloor + kBias) << kMant;
      } else {
        const uint32_t mf = (uint32_t)((nb >= kMant + 1 ? (mant >> (nb - kMant - 1)) : (mant << (kMant + 1 - nb))) &
                                       ((1u << kMant) - 1u));
        h[v] = ((uint32_t)(eb + kBias) << kMant) | mf;
      }
      low = min(low, -1074 + __ffsll((long long)mant) - 1);
      em = min(em, nb - 1074);
      const float vf = scaled_magnitude(x[v], sg);
      acc += vf;
      sq = fmaf(vf, vf, sq);
    }
  }
  if (row_in && pbase < K) {
    uint8_t* row = D + r * kp + pbase;
    if (pbase + kPerThread <= K) {
      *reinterpret_cast<uint2*>(row) = make_uint2(h[0] | (h[1] << 8) | (h[2] << 16) | (h[3] << 24),
                                                  h[4] | (h[5] << 8) | (h[6] << 16) | (h[7] << 24));
    } else {
      for (int v = 0; v < kPerThread && pbase + v < K; ++v) row[v] = (uint8_t)h[v];
    }
  }
  // the row's partials over its eight threads: a fixed butterfly, so every lane holds the same bits
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    em = min(em, __shfl_xor_sync(0xffffffffu, em, o));
    low = min(low, __shfl_xor_sync(0xffffffffu, low, o));
  }
  if ((tid & 7) == 0 && row_in) {
    const int64_t o = r * st.nkt + bx;
    st.e[o] = emax;
    st.b[o] = bad;
    st.s[o] = acc;
    st.q[o] = sq;
    st.lo[o] = em;
    st.low[o] = low;
  }
}

__global__ void __launch_bounds__(kSplitThreads, 3) k_statplane_pair(const __grid_constant__ PrepPair pp) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = (int64_t)blockIdx.x >= pp.j[1].split_begin ? 1 : 0;
  const PrepJob& j = pp.j[ji];
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  uint8_t* D = static_cast<uint8_t*>(static_cast<void*>(j.D));
  const int64_t kp = (j.K + 15) / 16 * 16;  // FP8 plane pitch
  if (j.rows_contig) statplane_tile<true>(j.X, j.ld, j.R, j.K, D, kp, j.st, bx, by, tile);
  else statplane_tile<false>(j.X, j.ld, j.R, j.K, D, kp, j.st, bx, by, tile);
}

__global__ void __launch_bounds__(kSplitThreads, 3) k_statplane_batched(const PrepJob* __restrict__ jobs, int njobs,
                                                                     const __grid_constant__ JobBegins jb) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = find_job(jb, jobs, njobs, blockIdx.x, true);
  const PrepJob& j = jobs[ji];
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  uint8_t* D = static_cast<uint8_t*>(static_cast<void*>(j.D));
  const int64_t kp = (j.K + 15) / 16 * 16;
  if (j.rows_contig) statplane_tile<true>(j.X, j.ld, j.R, j.K, D, kp, j.st, bx, by, tile);
  else statplane_tile<false>(j.X, j.ld, j.R, j.K, D, kp, j.st, bx, by, tile);
}

// The square sum of a row is computed in FP32 from at most K terms v^2 (v = |x| 2^-E_t rounded
// toward zero to FP32, v^2 added by a fused multiply-add), three butterfly levels per tile, and the
// row's merge (at most ceil(nkt/32) additions per lane and five butterfly levels), each a rounding
// of a sum of non-negative values; the rescalings by powers of two are exact except where they
// underflow, which drops parts below K 2^-126 in all.  So the computed q satisfies
// sum_p (x_p 2^-sigma)^2 <= q (1 + (K + 4 nkt + 16) 2^-24 (1 + 2^-20)) + K 2^-126, and
// q (1 + (K + 8 nkt + 64) 2^-22) + K 2^-125, rounded upward, covers it.
__device__ __forceinline__ float square_grow(int64_t K, int nkt) {
  return __fadd_ru(1.0f, __fmul_ru((float)(K + 8 * (int64_t)nkt + 64), 0x1p-22f));
}
__device__ __forceinline__ float square_floor(int64_t K) { return __fmul_ru((float)K, 0x1p-125f); }

// FP8 E5M2 plane bytes scaled by 2^-d (d >= 0, four bytes of a word): the exponent field lowered
// by d, the smallest normal value (0x04) where it would fall below it; zeros stay zero.  A byte
// v = RZ(max(|x| 2^-E_t, w) 2^S) so becomes RZ(max(|x| 2^-sigma, w) 2^S) for d = sigma - E_t:
// scaling by a power of two commutes with rounding toward zero while the result stays normal,
// and below the smallest normal both sides take the floor.
__device__ __forceinline__ uint32_t plane_shift4(uint32_t w, int d) {
  uint32_t out = 0u;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    uint32_t v = (w >> (8 * b)) & 0xFFu;
    if (v) {
      const int ne = (int)(v >> 2) - d;
      v = ne >= 1 ? ((uint32_t)ne << 2) | (v & 3u) : 0x04u;
    }
    out |= v << (8 * b);
  }
  return out;
}

// Row r of job j, on one warp: its tile partials merged (sigma = the largest tile exponent, bad,
// mu and the square sum rescaled to sigma, added per lane in tile order and then over a fixed
// butterfly, so every lane holds the same bits; the smallest exponents), written to sig, bad, mu
// and emin; the FP8 plane bytes of the row's tiles below sigma moved to sigma; returns (to every
// lane) the row's square-sum bound and exactness width (0 for a row without a non-zero entry).
__device__ __forceinline__ void merge_row_warp(const PrepJob& j, int64_t r, int lane, float grow, float floor_add,
                                               float& sq_up, int& width) {
  const StatSide& st = j.st;
  const int64_t o = r * st.nkt;
  int E = kExpEmpty, bd = 0, mn = kEminNone, lw = kEminNone;
  for (int q = lane; q < st.nkt; q += 32) {
    E = max(E, st.e[o + q]);
    bd |= st.b[o + q];
    mn = min(mn, st.lo[o + q]);
    lw = min(lw, st.low[o + q]);
  }
  for (int d = 16; d; d >>= 1) {
    E = max(E, __shfl_xor_sync(0xffffffffu, E, d));
    bd |= __shfl_xor_sync(0xffffffffu, bd, d);
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    lw = min(lw, __shfl_xor_sync(0xffffffffu, lw, d));
  }
  float mu = 0.0f, sq = 0.0f;
  if (E != kExpEmpty) {
    uint8_t* prow = static_cast<uint8_t*>(static_cast<void*>(j.D)) + r * ((j.K + 15) / 16 * 16);
    for (int q = lane; q < st.nkt; q += 32) {
      const int e = st.e[o + q];
      if (e == kExpEmpty) continue;
      mu += st.s[o + q] * pow2f_nonpos(e - E);
      sq += st.q[o + q] * pow2f_nonpos(2 * (e - E));
      const int d = E - e;
      if (d > 0) {  // this tile's plane bytes, relative to its own exponent: move them to sigma
        const int64_t p0 = (int64_t)q * kTile;
        const int64_t nb = j.K - p0 < kTile ? j.K - p0 : kTile;
        uint8_t* b = prow + p0;
        if (nb == kTile) {
          uint4* b4 = reinterpret_cast<uint4*>(b);  // 16-byte aligned: the pitch and p0 are multiples of 16
#pragma unroll
          for (int v = 0; v < kTile / 16; ++v) {
            uint4 w = b4[v];
            w.x = plane_shift4(w.x, d);
            w.y = plane_shift4(w.y, d);
            w.z = plane_shift4(w.z, d);
            w.w = plane_shift4(w.w, d);
            b4[v] = w;
          }
        } else {
          for (int64_t v = 0; v < nb; ++v) b[v] = (uint8_t)plane_shift4(b[v], d);
        }
      }
    }
    for (int d = 16; d; d >>= 1) {
      mu += __shfl_xor_sync(0xffffffffu, mu, d);
      sq += __shfl_xor_sync(0xffffffffu, sq, d);
    }
  }
  if (lane == 0) {
    j.sig[r] = E;
    j.bad[r] = bd;
    if (j.mu) j.mu[r] = magnitude_fixed(mu);
    if (j.emin) j.emin[r] = mn;
  }
  width = (E != kExpEmpty && lw != kEminNone) ? min(255, E - lw) : 0;
  sq_up = E != kExpEmpty ? __fmaf_ru(sq, grow, floor_add) : 0.0f;
}

// the block's maxima of (sq_up, width) over its warps into *norm and *tex (atomic maxima)
__device__ __forceinline__ void flush_row_maxima(float mx, int wmax, unsigned int* norm, unsigned int* tex) {
  __shared__ float s_mx[8];
  __shared__ int s_w[8];
  if ((threadIdx.x & 31) == 0) {
    s_mx[threadIdx.x >> 5] = mx;
    s_w[threadIdx.x >> 5] = wmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      mx = fmaxf(mx, s_mx[q]);
      wmax = max(wmax, s_w[q]);
    }
    if (mx > 0.0f) atomicMax(norm, __float_as_uint(mx));  // non-negative floats order as their bits
    if (wmax > 0) atomicMax(tex, (unsigned int)wmax);
  }
}

// per row of both sides (a warp per row): the merged statistics and the planes moved to sigma;
// then each side's largest square-sum bound and exactness width into norms[side] and tex[side]
__global__ void __launch_bounds__(256) k_rowstats_pair(const __grid_constant__ PrepPair pp, unsigned int* tex,
                                                       unsigned int* norms) {
  const int ji = blockIdx.y;
  const PrepJob& j = pp.j[ji];
  const float grow = square_grow(j.K, j.st.nkt), floor_add = square_floor(j.K);
  const int lane = threadIdx.x & 31;
  float mx = 0.0f;
  int wmax = 0;
  for (int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); r < j.R; r += (int64_t)gridDim.x * 8) {
    float sq_up;
    int width;
    merge_row_warp(j, r, lane, grow, floor_add, sq_up, width);
    mx = fmaxf(mx, sq_up);
    wmax = max(wmax, width);
  }
  flush_row_maxima(mx, wmax, norms + ji, tex + ji);
}

// grouped modular problems: the same per-row work (the job's norm and width words), a block row
// per job (blockIdx.y)
__global__ void __launch_bounds__(256) k_rowstats_batched(const PrepJob* __restrict__ jobs) {
  const PrepJob& j = jobs[blockIdx.y];
  const float grow = square_grow(j.K, j.st.nkt), floor_add = square_floor(j.K);
  const int lane = threadIdx.x & 31;
  float mx = 0.0f;
  int wmax = 0;
  for (int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); r < j.R; r += (int64_t)gridDim.x * 8) {
    float sq_up;
    int width;
    merge_row_warp(j, r, lane, grow, floor_add, sq_up, width);
    mx = fmaxf(mx, sq_up);
    wmax = max(wmax, width);
  }
  flush_row_maxima(mx, wmax, j.norm, j.tex);
}

// The same over the rows of all jobs numbered one after the other (jb: each job's first row): warp
// w of the grid takes the rows [w c, (w + 1) c), and its maxima go to a job's words when the job
// changes and at the end
__global__ void __launch_bounds__(256) k_rowstats_flat(const PrepJob* __restrict__ jobs, int njobs, int64_t rows,
                                                       const __grid_constant__ JobBegins jb) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * 8, w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t c = (rows + warps - 1) / warps;
  const int64_t g0 = w * c, g1 = g0 + c < rows ? g0 + c : rows;
  if (g0 >= g1) return;
  int lo = 0, hi = njobs - 1;  // the job of row g0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jb.b[mid] <= g0) lo = mid;
    else hi = mid - 1;
  }
  int ji = lo;
  float mx = 0.0f;
  int wmax = 0;
  for (int64_t g = g0; g < g1; ++g) {
    while (ji + 1 < njobs && jb.b[ji + 1] <= g) {  // the next job: flush this one's maxima
      if (lane == 0) {
        if (mx > 0.0f) atomicMax(jobs[ji].norm, __float_as_uint(mx));
        if (wmax > 0) atomicMax(jobs[ji].tex, (unsigned int)wmax);
      }
      mx = 0.0f;
      wmax = 0;
      ++ji;
    }
    const PrepJob& j = jobs[ji];
    float sq_up;
    int width;
    merge_row_warp(j, g - jb.b[ji], lane, square_grow(j.K, j.st.nkt), square_floor(j.K), sq_up, width);
    mx = fmaxf(mx, sq_up);
    wmax = max(wmax, width);
  }
  if (lane == 0) {
    if (mx > 0.0f) atomicMax(jobs[ji].norm, __float_as_uint(mx));
    if (wmax > 0) atomicMax(jobs[ji].tex, (unsigned int)wmax);
  }
}

__global__ void __launch_bounds__(kSplitThreads, 3) k_split_pair(const __grid_constant__ PrepPair pp) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = (int64_t)blockIdx.x >= pp.j[1].split_begin ? 1 : 0;
  const PrepJob& j = pp.j[ji];
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  const DigitWriter w{j.slices, j.R, j.K, j.D, j.kp};
  if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
  else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
}

__global__ void __launch_bounds__(kSplitThreads, 3) k_residue_pair(const __grid_constant__ PrepPair pp,
                                                                const __grid_constant__ ModSplit mp) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  const int ji = (int64_t)blockIdx.x >= pp.j[1].split_begin ? 1 : 0;
  const PrepJob& j = pp.j[ji];
  const int64_t local = (int64_t)blockIdx.x - j.split_begin;
  const int64_t bx = local % j.split_gx, by = local / j.split_gx;
  const ModPlan pl = *mp.plan;
  const ResidueWriter w{&mp, pl.n, pl.t, j.R, j.K, j.D, j.kp};
  if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
  else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
}

// the magnitude planes of both sides (plane scale S, rows of kp elements): job j writes its D,
// side j's width to tex[j]
template <bool FP8>
// a grid-stride loop over the nblocks blocks of both sides (a gated retry runs on a small grid
// and returns at once when the certification it would repeat succeeded)
__global__ void __launch_bounds__(kSplitThreads, 3) k_magplane_pair(const __grid_constant__ PrepPair pp, int S,
                                                                 int64_t kp, unsigned int* tex, const ModPlan* gate,
                                                                 int64_t nblocks) {
  __shared__ uint64_t tile[kTile][kTile + 1];
  __shared__ unsigned int s_tex;
  __shared__ int s_emin[kTile];
  if (gate && gate->feasible) return;  // the retry of a certification that already succeeded
  mag_shared_init(&s_tex, s_emin);
  __syncthreads();
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int ji = b >= pp.j[1].split_begin ? 1 : 0;
    const PrepJob& j = pp.j[ji];
    const int64_t local = b - j.split_begin;
    const int64_t bx = local % j.split_gx, by = local / j.split_gx;
    const MagWriter<FP8> w{S, j.R, j.K, j.D, kp, &s_tex, j.emin ? s_emin : nullptr};
    if (j.rows_contig) split_body<true>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
    else split_body<false>(j.X, j.ld, j.R, j.K, j.sig, bx, by, tile, w);
    __syncthreads();  // the block's width and row minima are complete (and the tile free)
    mag_shared_flush(&s_tex, s_emin, tex + ji, j.emin, by * kTile, j.R);
    if ((int64_t)gridDim.x >= nblocks) break;  // one block per grid index
    __syncthreads();
  }
}

int launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBD_OK : cuda_fail(e, what);
}

}  // namespace

int split_count(int64_t m, int64_t n, int64_t k) {
  if (m <= 0 || n <= 0 || k <= 0) return 1;
  const int64_t tiles = ((m + 127) / 128) * ((n + 127) / 128);
  const int64_t nkb = (k + kBK - 1) / kBK;
  const int64_t nsegs = (nkb + kSegBlocks - 1) / kSegBlocks;
  if (tiles * nsegs * 2 > kSplitTargetItems) return 1;
  int64_t sp = kSplitTargetItems / (tiles * nsegs);
  const int64_t seg_len = nkb < kSegBlocks ? nkb : kSegBlocks;
  if (sp > seg_len / 2) sp = seg_len / 2;  // at least two k-blocks per sub-range
  return sp < 1 ? 1 : (int)sp;
}

size_t layout(int64_t m, int64_t n, int64_t k, int s, void* base, Workspace* ws, bool pair_scratch) {
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
  const size_t o_cert = off; off = up(off + sizeof(unsigned int) * kCertWords);
  const size_t o_emin = off; off = up(off + sizeof(int) * (size_t)(m + n));
  const int64_t nkt = (k + kTile - 1) / kTile;  // 64-wide k tiles of the one-pass statistics
  size_t o_part[2][6];
  for (int side = 0; side < 2; ++side)
    for (int f = 0; f < 6; ++f) {
      o_part[side][f] = off;
      off = up(off + 4 * (size_t)(side == 0 ? m : n) * (size_t)nkt);
    }
  const size_t o_DA = off; off = up(off + 2 * (size_t)s * (size_t)m * (size_t)kp);
  const size_t o_DB = off; off = up(off + 2 * (size_t)s * (size_t)n * (size_t)kp);
  // two-SM kernel: one 128 x 256 FP64 running-sum slot per CTA (at most one pair per 256 x 256 tile)
  // and kParkSlots 128 x 256 int32 slots per CTA for the parked level sums; the one-SM kernel
  // keeps its sums in TMEM
  const int64_t pair_tiles = ((m + 255) / 256) * ((n + 255) / 256);
  const int scratch_ctas =
      pair_scratch ? (int)(2 * pair_tiles < kMaxPairCtas ? 2 * pair_tiles : kMaxPairCtas) : 0;
  const size_t o_scr = off; off = up(off + sizeof(double) * 128 * 256 * (size_t)scratch_ctas);
  const size_t o_scp = off; off = up(off + sizeof(int32_t) * kParkSlots * 128 * 256 * (size_t)scratch_ctas);
  // single calls: exact group sums of the split one-SM kernel and its per-tile counters
  const int splits = pair_scratch ? split_count(m, n, k) : 1;
  const int64_t tiles128 = ((m + 127) / 128) * ((n + 127) / 128);
  const int64_t nsegs = ((k + kBK - 1) / kBK + kSegBlocks - 1) / kSegBlocks;
  const int64_t ngroups = (s + kGroupLevels - 1) / kGroupLevels;
  const size_t ysum_bytes =
      splits > 1 ? sizeof(unsigned long long) * 128 * 128 * (size_t)(tiles128 * nsegs * ngroups) : 0;
  const size_t done_bytes = splits > 1 ? sizeof(unsigned int) * (size_t)tiles128 : 0;
  const size_t o_ysum = off;
  off = up(off + ysum_bytes + done_bytes);
  if (base && ws) {
    char* b = static_cast<char*>(base);
    ws->sigA = reinterpret_cast<int*>(b + o_sigA);
    ws->sigB = reinterpret_cast<int*>(b + o_sigB);
    ws->badA = reinterpret_cast<int*>(b + o_badA);
    ws->badB = reinterpret_cast<int*>(b + o_badB);
    ws->muA = reinterpret_cast<unsigned long long*>(b + o_muA);
    ws->muB = reinterpret_cast<unsigned long long*>(b + o_muB);
    ws->stats = reinterpret_cast<float*>(b + o_stats);
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
    ws->DA = reinterpret_cast<uint16_t*>(b + o_DA);
    ws->DB = reinterpret_cast<uint16_t*>(b + o_DB);
    ws->scratch = reinterpret_cast<double*>(b + o_scr);
    ws->scratch_p = reinterpret_cast<int32_t*>(b + o_scp);
    ws->scratch_ctas = scratch_ctas;
    ws->kp = kp;
    ws->splits = splits;
    ws->ysum = reinterpret_cast<unsigned long long*>(b + o_ysum);
    ws->tile_done = reinterpret_cast<unsigned int*>(b + o_ysum + ysum_bytes);
    ws->zero_bytes = up(ysum_bytes + done_bytes);
  }
  return off;
}

int launch_min_stats(const unsigned long long* muA, int64_t m, const unsigned long long* muB, int64_t n,
                     const int* badA, const int* badB, float* stats, cudaStream_t s) {
  k_min_stats<<<1, 256, 0, s>>>(muA, m, muB, n, badA, badB, stats);
  return launch_check("statistics kernel launch");
}

void prep_job_blocks(PrepJob& j, int64_t& exp_blocks, int64_t& split_blocks) {
  const int64_t gy = (j.K + kRedChunk - 1) / kRedChunk;
  j.exp_gx = (int)(j.rows_contig ? (j.R + 31) / 32 : (j.R + 7) / 8);
  j.exp_begin = exp_blocks;
  exp_blocks += (j.R > 0 && j.K > 0) ? (int64_t)j.exp_gx * gy : 0;
  j.split_gx = (int)((j.K + kTile - 1) / kTile);
  j.split_begin = split_blocks;
  split_blocks += (j.R > 0 && j.K > 0) ? (int64_t)j.split_gx * ((j.R + kTile - 1) / kTile) : 0;
}

int64_t job_begins(const PrepJob* jobs_host, int njobs, JobNumbering which, JobBegins& out) {
  out.n = njobs <= kBeginCache ? njobs : 0;
  out.pad = 0;
  int64_t total = 0;
  for (int q = 0; q < njobs; ++q) {
    const PrepJob& j = jobs_host[q];
    const int64_t begin = which == kByExponentBlock ? j.exp_begin : which == kBySplitTile ? j.split_begin : total;
    if (q < kBeginCache) out.b[q] = begin;
    if (which == kByRow) total += j.R;
  }
  return total;
}

int launch_prep_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t exp_blocks,
                        int64_t split_blocks, bool exponents, bool split, cudaStream_t s) {
  if (njobs <= 0) return GBD_OK;
  static thread_local JobBegins jb;  // 15 KB: not on the stack
  if (exponents) {
    k_prep_init_batched<<<njobs, 256, 0, s>>>(jobs_dev);
    int rc = launch_check("batched init launch");
    if (rc) return rc;
    if (exp_blocks > 0) {
      if (exp_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "grouped: too many exponent blocks");
      job_begins(jobs_host, njobs, kByExponentBlock, jb);
      k_exponents_batched<<<(unsigned)exp_blocks, 256, 0, s>>>(jobs_dev, njobs, jb);
      if ((rc = launch_check("batched exponent launch"))) return rc;
    }
  }
  if (split && split_blocks > 0) {
    if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "grouped: too many split blocks");
    job_begins(jobs_host, njobs, kBySplitTile, jb);
    k_split_batched<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(jobs_dev, njobs, jb);
    return launch_check("batched split launch");
  }
  return GBD_OK;
}

int launch_magplane_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t split_blocks,
                            cudaStream_t s, int prec, const unsigned int* retry_if) {
  if (njobs <= 0 || split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "grouped: too many split blocks");
  static thread_local JobBegins jb;
  job_begins(jobs_host, njobs, kBySplitTile, jb);
  unsigned g = (unsigned)split_blocks;
  if (retry_if) {
    int sms = 0;
    if (int rc = current_device(nullptr, &sms)) return rc;
    const int64_t cap = 3 * (int64_t)sms;  // resident blocks of one wave
    if ((int64_t)g > cap) g = (unsigned)cap;
  }
  if (prec == kCertFP8) {
    if (retry_if) k_magplane_batched<true, true><<<g, kSplitThreads, 0, s>>>(jobs_dev, njobs, split_blocks, retry_if, jb);
    else k_magplane_batched<true, false><<<g, kSplitThreads, 0, s>>>(jobs_dev, njobs, split_blocks, nullptr, jb);
  } else {
    if (retry_if) k_magplane_batched<false, true><<<g, kSplitThreads, 0, s>>>(jobs_dev, njobs, split_blocks, retry_if, jb);
    else k_magplane_batched<false, false><<<g, kSplitThreads, 0, s>>>(jobs_dev, njobs, split_blocks, nullptr, jb);
  }
  return launch_check("batched magnitude plane launch");
}

int launch_residue_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, const ModSplit& mp,
                           int64_t split_blocks, cudaStream_t s) {
  if (njobs <= 0 || split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "grouped: too many split blocks");
  static thread_local JobBegins jb;
  job_begins(jobs_host, njobs, kBySplitTile, jb);
  k_residue_batched<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(jobs_dev, njobs, mp, jb);
  return launch_check("batched residue launch");
}

void prep_pair_blocks(PrepPair& pp, int64_t& exp_blocks, int64_t& split_blocks) {
  exp_blocks = 0;
  split_blocks = 0;
  prep_job_blocks(pp.j[0], exp_blocks, split_blocks);
  prep_job_blocks(pp.j[1], exp_blocks, split_blocks);
}

int launch_statplane_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t split_blocks,
                             int64_t max_rows, cudaStream_t s) {
  if (njobs <= 0 || split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "grouped: too many split blocks");
  if (njobs > 65535) return set_error(GBD_ERR_LIMIT, "grouped: too many modular problems for one batch");
  static thread_local JobBegins jb;
  job_begins(jobs_host, njobs, kBySplitTile, jb);
  k_statplane_batched<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(jobs_dev, njobs, jb);
  int rc = launch_check("batched statistics and planes launch");
  if (rc) return rc;
  // the rows of all jobs in equal ranges over one wave of warps when the begins fit the
  // parameters, else a block row per job
  const int64_t rows = job_begins(jobs_host, njobs, kByRow, jb);
  if (jb.n == njobs) {
    int sms = 0;
    if ((rc = current_device(nullptr, &sms))) return rc;
    const int64_t blocks = (rows + 7) / 8 < 8 * (int64_t)sms ? (rows + 7) / 8 : 8 * (int64_t)sms;
    if (blocks > 0) k_rowstats_flat<<<(unsigned)blocks, 256, 0, s>>>(jobs_dev, njobs, rows, jb);
  } else {
    const int64_t gx = (max_rows + 7) / 8 < 64 ? (max_rows + 7) / 8 : 64;  // warps per row, blocks per job
    k_rowstats_batched<<<dim3((unsigned)(gx > 0 ? gx : 1), (unsigned)njobs), 256, 0, s>>>(jobs_dev);
  }
  return launch_check("batched row statistics launch");
}


int launch_exponents_pair(const PrepPair& pp, int64_t exp_blocks, void* zero, size_t zero_bytes, cudaStream_t s) {
  if (exp_blocks <= 0) return GBD_OK;
  if (exp_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "too many exponent blocks");
  const bool direct = pp.j[0].K <= kRedChunk;  // both sides share K: one block per row
  if (!direct) {  // several blocks per row merge atomically into zeroed arrays
    const int64_t rmax = pp.j[0].R > pp.j[1].R ? pp.j[0].R : pp.j[1].R;
    const unsigned gx = (unsigned)((rmax + 255) / 256 < 1024 ? (rmax + 255) / 256 : 1024);
    k_prep_init_pair<<<dim3(gx > 0 ? gx : 1, 2), 256, 0, s>>>(pp);
    int rc = launch_check("exponent initialisation launch");
    if (rc) return rc;
  }
  k_exponents_pair<<<(unsigned)exp_blocks, 256, 0, s>>>(pp, direct, static_cast<uint4*>(zero),
                                                        (int64_t)(zero_bytes / sizeof(uint4)));
  return launch_check("exponent launch");
}

int launch_magnitudes_pair(const PrepPair& pp, int64_t exp_blocks, cudaStream_t s) {
  if (exp_blocks <= 0) return GBD_OK;
  k_magnitudes_pair<<<(unsigned)exp_blocks, 256, 0, s>>>(pp, pp.j[0].K <= kRedChunk);
  return launch_check("magnitude launch");
}

int launch_statplane_pair(const PrepPair& pp, int64_t split_blocks, unsigned int* tex, unsigned int* norms,
                          cudaStream_t s) {
  if (split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "too many split blocks");
  k_statplane_pair<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(pp);
  int rc = launch_check("statistics and planes launch");
  if (rc) return rc;
  const int64_t rmax = pp.j[0].R > pp.j[1].R ? pp.j[0].R : pp.j[1].R;
  const int64_t gx = (rmax + 7) / 8 < 4096 ? (rmax + 7) / 8 : 4096;  // a warp per row
  k_rowstats_pair<<<dim3((unsigned)(gx > 0 ? gx : 1), 2), 256, 0, s>>>(pp, tex, norms);
  return launch_check("row statistics launch");
}

int launch_residue_pair(const PrepPair& pp, const ModSplit& mp, int64_t split_blocks, cudaStream_t s) {
  if (split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "too many split blocks");
  k_residue_pair<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(pp, mp);
  return launch_check("residue launch");
}

int launch_split_pair(const PrepPair& pp, int64_t split_blocks, cudaStream_t s) {
  if (split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "too many split blocks");
  k_split_pair<<<(unsigned)split_blocks, kSplitThreads, 0, s>>>(pp);
  return launch_check("split launch");
}

int launch_magplane_pair(const PrepPair& pp, int prec, unsigned int* tex, int64_t split_blocks, cudaStream_t s,
                         const ModPlan* gate) {
  if (split_blocks <= 0) return GBD_OK;
  if (split_blocks > 0x7FFFFFFF) return set_error(GBD_ERR_LIMIT, "too many split blocks");
  const int64_t K = pp.j[0].K;
  unsigned g = (unsigned)split_blocks;
  if (gate) {  // a retry: usually returns at once, so one wave of blocks loops over the rest
    int sms = 0;
    if (int rc = current_device(nullptr, &sms)) return rc;
    const int64_t cap = 3 * (int64_t)sms;
    if ((int64_t)g > cap) g = (unsigned)cap;
  }
  if (prec == kCertFP8)
    k_magplane_pair<true><<<g, kSplitThreads, 0, s>>>(pp, plane_scale(K, prec), plane_pitch(K, prec), tex, gate,
                                                      split_blocks);
  else
    k_magplane_pair<false><<<g, kSplitThreads, 0, s>>>(pp, plane_scale(K, prec), plane_pitch(K, prec), tex, gate,
                                                       split_blocks);
  return launch_check("magnitude plane launch");
}


}  // namespace emu
}  // namespace gbd
