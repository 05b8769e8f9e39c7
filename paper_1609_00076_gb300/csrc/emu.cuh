// emu.cuh -- internal interfaces of the split (Ozaki-scheme) emulation of DGEMM.
//
// Method: Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012), in fixed-point digit form:
//   1. row exponents sigma_i of op(A) and column exponents tau_j of op(B);
//   2. s digits of kDigitBits bits per entry (truncation of the scaled value);
//   3. for every level g = 2..s+1 the exact integer sum over the digit pairs
//      t + u = g, computed on the BF16 tensor cores with FP32 accumulation that is
//      exact by construction (all partial sums are integers below 2^24);
//   4. C := beta*C; then, segment by segment of the inner dimension, the levels are
//      taken from the smallest in groups of up to kGroupLevels consecutive levels
//      whose sums are combined exactly in 64-bit integers,
//          Y = sum_{g in group} P_g 2^(b (h - g))   (h the group's smallest level),
//      and C := fma(alpha*2^(sigma_i + tau_j - h*b), Y, C) in FP64, once per group.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gbd {
namespace emu {

constexpr int kDigitBits = 7;      // digits in [-127, 127]: exact in BF16, products < 2^14
constexpr int kMaxSlices = 9;      // s * kDigitBits <= 63 bits of the scaled magnitude
constexpr int kBK = 64;            // k elements per pipeline stage (128 bytes of BF16)
constexpr int kChunkBlocks = 16;   // k-blocks per exact FP32 chunk: 1024 * 127^2 < 2^24
constexpr int kSegBlocks = 128;    // k-blocks per integer level segment: 9 * 8192 * 127^2 < 2^31
constexpr int kGroupLevels = 4;    // levels per exact group: 2^30.2 * (1 + 2^7 + 2^14 + 2^21) < 2^52
constexpr int kParkSlots = 2 * kGroupLevels;  // parked level sums: the group being drained + the pending one
constexpr int kExpEmpty = (int)0x80808080;  // exponent of a row/column with no non-zero entry

// Layout of the caller's workspace (every array 256-byte aligned).
// Partials of the one-pass statistics of one operand side, per row and 64-wide k tile ([R][nkt]
// each): the tile's largest exponent (kExpEmpty: no non-zero finite entry), a non-finite flag, the
// smallest frexp exponent of a non-zero entry and the smallest exponent of a lowest set bit
// (kEminNone: none), and the magnitude and square sums relative to the tile's exponent.
struct StatSide {
  int* e;
  int* b;
  int* lo;
  int* low;
  float* s;
  float* q;
  int nkt;
};

struct Workspace {
  int* sigA;        // [m] row exponents of op(A)
  int* sigB;        // [n] column exponents of op(B)
  int* badA;        // [m] non-zero when the row holds Inf/NaN
  int* badB;        // [n]
  unsigned long long* muA;  // [m] sum_p |a_ip| 2^-sigma_i in 32.32 fixed point (automatic slice counts)
  unsigned long long* muB;  // [n]
  float* stats;     // [4] min mu, min nu, any bad row, any bad column (grouped plans)
  unsigned int* cert;  // [kCertWords] the certification's maxima and exactness widths
  int* eminA;       // [m] smallest exponent of a row's non-zero entries (the certification)
  int* eminB;       // [n]
  StatSide st[2];   // automatic slices: the one-pass statistics' tile partials of op(A), op(B)^T
  uint16_t* DA;     // [s][m][kp] BF16 digit slices of op(A), k contiguous
  uint16_t* DB;     // [s][n][kp] BF16 digit slices of op(B)^T, k contiguous
  double* scratch;     // [scratch_ctas][128 * 256] FP64 running sums of the two-SM kernel
  int32_t* scratch_p;  // [scratch_ctas][kParkSlots][128 * 256] parked integer level sums of the two-SM kernel
  int scratch_ctas;
  int64_t kp;       // k rounded up to 8 (16-byte rows for the tensor maps)
  // one-SM kernel with a split inner dimension (small m x n, deep k; see split_count)
  int splits;                  // sub-ranges per k segment, 1 = no split
  unsigned long long* ysum;    // [tiles][segments][groups][128 x 128] exact group sums
  unsigned int* tile_done;     // [tiles] finished items
  size_t zero_bytes;           // ysum and tile_done are contiguous and zeroed before each call
};

constexpr int kMaxPairCtas = 256;  // scratch slots reserved for the two-SM kernel (128 pairs)

// Sub-ranges per k segment for the one-SM kernel on a single problem.  Few output tiles
// leave most SMs idle; cutting each 8192-deep segment of a tile into sub-ranges (at least two
// k-blocks each) gives about kSplitTargetItems work items.  The items' group sums are added
// as exact integers, so the result does not depend on the count, which is a function of the
// sizes alone (the workspace size needs no device).
constexpr int kSplitTargetItems = 152;
int split_count(int64_t m, int64_t n, int64_t k);

// bytes needed for (m, n, k, s) and, when base != nullptr, the pointers into it
size_t layout(int64_t m, int64_t n, int64_t k, int s, void* base, Workspace* ws, bool pair_scratch = true);
// min over rows of muA, over columns of muB, any bad row, any bad column -> stats[0..3]
int launch_min_stats(const unsigned long long* muA, int64_t m, const unsigned long long* muB, int64_t n,
                     const int* badA, const int* badB, float* stats, cudaStream_t s);

// One operand side of one problem for the preparation kernels.  Rows r of op(X) (R rows, K
// columns): element (r, p) is X[p*ld + r] when rows_contig, X[r*ld + p] otherwise.
struct PrepJob {
  const double* X;
  int64_t ld, R, K;
  int* sig;
  int* bad;
  unsigned long long* mu;  // magnitude sums in 32.32 fixed point (automatic slice counts), or null
  uint16_t* D;
  int64_t kp;
  int rows_contig, slices;
  int64_t exp_begin, split_begin;  // first block of this job in the batched launches
  int exp_gx, split_gx;            // blocks along the first grid dimension of each launch
  // grouped modular problems: the side's exactness-width word and the problem's device plan
  unsigned int* tex;
  const struct ModPlan* plan;
  // the smallest frexp exponent of each row's non-zero finite entries (atomic minimum by the
  // magnitude planes; kEminNone until then), or null
  int* emin;
  // the modular emulation's automatic mode: the one-pass statistics' tile partials, and (grouped
  // problems) the words that receive the side's largest square-sum bound (float bits) and, in
  // `tex`, its exactness width
  StatSide st;
  unsigned int* norm;
};
constexpr int kEminNone = 0x7F7F7F7F;  // a row without a non-zero finite entry (memset byte 0x7F)
// fills j's block ranges, advancing the running block counts of both launches
void prep_job_blocks(PrepJob& j, int64_t& exp_blocks, int64_t& split_blocks);
// The first block of every job of a batched launch (exponent blocks, 64 x 64 split tiles or rows),
// passed by value in the kernel parameters when there are at most kBeginCache jobs: a
// block then finds its job by a binary search in constant memory instead of one through the job
// table in device memory (a chain of dependent loads per block)
constexpr int kBeginCache = 1900;
struct JobBegins {
  int n;  // jobs whose begins are here (0: search the table)
  int pad;
  int64_t b[kBeginCache];
};
enum JobNumbering { kByExponentBlock = 0, kBySplitTile = 1, kByRow = 2 };
// fills `out` from the host copy of the job table; returns the launch's block count
int64_t job_begins(const PrepJob* jobs_host, int njobs, JobNumbering which, JobBegins& out);

// Both operand sides of one problem (j[0] = op(A), j[1] = op(B)^T), passed to the kernels by
// value: a single call prepares them with one launch per step.
struct PrepPair {
  PrepJob j[2];
};
void prep_pair_blocks(PrepPair& pp, int64_t& exp_blocks, int64_t& split_blocks);
// exponents (and, when the jobs carry magnitude arrays, their zeroing) of both sides; with
// K <= 1024 every row has one block, which stores its result and needs no initialisation
int launch_exponents_pair(const PrepPair& pp, int64_t exp_blocks, void* zero, size_t zero_bytes, cudaStream_t s);
int launch_magnitudes_pair(const PrepPair& pp, int64_t exp_blocks, cudaStream_t s);
// The modular emulation's automatic mode, both sides in one pass over the operands: per row and
// 64-wide k tile the partial statistics (the jobs' `st`) and the FP8 magnitude planes relative to
// the tile's exponent (into the jobs' D, pitch round_up(K, 16)); then, a warp per row, sig, bad, mu
// and emin, the planes moved to each row's sigma, and the sides' exactness widths (tex[2]) and
// square-sum bounds (norms[2], float bits) by atomic maxima (the words zeroed beforehand).  Two
// launches.
int launch_statplane_pair(const PrepPair& pp, int64_t split_blocks, unsigned int* tex, unsigned int* norms,
                          cudaStream_t s);
int launch_split_pair(const PrepPair& pp, int64_t split_blocks, cudaStream_t s);

// ---- modular emulation (Ozaki scheme II) ----
// precision of the magnitude planes: BF16 (7 stored fraction bits) or FP8 E5M2 (2 bits, products on
// the FP8 tensor-core rate)
constexpr int kCertBF16 = 0;
constexpr int kCertFP8 = 1;
constexpr int kMaxModuli = 16;  // the product of the moduli stays below 2^126
// pairwise coprime moduli up to 256 (greedily from 256 down), so that every symmetric
// residue is at most 128 in magnitude: exact in BF16, products at most 2^14
constexpr int kModuli[kMaxModuli] = {256, 255, 253, 251, 247, 241, 239, 233,
                                     229, 227, 223, 217, 211, 199, 197, 193};
// The modular emulation's choice for one call, written on the device (so that the automatic
// mode needs no host round trip) and read by every later kernel of the call.
struct ModPlan {
  int t;         // integer bits
  int n;         // moduli used (1 when infeasible)
  int feasible;  // 0: the target needs more than kMaxModuli moduli; the call writes NaN
  int want;      // the bits the target asked for (also when infeasible; 63: none up to 62)
  int exact;     // automatic mode: 1 when t is the exactness width (no truncation error)
  int pad;
  double rho, gamma, bound;  // automatic mode: the certification's maxima and the certified bound
};
// One problem of a grouped launch of the modular products (device table entry; the tensor
// maps keep it 64-byte aligned).  Its plan is made on the device by every run.
struct ModTableEntry {
  CUtensorMap tmA;  // residue planes of op(A): dims {k, m, kMaxModuli}, box {64, 128, 1}
  CUtensorMap tmB;  // residue planes of op(B)^T: dims {k, n, kMaxModuli}, box {64, 128, 1}
  int64_t m, n;
  const ModPlan* plan;  // the problem's t, n and feasibility
  uint8_t* park;        // the problem's parked residues (layout of ModArgs::park)
  int64_t tile_begin;   // first tile of this problem in the launch
  int nkb, tiles_m, group_m, num_tiles;  // tiles of 128 x 128, or 256 x 256 in the two-SM launch
  int park_mods, nbn;   // moduli per block of the park array; 128-column blocks of C
};
// The reconstruction of one product from its parked residues: every 128 x 128 block of C (in a
// batched launch, the jobs' blocks one after the other from blk_begin)
struct CrtJob {
  const uint8_t* park;  // [nbm * nbn blocks][park_mods][128 x 128 bytes]
  const ModPlan* plan;
  double* C;
  const int* sigA;      // row exponents of op(A) (and non-finite flags)
  const int* badA;
  const double* cs;     // [n] alpha 2^(tau_j - 2t) (NaN for a column with a non-finite entry)
  int64_t m, n, ldc;
  double beta;
  int64_t blk_begin;
  int park_mods, nbm, nbn;
  int tri;              // 0: all of C; 1: its lower triangle (i >= j); 2: its upper one
  int skip_infeasible;  // grouped: a problem whose plan is infeasible is left to the FP64 kernel
  int pad;
};
// the device plan of one problem of a grouped launch, and its column scales
struct ModPlanJob {
  const unsigned int* words;  // the problem's certification words
  ModPlan* plan;
  int64_t k;
  double tol;   // the target (already the FP64 bound when the caller gave none)
  int fixed_t;  // > 0: given bits (no certification)
  int pad;
};
struct ColJob {
  const int* sigB;
  const int* badB;
  double* cs;
  const ModPlan* plan;
  double alpha;
  int64_t n;
};
// residue split parameters: all kMaxModuli moduli (as float), 1/p, and 256^d mod p for
// d = 0..3 (wlo) and 4..7 (whi) packed one byte per d; t and n come from the plan
struct ModSplit {
  float pf[kMaxModuli];
  float inv[kMaxModuli];
  uint32_t wlo[kMaxModuli], whi[kMaxModuli];
  uint32_t wbias[kMaxModuli];  // 0x4B000000 + (-2^23 mod p): the byte sum read as 2^23 + s in FP32
  const ModPlan* plan;
};
// residue slices D[i][r][kp] of both sides (slices = n) from the rounded scaled integers
int launch_residue_pair(const PrepPair& pp, const ModSplit& mp, int64_t split_blocks, cudaStream_t s);
// grouped modular problems: the magnitude planes (FP8 E5M2) of every job into its D, widths to
// its tex; then, after the plans, the residues of every job with its problem's plan (nothing for
// an infeasible plan)
// (jobs_host: the host copy of the device job table jobs_dev, for the block begins)
int launch_magplane_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t split_blocks,
                            cudaStream_t s, int prec = kCertFP8, const unsigned int* retry_if = nullptr);
int launch_residue_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, const ModSplit& mp,
                           int64_t split_blocks, cudaStream_t s);
// exponents: initialise, then one launch for every job; split: one launch for every job
int launch_prep_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t exp_blocks,
                        int64_t split_blocks, bool exponents, bool split, cudaStream_t s);
// grouped modular problems: launch_statplane_pair's three steps over every job (each job's width
// and norm words): the same arithmetic in the same order, so a problem gets the same statistics
// and planes alone and in a batch
int launch_statplane_batched(const PrepJob* jobs_dev, const PrepJob* jobs_host, int njobs, int64_t split_blocks,
                             int64_t max_rows, cudaStream_t s);

// ---- the certified precision choice (emu_cert.cu, emu_split.cu) ----
// The choice certifies, for every element with a non-zero |A||B| term, that the a-priori
// truncation bound stays within (tol - r u) (|op(A)||op(B)|)_ij (r u: the final roundings).
// cert words (device, zeroed before the magnitude planes): rhoA = max_i mu_i / min_j G_ij, rhoB =
// max_j nu_j / min_i G_ij and gamma = 1 / min G_ij (float bits; G the certified lower bound of
// (|A||B|)_ij 2^-(sigma_i + tau_j)), and the exactness widths of op(A) and op(B).
constexpr int kCertRhoA = 0, kCertRhoB = 1, kCertGamma = 2, kCertTexA = 3, kCertTexB = 4;
// the modular emulation's automatic mode also keeps, from the exponent and magnitude pass, upper
// bounds of max_i ||a^_i||_2^2 and max_j ||b^_j||_2^2 (rows of op(A) and columns of op(B) scaled by
// 2^-sigma_i and 2^-tau_j; float bits), which bound |A'B'| for the moduli count
constexpr int kCertNormA = 5, kCertNormB = 6;
// two sets of words: the FP8 certification's, then (kCertRetry on) the BF16 one's, which runs only
// when the FP8 planes' looser bound leaves the target out of reach
constexpr int kCertRetry = 8;
constexpr int kCertWords = 16;
// rho = rhoA + rhoB (rounded up) and gamma from the words
__host__ __device__ inline void cert_rho_gamma(const unsigned int* w, double* rho, double* gamma) {
  float a, b, g;
  memcpy(&a, &w[kCertRhoA], 4);
  memcpy(&b, &w[kCertRhoB], 4);
  memcpy(&g, &w[kCertGamma], 4);
  *rho = ((double)a + (double)b) * (1.0 + 1e-15);
  *gamma = (double)g;
}
// the planes' precision of the emulations' automatic modes: FP8 unless GBD_CERT_DTYPE=bf16
int cert_prec_default();
// scale exponent S of the magnitude planes at inner dimension k (k 2^(2S) < 2^124)
int plane_scale(int64_t k, int prec);
// row pitch of a plane, in elements (16 bytes at least per row)
int64_t plane_pitch(int64_t k, int prec);
// magnitude planes of both sides into their jobs' D (one plane each); widths to tex[0], tex[1];
// with a gate, nothing is done when the gate's plan is feasible (the retry of the certification)
int launch_magplane_pair(const PrepPair& pp, int prec, unsigned int* tex, int64_t split_blocks, cudaStream_t s,
                         const struct ModPlan* gate = nullptr);
// the certification product of the planes PA [m][pitch], PB [n][pitch]: rho and gamma into
// words[0..1]; Lout (optional, m x n, leading dimension ldl) receives the lower bound of (|A||B|)_ij
int launch_cert(int64_t m, int64_t n, int64_t k, int prec, const void* PA, const void* PB,
                const unsigned long long* muA, const unsigned long long* muB, const int* badA, const int* badB,
                const int* sigA, const int* sigB, const int* eminA, const int* eminB, unsigned int* words,
                double* Lout, int64_t ldl, int sms, cudaStream_t stream, const struct ModPlan* gate = nullptr);

// Arguments of the certification product of one problem (emu_cert.cu)
struct CertArgs {
  int64_t m, n;
  int nkb, chunk_blocks, tiles_m, num_tiles, group_m;
  float f;         // (1 - delta) 2^-2S, rounded down
  float slack;     // k (2 w + w^2), rounded up
  float mu_scale;  // upper-bound factor of the magnitude sums
  const unsigned long long* muA;  // [m] sum_p |a^_ip| in 32.32 fixed point
  const unsigned long long* muB;  // [n]
  const int* badA;
  const int* badB;
  const int* sigA;
  const int* sigB;
  const int* eminA;     // [m] smallest exponent of each row's non-zero entries (kEminNone: none)
  const int* eminB;     // [n]
  float kinv;           // 1/k, rounded up
  const struct ModPlan* gate;  // the retry: nothing to do when this plan is already feasible
  unsigned int* words;  // the certification words: rhoA, rhoB, gamma (bits of non-negative floats)
  double* L;            // optional [m x n] output G_ij 2^(sigma_i + tau_j), leading dimension ldl
  int64_t ldl;
  unsigned int* err;
};

// one problem of a grouped certification launch (FP8 planes, one SM per 128 x 128 tile)
struct CertTableEntry {
  CUtensorMap tmA;  // the FP8 magnitude plane of op(A): dims {k, m, 1}, box {128, 128, 1}
  CUtensorMap tmB;
  CertArgs a;
  int64_t tile_begin;  // first tile of this problem in the launch
};
int make_cert_entry(int64_t m, int64_t n, int64_t k, int prec, const void* PA, const void* PB,
                    const unsigned long long* muA, const unsigned long long* muB, const int* badA, const int* badB,
                    const int* sigA, const int* sigB, const int* eminA, const int* eminB, unsigned int* words,
                    const struct ModPlan* gate, CertTableEntry* e);
// run_if: when given, the launch returns at once unless *run_if is non-zero (the BF16 retry)
int launch_cert_grouped(const CertTableEntry* table_dev, int count, int total_tiles, int prec, int sms,
                        cudaStream_t stream, const unsigned int* run_if = nullptr);

constexpr double kUnitRoundoff = 1.1102230246251565e-16;  // 2^-53
// exactness width of the modular integers: t at which every scaled entry is an integer (0: both
// sides zero), from the two side widths
__host__ __device__ inline int cert_exact_width(int texA, int texB) { return texA > texB ? texA : texB; }
// Modular emulation: the smallest t in 1..62 with 2^(-t-1) (rho + k 2^(-t-1) gamma) <= tol - 3u,
// or the exactness width when smaller (and tol >= 2u: an exact product keeps only the rounding
// of its conversion and of the update); 63 when neither exists.  *bound: the certified
// relative truncation bound at the choice (0 when exact).
__host__ __device__ inline int cert_mod_bits(double rho, double gamma, int texA, int texB, int64_t k, double tol,
                                             double* bound, int* exact) {
  const double kd = (double)k, tau = tol - 3.0 * kUnitRoundoff;
  int t = 63;
  double b = 0.0;
  if (tau > 0.0)
    for (int tt = 1; tt <= 62; ++tt) {
      const double h = ldexp(1.0, -tt - 1);
      const double bb = h * (rho + kd * h * gamma);
      if (bb <= tau) {
        t = tt;
        b = bb;
        break;
      }
    }
  int ex = 0;
  const int tx = cert_exact_width(texA, texB);
  if (tx <= 62 && tol >= 2.0 * kUnitRoundoff) {
    const int te = tx < 1 ? 1 : tx;
    if (te < t) {
      t = te;
      b = 0.0;
      ex = 1;
    }
  }
  if (bound) *bound = b;
  if (exact) *exact = ex;
  return t;
}
// Split emulation: the smallest s in 1..kMaxSlices with 2^-7s (rho + (s-1)(1+2^-7) k gamma) <=
// tol - (3g + 3)u, g = ceil(k / 8192) segments, or the slices that make the digits exact and keep
// every digit product (ceil(tA/7) + ceil(tB/7) - 1) when fewer, if tol covers their g ceil(s/4) + 1
// roundings; kMaxSlices + 1 when neither exists.
__host__ __device__ inline int cert_split_slices(double rho, double gamma, int texA, int texB, int64_t k,
                                                 double tol, double* bound, int* exact) {
  const double kd = (double)k;
  const double segs = (double)((k + 8191) / 8192);
  const double tau = tol - (3.0 * segs + 3.0) * kUnitRoundoff;
  int s = kMaxSlices + 1;
  double b = 0.0;
  if (tau > 0.0)
    for (int ss = 1; ss <= kMaxSlices; ++ss) {
      const double bb = ldexp(1.0, -kDigitBits * ss) * (rho + (ss - 1) * (1.0 + ldexp(1.0, -kDigitBits)) * kd * gamma);
      if (bb <= tau) {
        s = ss;
        b = bb;
        break;
      }
    }
  int ex = 0;
  const int dA = (texA + kDigitBits - 1) / kDigitBits, dB = (texB + kDigitBits - 1) / kDigitBits;
  int sx = dA + dB - 1;
  if (sx < 1) sx = 1;
  if (sx <= kMaxSlices && sx < s && tol >= (segs * (double)((sx + kGroupLevels - 1) / kGroupLevels) + 1.0) * kUnitRoundoff) {
    s = sx;
    b = 0.0;
    ex = 1;
  }
  if (bound) *bound = b;
  if (exact) *exact = ex;
  return s;
}

struct GemmParams {
  int64_t m, n, k;
  int slices;
  double alpha, beta;
  double* C;
  int64_t ldc;
  const int* sigA;
  const int* sigB;
  const int* badA;
  const int* badB;
};
int launch_slice_gemm(const GemmParams& p, const Workspace& ws, cudaStream_t s);

// One problem of a grouped launch of the one-SM slice kernel (device table entry).
struct EmuTableEntry {  // CUtensorMap members keep it 64-byte aligned
  CUtensorMap tmA;  // digit slices of op(A): dims {k, m, s}, box {64, 128, 1}
  CUtensorMap tmB;  // digit slices of op(B)^T: dims {k, n, s}, box {64, BN, 1}
  int64_t m, n, k, ldc;
  double alpha, beta;
  double* C;
  const int* sigA;
  const int* sigB;
  const int* badA;
  const int* badB;
  int64_t tile_begin;  // first index of this problem in the grouped tile sequence
  int slices, nkb, tiles_m, group_m, num_tiles, pad;
};
constexpr int kGroupedBN = 128;  // column tile of the grouped one-SM slice kernel
// grouped problems with m, n >= kGroupedPairMinMN and k >= kGroupedPairMinK use the two-SM 256 x 256
// kernel.  Measured per SM, it needs k >= 1024 to amortise its deferred FP64 update and is about
// 1.5x the one-SM kernel from k = 2048; in a batch its separate launch and the 256 x 256 padding
// have to be paid for as well, so only large problems qualify
constexpr int kGroupedPairMinMN = 1024;
constexpr int kGroupedPairMinK = 2048;

// tensor maps of one problem's slices for the grouped kernel
int encode_slice_maps(const Workspace& ws, int64_t m, int64_t n, int64_t k, int slices, EmuTableEntry* e);
// one launch over `count` problems of a device table that all use `slices` slices (entries
// sorted by decreasing tile cost, tile_begin counted from the first of them)
int launch_slice_gemm_grouped(const EmuTableEntry* table_dev, int count, int total_tiles, int slices,
                              cudaStream_t stream);
// the same with the two-SM kernel on 256 x 256 tiles (entries tiled by 256 x 256); scratch and
// scratch_p hold max_ctas running-sum slots and max_ctas x kParkSlots park slots of 128 x 256
int launch_slice_gemm_grouped_pair(const EmuTableEntry* table_dev, int count, int total_tiles, int slices,
                                   double* scratch, int32_t* scratch_p, int max_ctas, cudaStream_t stream);

// ---- grouped modular problems (emu_mod.cu) ----
// The modular problems of a grouped plan.  Every run certifies and plans each problem on the
// device (no host round trip), then computes all of them in one persistent launch of the
// table-driven one-SM product kernel; a problem whose plan is infeasible is skipped there and
// computed by the grouped FP64 kernel (its fallback entry tests the same plan).
struct ModGrouped {
  int count = 0;
  std::vector<int> index;                  // the caller's position of each problem
  std::vector<const ModPlan*> plans;       // the device plan of each problem
  std::vector<PrepJob> jobs;               // op(A), op(B)^T of each problem
  std::vector<CertTableEntry> cert;        // FP8 certification, then its BF16 retry (count each)
  std::vector<ModPlanJob> planjobs;
  std::vector<ColJob> coljobs;
  // in launch order: the pair_count problems of the two-SM launch (pair_tiles tiles of 256 x 256),
  // then those of the one-SM launch (mod_tiles tiles of 128 x 128), each part by decreasing k
  std::vector<ModTableEntry> table;
  int64_t exp_blocks = 0, split_blocks = 0;
  int cert_tiles = 0, mod_tiles = 0, pair_tiles = 0, pair_count = 0;
  // device memory in the grouped workspace
  PrepJob* jobs_dev = nullptr;
  CertTableEntry* cert_dev = nullptr;
  ModPlanJob* planjobs_dev = nullptr;
  ColJob* coljobs_dev = nullptr;
  ModTableEntry* table_dev = nullptr;
  unsigned int* words_dev = nullptr;       // kCertWords per problem
  // [0]: some problem's first plan found no feasible t (the BF16 retry runs); [1]: some problem's
  // final plan did (its FP64 fallback tiles run); [2]: the largest moduli count of a feasible plan
  unsigned int* flags_dev = nullptr;
  std::vector<CrtJob> crt;                 // the reconstructions, in the product table's order
  CrtJob* crt_dev = nullptr;
  int64_t crt_blocks = 0;
};
// Bytes of the grouped modular part for the problems probs[which[q]], q < count (host-only).
// With base, lays out the workspace from there and builds the host tables into g.
size_t mod_grouped_layout(const gbd_problem* probs, const int* which, int count, void* base, ModGrouped* g, int* rc);
// one run: preparation, certification, plans, residues, column scales and the products
int mod_grouped_run(const ModGrouped& g, int sms, cudaStream_t s);

}  // namespace emu
}  // namespace gbd
