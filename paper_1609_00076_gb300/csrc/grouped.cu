// grouped.cu -- many independent DGEMMs (native and emulated) in one launch each.
//
// A plan turns a host array of problems into device tables in the caller's
// workspace:
//  * native problems (and every problem's BLAS quick path) go to a persistent
//    FP64-MMA kernel whose CTAs take tiles from one atomic counter over the
//    concatenated tile space, longest tiles (largest k) first;
//  * emulated problems get their exponent and split kernels, then one persistent
//    launch of the table-driven one-SM tcgen05 slice kernel over all their tiles,
//    ordered by decreasing tile cost.
// Every tile computes exactly what the single-problem call computes (same k
// order, same epilogue), so a problem's result is the same bits alone and in any
// batch.  Running a plan issues only kernel launches and memsets on the stream,
// so it can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "emu.cuh"
#include "native_tile.cuh"

static_assert(sizeof(gbd_problem) == 112 && offsetof(gbd_problem, m) == 16 && offsetof(gbd_problem, A) == 56 &&
                  offsetof(gbd_problem, tol) == 104,
              "gbd_problem layout is part of the ABI");

namespace gbd {
namespace {

struct NativeTableEntry {
  NativeArgs a;
  int64_t tile_begin;
  int32_t ta, tb, tile, tiles_m;
  // the FP64 fallback of a modular problem: its tiles run only when the problem's device plan
  // found the target out of reach (otherwise the modular kernel computes it)
  const emu::ModPlan* only_if_infeasible;
  // inner-dimension split: `ksplit` parts per tile (work items tile * ksplit + part), each
  // tile's part slots at part + tile * ksplit * tile^2 and its arrival counter at done + tile
  int32_t ksplit, nkb;
  double* part;
  unsigned int* done;
};

// run_if: when given, the launch returns at once unless *run_if is non-zero (the fallback launch,
// which has work only when some modular plan found no certified bit count)
__global__ void __launch_bounds__(kNativeThreads)
    k_grouped_native(const NativeTableEntry* __restrict__ table, int count, int64_t total_tiles,
                     unsigned long long* __restrict__ counter, const unsigned int* __restrict__ run_if) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_tile;
  if (run_if && *run_if == 0u) return;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();  // every thread has read s_tile
    if (tile >= total_tiles) break;
    int lo = 0, hi = count - 1;  // last entry whose first tile is <= tile
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (table[mid].tile_begin <= tile) lo = mid;
      else hi = mid - 1;
    }
    const NativeTableEntry& e = table[lo];
    if (e.only_if_infeasible && e.only_if_infeasible->feasible) continue;  // uniform over the block
    const NativeArgs a = e.a;
    int64_t local = tile - e.tile_begin;
    KSplit split;
    const KSplit* ks = nullptr;
    if (e.ksplit > 1) {  // item = output tile * ksplit + part
      const int part = (int)(local % e.ksplit);
      local /= e.ksplit;
      split.kb0 = (int)((int64_t)part * e.nkb / e.ksplit);
      split.kb1 = (int)((int64_t)(part + 1) * e.nkb / e.ksplit);
      split.parts = e.ksplit;
      split.index = part;
      split.part = e.part + local * e.ksplit * (int64_t)e.tile * e.tile;
      split.done = e.done + local;
      ks = &split;
    }
    const int64_t tm = local % e.tiles_m, tn = local / e.tiles_m;
    const int code = (e.ta << 2) | (e.tb << 1) | (e.tile == 32 ? 1 : 0);
    switch (code) {
      case 0: native_tile<false, false, 64, 64, false>(a, nullptr, nullptr, tm * 64, tn * 64, smem_raw, ks); break;
      case 1: native_tile<false, false, 32, 32, false>(a, nullptr, nullptr, tm * 32, tn * 32, smem_raw, ks); break;
      case 2: native_tile<false, true, 64, 64, false>(a, nullptr, nullptr, tm * 64, tn * 64, smem_raw, ks); break;
      case 3: native_tile<false, true, 32, 32, false>(a, nullptr, nullptr, tm * 32, tn * 32, smem_raw, ks); break;
      case 4: native_tile<true, false, 64, 64, false>(a, nullptr, nullptr, tm * 64, tn * 64, smem_raw, ks); break;
      case 5: native_tile<true, false, 32, 32, false>(a, nullptr, nullptr, tm * 32, tn * 32, smem_raw, ks); break;
      case 6: native_tile<true, true, 64, 64, false>(a, nullptr, nullptr, tm * 64, tn * 64, smem_raw, ks); break;
      default: native_tile<true, true, 32, 32, false>(a, nullptr, nullptr, tm * 32, tn * 32, smem_raw, ks); break;
    }
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int default_tile(int64_t, int64_t) {
  // Measured on GB300 (autotune.py, output edges 32..4095): 32 x 32 tiles are never
  // slower in the grouped kernel (FP64-bound at large sizes, up to 3.8x faster at
  // small ones), so they are the default; the autotuner may still pick 64 per problem.
  return 32;
}

}  // namespace
}  // namespace gbd

struct gbd_plan {
  // native part
  std::vector<gbd::NativeTableEntry> native;
  int64_t native_tiles = 0;
  gbd::NativeTableEntry* native_dev = nullptr;
  // split-k native problems: their tiles' part slots and arrival counters (zeroed by the plan)
  double* ksplit_parts = nullptr;
  unsigned int* ksplit_done = nullptr;
  size_t ksplit_done_count = 0;
  unsigned long long* counter_dev = nullptr;  // [0] native launch, [1] fallback launch
  // the FP64 fallbacks of the modular problems: a second launch, after the native table, that runs
  // only when some modular plan found no certified bit count
  std::vector<gbd::NativeTableEntry> fallback;
  int64_t fallback_tiles = 0;
  // emulated part
  struct Emu {
    gbd_problem p;
    int index;   // position in the caller's problem array
    int slices;
    gbd::emu::Workspace ws;
  };
  std::vector<Emu> emu;
  std::vector<gbd::emu::EmuTableEntry> emu_table;
  gbd::emu::EmuTableEntry* emu_dev = nullptr;
  int64_t emu_tiles = 0;
  // one slice-product launch per kernel and slice count: table entries [first, first + count),
  // `tiles` tiles of 256 x 256 (pair) or 128 x 128
  struct Segment {
    int first, count, slices;
    bool pair;
    int64_t tiles;
  };
  std::vector<Segment> segments;
  // two-SM kernel scratch: FP64 running sums and parked level sums, per CTA
  double* pair_scratch = nullptr;
  int32_t* pair_scratch_p = nullptr;
  int pair_ctas = 0;
  // batched preparation: jobs 2q, 2q+1 are op(A) and op(B)^T of emulated problem q
  std::vector<gbd::emu::PrepJob> jobs;
  gbd::emu::PrepJob* jobs_dev = nullptr;
  float* stats_dev = nullptr;
  int64_t exp_blocks = 0, split_blocks = 0;
  // modular problems: prepared, certified and planned on the device by every run
  gbd::emu::ModGrouped mod;
};

namespace gbd {
namespace {

// Emulated problems large enough for the two-SM 256 x 256 kernel
// (the tile field chooses it: 256 the two-SM kernel, 128 the one-SM kernel, 0 this default)
bool pair_class(const gbd_problem& p) {
  if (p.tile == 256) return true;
  if (p.tile == 128) return false;
  return p.m >= emu::kGroupedPairMinMN && p.n >= emu::kGroupedPairMinMN && p.k >= emu::kGroupedPairMinK;
}

int default_tile(int64_t, int64_t);

// the effective inner-dimension split of a native problem (1: none)
int native_ksplit(const gbd_problem& p) {
  const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
  if (p.mode != GBD_MODE_NATIVE || quick || p.ksplit <= 1) return 1;
  const int64_t nkb = (p.k + kNativeBK - 1) / kNativeBK;
  return (int)(p.ksplit < nkb ? p.ksplit : nkb);
}
int native_edge(const gbd_problem& p) { return (p.mode == GBD_MODE_NATIVE && p.tile) ? p.tile : default_tile(p.m, p.n); }
int64_t native_tiles_of(const gbd_problem& p, int edge) { return ((p.m + edge - 1) / edge) * ((p.n + edge - 1) / edge); }

// Layout of the grouped workspace; with base == nullptr only the size is computed.
size_t grouped_layout(const gbd_problem* probs, int count, const int* slices_override, void* base, gbd_plan* plan) {
  size_t off = 256;  // tile counters (native launch, fallback launch)
  // split-k native problems: part slots (one tile of doubles per part) and a counter per tile
  size_t ks_doubles = 0, ks_counters = 0;
  for (int i = 0; i < count; ++i) {
    const int S = native_ksplit(probs[i]);
    if (S <= 1) continue;
    const int e = native_edge(probs[i]);
    const int64_t t = native_tiles_of(probs[i], e);
    ks_doubles += (size_t)t * S * e * e;
    ks_counters += (size_t)t;
  }
  const size_t o_ksp = off;
  off = up256(off + sizeof(double) * ks_doubles);
  const size_t o_ksd = off;
  off = up256(off + sizeof(unsigned int) * ks_counters);
  const size_t o_native = off;
  int nnat = 0, nemu = 0;
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
    if (p.mode == GBD_MODE_EMULATED && !quick) ++nemu;
    else ++nnat;  // native problems, quick returns and modular problems' fallback entries
  }
  // room for every problem: emulated ones whose target cannot be certified run natively
  off = up256(off + sizeof(NativeTableEntry) * (size_t)(nnat + nemu));
  const size_t o_emu = off;
  off = up256(off + sizeof(emu::EmuTableEntry) * (size_t)nemu);
  const size_t o_jobs = off;
  off = up256(off + sizeof(emu::PrepJob) * 2 * (size_t)nemu);
  const size_t o_stats = off;  // statistics, then the certification words of each emulated problem
  off = up256(off + sizeof(unsigned int) * emu::kCertWords * (size_t)nemu);
  // two-SM kernel scratch for the large emulated problems (at most one CTA pair per 256 x 256 tile)
  int64_t pair_tiles = 0;
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
    if (p.mode == GBD_MODE_EMULATED && !quick && pair_class(p)) pair_tiles += ((p.m + 255) / 256) * ((p.n + 255) / 256);
  }
  const int pair_ctas = (int)(2 * pair_tiles < emu::kMaxPairCtas ? 2 * pair_tiles : emu::kMaxPairCtas);
  const size_t o_pscr = off;
  off = up256(off + sizeof(double) * 128 * 256 * (size_t)pair_ctas);
  const size_t o_pscp = off;
  off = up256(off + sizeof(int32_t) * emu::kParkSlots * 128 * 256 * (size_t)pair_ctas);
  // modular problems: their workspaces, tables and the product launch's park slots
  std::vector<int> mod_which;
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
    if (p.mode == GBD_MODE_MODULAR && !quick) mod_which.push_back(i);
  }
  const size_t o_mod = off;
  int mrc = GBD_OK;
  off = up256(off + emu::mod_grouped_layout(probs, mod_which.data(), (int)mod_which.size(),
                                            (base && plan) ? static_cast<char*>(base) + o_mod : nullptr,
                                            (base && plan) ? &plan->mod : nullptr, &mrc));
  if (mrc && plan) plan->mod.count = -1;  // an invalid fixed bit count: reported by the plan
  int ei = 0;
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
    if (p.mode != GBD_MODE_EMULATED || quick) continue;
    int s = slices_override ? slices_override[i] : p.slices;
    if (s <= 0) s = emu::kMaxSlices;
    const size_t need = emu::layout(p.m, p.n, p.k, s, nullptr, nullptr, false);
    if (base && plan) emu::layout(p.m, p.n, p.k, s, static_cast<char*>(base) + off, &plan->emu[ei].ws, false);
    off = up256(off + need);
    ++ei;
  }
  if (base && plan) {
    plan->counter_dev = reinterpret_cast<unsigned long long*>(base);
    plan->ksplit_parts = reinterpret_cast<double*>(static_cast<char*>(base) + o_ksp);
    plan->ksplit_done = reinterpret_cast<unsigned int*>(static_cast<char*>(base) + o_ksd);
    plan->ksplit_done_count = ks_counters;
    plan->native_dev = reinterpret_cast<NativeTableEntry*>(static_cast<char*>(base) + o_native);
    plan->emu_dev = reinterpret_cast<emu::EmuTableEntry*>(static_cast<char*>(base) + o_emu);
    plan->jobs_dev = reinterpret_cast<emu::PrepJob*>(static_cast<char*>(base) + o_jobs);
    plan->stats_dev = reinterpret_cast<float*>(static_cast<char*>(base) + o_stats);
    plan->pair_scratch = reinterpret_cast<double*>(static_cast<char*>(base) + o_pscr);
    plan->pair_scratch_p = reinterpret_cast<int32_t*>(static_cast<char*>(base) + o_pscp);
    plan->pair_ctas = pair_ctas;
  }
  return off;
}

// the FP64-MMA table entry of a problem (quick: its C := beta C path, as a k = 0 problem)
NativeTableEntry native_entry(const gbd_problem& p, bool quick) {
  NativeTableEntry t;
  memset(&t, 0, sizeof(t));
  NativeArgs& a = t.a;
  a.m = p.m; a.n = p.n; a.k = quick ? 0 : p.k;
  a.alpha = quick ? 0.0 : p.alpha; a.beta = p.beta;
  a.A = p.A; a.lda = p.lda; a.B = p.B; a.ldb = p.ldb; a.C = p.C; a.ldc = p.ldc;
  a.err = device_error_word();
  a.vec_c = ((reinterpret_cast<uintptr_t>(p.C) & 15u) == 0 && (p.ldc & 1) == 0) ? 1 : 0;
  t.ta = trans_code(p.transa);
  t.tb = trans_code(p.transb);
  t.tile = (p.mode == GBD_MODE_NATIVE && p.tile) ? p.tile : default_tile(p.m, p.n);  // emulated tiles name kernels
  t.tiles_m = (int32_t)((p.m + t.tile - 1) / t.tile);
  t.ksplit = quick ? 1 : native_ksplit(p);
  t.nkb = (int32_t)((a.k + kNativeBK - 1) / kNativeBK);
  return t;
}

int validate(const gbd_problem* probs, int count) {
  if (count < 0 || (count > 0 && !probs)) return set_error(GBD_ERR_ARG, "grouped: bad problem array");
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    const int bad = check_dgemm_args(p.transa, p.transb, p.m, p.n, p.k, p.lda, p.ldb, p.ldc);
    if (bad) return set_error(GBD_ERR_ARG, "grouped problem %d: parameter %d had an illegal value", i, bad);
    if (p.mode != GBD_MODE_NATIVE && p.mode != GBD_MODE_EMULATED && p.mode != GBD_MODE_MODULAR)
      return set_error(GBD_ERR_ARG, "grouped problem %d: mode %d", i, p.mode);
    if (p.mode == GBD_MODE_EMULATED && (p.slices < 0 || p.slices > emu::kMaxSlices))
      return set_error(GBD_ERR_ARG, "grouped problem %d: slices %d", i, p.slices);
    if (p.mode == GBD_MODE_MODULAR && (p.slices < 0 || p.slices > 62))
      return set_error(GBD_ERR_ARG, "grouped problem %d: bits %d (0 automatic, or 1..62)", i, p.slices);
    if (p.mode == GBD_MODE_NATIVE && p.tile != 0 && p.tile != 32 && p.tile != 64)
      return set_error(GBD_ERR_ARG, "grouped problem %d: tile %d (0, 32 or 64)", i, p.tile);
    if (p.mode == GBD_MODE_EMULATED && p.tile != 0 && p.tile != 128 && p.tile != 256)
      return set_error(GBD_ERR_ARG, "grouped problem %d: tile %d (0, 128 or 256)", i, p.tile);
    if (p.mode == GBD_MODE_MODULAR && p.tile != 0 && p.tile != 128)
      return set_error(GBD_ERR_ARG, "grouped problem %d: tile %d (0 or 128)", i, p.tile);
    if (p.ksplit > 16) return set_error(GBD_ERR_ARG, "grouped problem %d: ksplit %d (0..16)", i, (int)p.ksplit);
    const int64_t lim = (int64_t)1 << 31;
    if (p.m >= lim || p.n >= lim || p.k >= lim || (p.m + 63) / 64 > 65535 || (p.n + 63) / 64 > 65535)
      return set_error(GBD_ERR_LIMIT, "grouped problem %d: size beyond the supported range", i);
  }
  return GBD_OK;
}

}  // namespace
}  // namespace gbd

extern "C" {

size_t gbd_dgemm_grouped_workspace_size(const gbd_problem* probs, int count) {
  if (count <= 0 || !probs) return 256;
  return gbd::grouped_layout(probs, count, nullptr, nullptr, nullptr);
}

int gbd_grouped_plan_create(const gbd_problem* probs, int count, void* workspace, size_t workspace_bytes,
                            int* slices_used, void* stream, gbd_plan** out) {
  using namespace gbd;
  if (!out) return set_error(GBD_ERR_ARG, "grouped: plan pointer is NULL");
  *out = nullptr;
  int rc = validate(probs, count);
  if (rc) return rc;
  rc = current_device(nullptr, nullptr);
  if (rc) return rc;
  const size_t need = gbd_dgemm_grouped_workspace_size(probs, count);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return set_error(GBD_ERR_WORKSPACE, "grouped: workspace must be 256-byte aligned and hold %zu bytes", need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gbd_plan* plan = new (std::nothrow) gbd_plan();
  if (!plan) return set_error(GBD_ERR_WORKSPACE, "grouped: host allocation failed");
  struct Guard {
    gbd_plan** keep;
    gbd_plan* p;
    ~Guard() {
      if (!*keep) delete p;
    }
  } guard{out, plan};

  // split problems; quick paths (alpha == 0 or k == 0) of both modes become k = 0 native tiles
  for (int i = 0; i < count; ++i) {
    const gbd_problem& p = probs[i];
    if (slices_used) slices_used[i] = 0;
    if (p.m == 0 || p.n == 0) continue;
    const bool quick = p.alpha == 0.0 || p.k == 0;
    if (p.mode == GBD_MODE_MODULAR && !quick) continue;  // the modular part (laid out below)
    if (p.mode == GBD_MODE_EMULATED && !quick) {
      gbd_plan::Emu e;
      e.p = p;
      e.index = i;
      e.slices = p.slices;
      plan->emu.push_back(e);
      continue;
    }
    if (quick && p.beta == 1.0) continue;  // nothing to do
    plan->native.push_back(native_entry(p, quick));
  }
  // the workspace holds one slice region per emulated problem (sized for the given or maximal slices)
  std::vector<int> s_override(count, 0);
  for (int i = 0; i < count; ++i) s_override[i] = probs[i].slices;
  grouped_layout(probs, count, s_override.data(), workspace, plan);
  if (plan->mod.count < 0) return GBD_ERR_LIMIT;  // a fixed bit count beyond 16 moduli (message set)
  // each modular problem's FP64 fallback, gated by its device plan
  for (int q = 0; q < plan->mod.count; ++q) {
    NativeTableEntry t = native_entry(probs[plan->mod.index[q]], false);
    t.only_if_infeasible = plan->mod.plans[q];
    plan->fallback.push_back(t);
  }

  // preparation jobs: op(A) and op(B)^T of every emulated problem
  cudaError_t e;
  plan->jobs.resize(2 * plan->emu.size());
  bool any_auto = false;
  for (size_t q = 0; q < plan->emu.size(); ++q) {
    const auto& em = plan->emu[q];
    const gbd_problem& p = em.p;
    const emu::Workspace& ws = em.ws;
    any_auto = any_auto || em.slices == 0;
    emu::PrepJob& ja = plan->jobs[2 * q];
    emu::PrepJob& jb = plan->jobs[2 * q + 1];
    memset(&ja, 0, sizeof(ja));
    memset(&jb, 0, sizeof(jb));
    // op(A) rows: A[p*lda + i] when 'N' (rows contiguous); op(B)^T rows: B[p*ldb + j] when 'T'
    ja.X = p.A; ja.ld = p.lda; ja.R = p.m; ja.K = p.k; ja.rows_contig = trans_code(p.transa) == 0;
    ja.sig = ws.sigA; ja.bad = ws.badA; ja.mu = ws.muA; ja.D = ws.DA; ja.kp = ws.kp; ja.emin = ws.eminA;
    jb.X = p.B; jb.ld = p.ldb; jb.R = p.n; jb.K = p.k; jb.rows_contig = trans_code(p.transb) != 0;
    jb.sig = ws.sigB; jb.bad = ws.badB; jb.mu = ws.muB; jb.D = ws.DB; jb.kp = ws.kp; jb.emin = ws.eminB;
    // automatic slices: the one-pass statistics' partials and the problem's certification words
    unsigned int* words = reinterpret_cast<unsigned int*>(plan->stats_dev) + emu::kCertWords * q;
    ja.st = ws.st[0]; ja.tex = words + emu::kCertTexA; ja.norm = words + emu::kCertNormA;
    jb.st = ws.st[1]; jb.tex = words + emu::kCertTexB; jb.norm = words + emu::kCertNormB;
    emu::prep_job_blocks(ja, plan->exp_blocks, plan->split_blocks);
    emu::prep_job_blocks(jb, plan->exp_blocks, plan->split_blocks);
  }
  // automatic slice counts, certified per problem: batched exponents and magnitude sums, then each
  // automatic problem's magnitude planes and certification product, one read-back for all
  if (any_auto) {
    int sms = 0;
    if ((rc = current_device(nullptr, &sms))) return rc;
    if ((e = cudaMemcpyAsync(plan->jobs_dev, plan->jobs.data(), sizeof(emu::PrepJob) * plan->jobs.size(),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "grouped: job table copy");
    unsigned int* words = reinterpret_cast<unsigned int*>(plan->stats_dev);  // kCertWords per emulated problem
    if ((e = cudaMemsetAsync(words, 0, sizeof(unsigned int) * emu::kCertWords * plan->emu.size(), s)) != cudaSuccess)
      return cuda_fail(e, "grouped: clearing the certification words");
    // one pass over every problem's operands: statistics and FP8 magnitude planes, as the single call
    int64_t max_rows = 0;
    for (const auto& j : plan->jobs) max_rows = j.R > max_rows ? j.R : max_rows;
    if ((rc = emu::launch_statplane_batched(plan->jobs_dev, plan->jobs.data(), (int)plan->jobs.size(), plan->split_blocks,
                                             max_rows, s)))
      return rc;
    const int prec = emu::cert_prec_default();
    if (prec == emu::kCertBF16 &&
        (rc = emu::launch_magplane_batched(plan->jobs_dev, plan->jobs.data(), (int)plan->jobs.size(), plan->split_blocks, s,
                                            prec)))
      return rc;
    for (size_t q = 0; q < plan->emu.size(); ++q) {
      const auto& em = plan->emu[q];
      if (em.slices != 0) continue;
      unsigned int* w = words + emu::kCertWords * q;
      if ((rc = emu::launch_cert(em.p.m, em.p.n, em.p.k, prec, em.ws.DA, em.ws.DB, em.ws.muA, em.ws.muB,
                                 em.ws.badA, em.ws.badB, em.ws.sigA, em.ws.sigB, em.ws.eminA, em.ws.eminB, w,
                                 nullptr, 0, sms, s)))
        return rc;
    }
    std::vector<unsigned int> cw(emu::kCertWords * plan->emu.size(), 0u);
    auto read_words = [&]() -> int {
      if ((e = cudaMemcpyAsync(cw.data(), words, sizeof(unsigned int) * cw.size(), cudaMemcpyDeviceToHost, s)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "grouped: reading the certification");
      return GBD_OK;
    };
    if ((rc = read_words())) return rc;
    // the slice count of problem q from its words of set `off` (0: the first certification, kCertRetry)
    auto slices_of = [&](size_t q, int off) {
      const auto& em = plan->emu[q];
      const unsigned int* w = &cw[emu::kCertWords * q + off];
      double rho, gamma;
      emu::cert_rho_gamma(w, &rho, &gamma);
      const double target = em.p.tol > 0.0 ? em.p.tol : 2.0 * (double)em.p.k * emu::kUnitRoundoff;
      return emu::cert_split_slices(rho, gamma, (int)w[emu::kCertTexA], (int)w[emu::kCertTexB], em.p.k, target,
                                    nullptr, nullptr);
    };
    // the FP8 planes' looser bound: the problems it leaves without a slice count, certified again
    // with BF16 planes
    if (prec == emu::kCertFP8) {
      bool again = false;
      for (size_t q = 0; q < plan->emu.size(); ++q) {
        const auto& em = plan->emu[q];
        if (em.slices != 0 || slices_of(q, 0) <= emu::kMaxSlices) continue;
        emu::PrepPair pp;
        pp.j[0] = plan->jobs[2 * q];
        pp.j[1] = plan->jobs[2 * q + 1];
        int64_t eb = 0, sb = 0;
        emu::prep_pair_blocks(pp, eb, sb);
        unsigned int* w = words + emu::kCertWords * q + emu::kCertRetry;
        if ((rc = emu::launch_magplane_pair(pp, emu::kCertBF16, w + emu::kCertTexA, sb, s))) return rc;
        if ((rc = emu::launch_cert(em.p.m, em.p.n, em.p.k, emu::kCertBF16, em.ws.DA, em.ws.DB, em.ws.muA, em.ws.muB,
                                   em.ws.badA, em.ws.badB, em.ws.sigA, em.ws.sigB, em.ws.eminA, em.ws.eminB, w,
                                   nullptr, 0, sms, s)))
          return rc;
        again = true;
      }
      if (again && (rc = read_words())) return rc;
    }
    // problems whose target no slice count can certify move to the FP64 path
    std::vector<gbd_plan::Emu> kept;
    std::vector<emu::PrepJob> kept_jobs;
    for (size_t q = 0; q < plan->emu.size(); ++q) {
      auto em = plan->emu[q];
      if (em.slices == 0) {
        em.slices = slices_of(q, 0);
        if (em.slices > emu::kMaxSlices && prec == emu::kCertFP8) em.slices = slices_of(q, emu::kCertRetry);
      }
      if (em.slices > emu::kMaxSlices) {
        plan->native.push_back(native_entry(em.p, false));
        continue;
      }
      kept.push_back(em);
      kept_jobs.push_back(plan->jobs[2 * q]);
      kept_jobs.push_back(plan->jobs[2 * q + 1]);
    }
    const bool dropped = kept.size() != plan->emu.size();
    plan->emu.swap(kept);  // the chosen slice counts
    plan->jobs.swap(kept_jobs);
    if (dropped) {  // renumber the preparation blocks of the remaining jobs
      plan->exp_blocks = 0;
      plan->split_blocks = 0;
      for (auto& j : plan->jobs) emu::prep_job_blocks(j, plan->exp_blocks, plan->split_blocks);
    }
  }
  for (size_t q = 0; q < plan->emu.size(); ++q) {
    plan->jobs[2 * q].slices = plan->emu[q].slices;
    plan->jobs[2 * q + 1].slices = plan->emu[q].slices;
    plan->jobs[2 * q].mu = nullptr;  // runs need no magnitude sums or spreads
    plan->jobs[2 * q + 1].mu = nullptr;
    plan->jobs[2 * q].emin = nullptr;
    plan->jobs[2 * q + 1].emin = nullptr;
  }
  // emulated table: tensor maps and tile counts.  Problems of the same kernel (two-SM for the large
  // ones) and slice count are contiguous (one launch each, most slices first), and the longest
  // tiles come first within them.
  std::vector<int> order(plan->emu.size());
  for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
  auto cost = [&](int q) {
    const auto& em = plan->emu[q];
    return (int64_t)em.slices * (em.slices + 1) / 2 * ((em.p.k + emu::kBK - 1) / emu::kBK);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const bool pa = pair_class(plan->emu[a].p), pb = pair_class(plan->emu[b].p);
    const int sa = plan->emu[a].slices, sb = plan->emu[b].slices;
    if (pa != pb) return pa;
    return sa != sb ? sa > sb : cost(a) > cost(b);
  });
  plan->emu_table.resize(plan->emu.size());
  plan->segments.clear();
  int64_t tiles = 0, seg_tiles = 0;
  for (size_t r = 0; r < order.size(); ++r) {
    const auto& em = plan->emu[order[r]];
    const bool pair = pair_class(em.p);
    if (plan->segments.empty() || plan->segments.back().slices != em.slices || plan->segments.back().pair != pair) {
      plan->segments.push_back({(int)r, 0, em.slices, pair, 0});
      seg_tiles = 0;
    }
    emu::EmuTableEntry& t = plan->emu_table[r];
    memset(&t, 0, sizeof(t));
    if ((rc = emu::encode_slice_maps(em.ws, em.p.m, em.p.n, em.p.k, em.slices, &t))) return rc;
    t.m = em.p.m; t.n = em.p.n; t.k = em.p.k; t.ldc = em.p.ldc;
    t.alpha = em.p.alpha; t.beta = em.p.beta; t.C = em.p.C;
    t.sigA = em.ws.sigA; t.sigB = em.ws.sigB; t.badA = em.ws.badA; t.badB = em.ws.badB;
    t.slices = em.slices;
    t.nkb = (int)((em.p.k + emu::kBK - 1) / emu::kBK);
    const int bm = pair ? 256 : 128, bn = pair ? 256 : emu::kGroupedBN;
    t.tiles_m = (int)((em.p.m + bm - 1) / bm);
    t.num_tiles = t.tiles_m * (int)((em.p.n + bn - 1) / bn);
    t.group_m = t.tiles_m;  // within one problem the tiles walk down the rows
    t.tile_begin = seg_tiles;  // counted from the first tile of its launch
    seg_tiles += t.num_tiles;
    tiles += t.num_tiles;
    plan->segments.back().count += 1;
    plan->segments.back().tiles = seg_tiles;
  }
  plan->emu_tiles = tiles;
  if (slices_used) {
    for (int i = 0; i < count; ++i) {
      const gbd_problem& p = probs[i];
      const bool quick = p.m == 0 || p.n == 0 || p.alpha == 0.0 || p.k == 0;
      if (p.mode == GBD_MODE_EMULATED && !quick) slices_used[i] = -1;  // unless it stayed emulated
    }
    for (const auto& em : plan->emu) slices_used[em.index] = em.slices;
  }
  // native table: longest tiles (largest k) first
  std::stable_sort(plan->native.begin(), plan->native.end(),
                   [](const NativeTableEntry& a, const NativeTableEntry& b) { return a.a.k > b.a.k; });
  int64_t nt = 0;
  size_t ks_at = 0, ks_tile = 0;  // running offsets into the part slots and the counters
  for (auto& t : plan->native) {
    t.tile_begin = nt;
    const int64_t tiles = (int64_t)t.tiles_m * ((t.a.n + t.tile - 1) / t.tile);
    if (t.ksplit > 1) {
      t.part = plan->ksplit_parts + ks_at;
      t.done = plan->ksplit_done + ks_tile;
      ks_at += (size_t)tiles * t.ksplit * t.tile * t.tile;
      ks_tile += (size_t)tiles;
    }
    nt += tiles * (t.ksplit > 1 ? t.ksplit : 1);
  }
  plan->native_tiles = nt;
  if (plan->ksplit_done_count &&
      (e = cudaMemsetAsync(plan->ksplit_done, 0, sizeof(unsigned int) * plan->ksplit_done_count, s)) != cudaSuccess)
    return cuda_fail(e, "grouped: clearing the split-k counters");
  std::stable_sort(plan->fallback.begin(), plan->fallback.end(),
                   [](const NativeTableEntry& a, const NativeTableEntry& b) { return a.a.k > b.a.k; });
  int64_t ft = 0;
  for (auto& t : plan->fallback) {
    t.tile_begin = ft;
    ft += (int64_t)t.tiles_m * ((t.a.n + t.tile - 1) / t.tile);
  }
  plan->fallback_tiles = ft;
  // tables to the device, through page-locked staging owned by the plan: the copies are stream-ordered
  // and need no synchronisation
  struct Part {
    void* dst;
    const void* src;
    size_t bytes;
  };
  const Part parts[] = {
      {plan->native_dev, plan->native.data(), sizeof(NativeTableEntry) * plan->native.size()},
      {plan->native_dev + plan->native.size(), plan->fallback.data(),
       sizeof(NativeTableEntry) * plan->fallback.size()},
      {plan->emu_dev, plan->emu_table.data(), sizeof(emu::EmuTableEntry) * plan->emu_table.size()},
      {plan->jobs_dev, plan->jobs.data(), sizeof(emu::PrepJob) * plan->jobs.size()},
      {plan->mod.jobs_dev, plan->mod.jobs.data(), sizeof(emu::PrepJob) * plan->mod.jobs.size()},
      {plan->mod.cert_dev, plan->mod.cert.data(), sizeof(emu::CertTableEntry) * plan->mod.cert.size()},
      {plan->mod.planjobs_dev, plan->mod.planjobs.data(), sizeof(emu::ModPlanJob) * plan->mod.planjobs.size()},
      {plan->mod.coljobs_dev, plan->mod.coljobs.data(), sizeof(emu::ColJob) * plan->mod.coljobs.size()},
      {plan->mod.table_dev, plan->mod.table.data(), sizeof(emu::ModTableEntry) * plan->mod.table.size()},
      {plan->mod.crt_dev, plan->mod.crt.data(), sizeof(emu::CrtJob) * plan->mod.crt.size()},
  };
  size_t staged = 0;
  for (const Part& q : parts) staged += up256(q.bytes);
  if (staged > 0) {
    int handle = -1;
    void* pinned = nullptr;
    if ((rc = staging_get(staged, &handle, &pinned))) return rc;
    size_t at = 0;
    for (const Part& q : parts) {
      if (q.bytes == 0) continue;
      char* h = static_cast<char*>(pinned) + at;
      memcpy(h, q.src, q.bytes);
      if ((e = cudaMemcpyAsync(q.dst, h, q.bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        staging_put(handle, s);
        return cuda_fail(e, "grouped: table copy");
      }
      at += up256(q.bytes);
    }
    if ((rc = staging_put(handle, s))) return rc;
  }
  *out = plan;
  return GBD_OK;
}

int gbd_grouped_plan_run(gbd_plan* plan, void* stream) {
  using namespace gbd;
  if (!plan) return set_error(GBD_ERR_ARG, "grouped: plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int sms = 0;
  int rc = current_device(nullptr, &sms);
  if (rc) return rc;
  cudaError_t e;
  // emulated: exponents and digit slices of every problem (three launches), then one slice-product
  // launch per slice count
  if (!plan->jobs.empty() &&
      (rc = emu::launch_prep_batched(plan->jobs_dev, plan->jobs.data(), (int)plan->jobs.size(), plan->exp_blocks,
                                     plan->split_blocks,
                                     true, true, s)))
    return rc;
  for (const auto& sg : plan->segments) {
    if (sg.tiles <= 0) continue;
    rc = sg.pair ? emu::launch_slice_gemm_grouped_pair(plan->emu_dev + sg.first, sg.count, (int)sg.tiles, sg.slices,
                                                       plan->pair_scratch, plan->pair_scratch_p, plan->pair_ctas, s)
                 : emu::launch_slice_gemm_grouped(plan->emu_dev + sg.first, sg.count, (int)sg.tiles, sg.slices, s);
    if (rc) return rc;
  }
  // modular: preparation, certification and plans on the device, then one persistent product launch
  if ((rc = emu::mod_grouped_run(plan->mod, sms, s))) return rc;
  // native: one persistent launch over all tiles; then the fallbacks of the modular problems whose
  // plans found no certified bit count (a launch that returns at once when there is none)
  if (plan->native_tiles > 0 || plan->fallback_tiles > 0) {
    if ((e = cudaMemsetAsync(plan->counter_dev, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "grouped: counter reset");
    constexpr size_t smem = native_smem_bytes<64, 64>();
    e = cudaFuncSetAttribute(k_grouped_native, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(grouped native)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grouped_native, kNativeThreads, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    const int64_t full = (int64_t)sms * per_sm;
    if (plan->native_tiles > 0) {
      const int64_t grid = full < plan->native_tiles ? full : plan->native_tiles;
      k_grouped_native<<<(unsigned)grid, kNativeThreads, smem, s>>>(plan->native_dev, (int)plan->native.size(),
                                                                   plan->native_tiles, plan->counter_dev, nullptr);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped native launch");
    }
    if (plan->fallback_tiles > 0) {
      const int64_t grid = full < plan->fallback_tiles ? full : plan->fallback_tiles;
      k_grouped_native<<<(unsigned)grid, kNativeThreads, smem, s>>>(
          plan->native_dev + plan->native.size(), (int)plan->fallback.size(), plan->fallback_tiles,
          plan->counter_dev + 1, plan->mod.flags_dev + 1);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "grouped fallback launch");
    }
  }
  return GBD_OK;
}

void gbd_grouped_plan_destroy(gbd_plan* plan) { delete plan; }

int gbd_dgemm_grouped(const gbd_problem* probs, int count, void* workspace, size_t workspace_bytes,
                      int* slices_used, void* stream) {
  gbd_plan* plan = nullptr;
  int rc = gbd_grouped_plan_create(probs, count, workspace, workspace_bytes, slices_used, stream, &plan);
  if (rc) return rc;
  rc = gbd_grouped_plan_run(plan, stream);
  gbd_grouped_plan_destroy(plan);
  return rc;
}

}  // extern "C"
