// C ABI of libaxpic (declared in include/axpic.h): context life cycle,
// argument validation, constant folding and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "misc.h"
#include "sr.h"
#include "step.h"
#include "merge.h"
#include "stream.h"

using namespace axpic;

namespace {

// An NVTX range over each public call, named for it (a no-op unless a
// profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
#define AXPIC_RANGE(name) NvtxRange axpic_range_(name)

// CODATA 2018 constants (binary64), folded into the binary32 record.
constexpr double kHbarcKeVcm = 1.973269804e-8;
constexpr double kHbarcGeVcm = 1.973269804e-14;
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kMu = 1.66053906660e-24;
constexpr double kC = 2.99792458e10;
constexpr double kKb = 8.617333262e-8;
constexpr double kKeVerg = 1.602176634e-9;
constexpr double kPi = 3.14159265358979323846;
constexpr int kDefaultWarps = 4;
// A replayed graph runs its cells as several independent branches (forked
// streams inside the graph), so that one branch's decisions overlap another
// branch's events and feedback. Each branch chains kGraphSteps steps with
// its own device step counter and the branches join only at the graph's end,
// so they drift apart within it. Default: 8 branches up to kBranchCells
// cells (c2, 65,536 cells, graphs of 32 steps: 0.1875 ms per step against
// 0.236 with one branch; 16 branches 0.1925), one above (1.57 M cells fill
// the GPU alone: branching measured 1 % slower).
#ifndef AXPIC_GRAPH_STEPS
#define AXPIC_GRAPH_STEPS 32
#endif
#ifndef AXPIC_MAX_BRANCHES
#define AXPIC_MAX_BRANCHES 8
#endif
constexpr int kMaxBranches = AXPIC_MAX_BRANCHES;
constexpr int kDefaultBranches = AXPIC_MAX_BRANCHES;
constexpr int kBranchCells = 1 << 20;
constexpr int kGraphSteps = AXPIC_GRAPH_STEPS;
constexpr int kInfoChunk = 4096;

}  // namespace

struct axpic_ctx {
  axpic_plasma_desc desc;
  axpic_params prm;
  std::vector<double> Z, A;
  cudaStream_t stream = nullptr;
  float* rec = nullptr;
  float* mom = nullptr;
  double* xbuf = nullptr;
  double* res = nullptr;
  double* diag = nullptr;
  int32_t* photon_start = nullptr;
  float* tables = nullptr;
  double* tally = nullptr;
  unsigned long long* counters = nullptr;
  int* err = nullptr;
  double* scratch = nullptr;  // totals (8) + counters (kNumCounters) + info chunk
  uint32_t* bits = nullptr;   // decision bit masks: axions, photons, electrons
  uint4* recA = nullptr;      // full decisions of flagged axion / photon slots
  uint4* recG = nullptr;
  uint32_t* recE = nullptr;   // event counts of flagged electrons
  CellConst cc;
  int warps = kDefaultWarps;
  int grid = 0;       // event-kernel CTAs
  int max_warps = 4;  // largest event CTA (warps) whose scratch fits
  int ctr_rows = 1;   // rows of per-CTA counters
  int dec_grid = 1;   // CTAs of the persistent decision kernel
  int dec_chunk = kDefaultDecChunk;
  uint32_t* step_dev = nullptr;      // step counter of replayed graphs
  int32_t* heavy = nullptr;          // cells left to the warp-path event kernel
  int32_t* heavy_n = nullptr;        // their count, per branch
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t graph_ev[2] = {nullptr, nullptr};
  int branches = 1;                  // independent cell ranges of a replayed step
  cudaStream_t br_stream[kMaxBranches] = {};
  cudaEvent_t br_ev[kMaxBranches + 1] = {};
  std::map<int, cudaGraphExec_t> graphs;  // per (channel mask, steps in the graph)
  std::map<int, cudaGraphExec_t> sgraphs;  // steps followed by axion streaming, for stream_sig
  std::vector<int64_t> stream_sig;         // the streaming parameters sgraphs were captured for
  // spectral records of rate models 1 and 2
  float* sr = nullptr;      // [ncells * kSrLen]
  float* srtab = nullptr;   // [2][nne][nkt][kSrTabOut]
  float* sur_P = nullptr;   // network parameters, output affine and trust map
  float* sur_mu = nullptr;
  float* sur_sigma = nullptr;
  float* sur_skip = nullptr;
  uint8_t* sur_trust = nullptr;
  uint8_t* sr_src = nullptr;       // [ncells] rate model 2: 1 = table record, 0 = network prefactors
  float* sur_uni = nullptr;        // [kSrLen] the network's cell-independent quantiles
  unsigned char* sur_img = nullptr;  // the network laid out for the fused kernels
  // axion streaming scratch, made by the first axpic_stream_axions call
  uint8_t* st_dir = nullptr;  // [ncells * axion capacity]
  int32_t* st_cnt = nullptr;  // [ncells * 27 * 2]: counts, then group offsets
  float* st_buf = nullptr;    // [ncells * axion capacity * 8]
  double* st_stats = nullptr; // [4]
  // axion merging scratch, made by the first axpic_merge_axions call
  uint8_t* mg_grp = nullptr;  // [ncells * axion capacity]
  double* mg_removed = nullptr;
  int sr_nkt = 0, sr_nne = 0, tnT = 0, tnne = 0, sur_set = 0, sur_any_trusted = 0;
  float ln_gP = 0.f, ln_gA = 0.f, lnK_CC = 0.f, lnK_CB = 0.f;
  int64_t last_absorb_step = -1;
  std::string last_error;
  std::vector<cudaEvent_t> prof_events;  // kStepKernels + 1 per recorded step, created by axpic_profile_begin
  int prof_max = 0, prof_used = 0;
};

static const char* kNoCtxMsg = "no context";

static axpic_status fail(axpic_ctx* c, axpic_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

static axpic_status cuda_fail(axpic_ctx* c, cudaError_t e, const char* where) {
  return fail(c, AXPIC_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

static SpeciesPtrs to_ptrs(const axpic_species& s) {
  SpeciesPtrs p;
  p.wp = reinterpret_cast<float4*>(s.wp);
  p.xyz = reinterpret_cast<float4*>(s.xyz);
  p.count = s.count;
  p.cap = s.capacity;
  return p;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static std::string check_species(const axpic_species& s, const char* name) {
  if (s.capacity < 0 || (s.capacity & 3)) return std::string(name) + ": capacity must be a non-negative multiple of 4";
  if (s.capacity > 65532) return std::string(name) + ": capacity above 65532";
  if (!s.count) return std::string(name) + ": count is NULL";
  if (s.capacity == 0) return "";
  const float* f[2] = {s.wp, s.xyz};
  for (auto p : f) {
    if (!p) return std::string(name) + ": a particle array is NULL";
    if (!aligned16(p)) return std::string(name) + ": particle arrays must be 16-byte aligned";
  }
  return "";
}

// The checks every entry point that takes a plasma description and options
// makes before launching anything: an empty string when they hold, else
// what failed.
// Words of the decision bit masks: per cell, a row per species (a bit per
// slot).
static size_t mask_words(const axpic_plasma_desc& d) {
  const size_t n = (size_t)std::max(d.ncells, 0);
  return n * ((d.axions.capacity + 31) / 32 + (d.photons.capacity + 31) / 32 + (d.electrons.capacity + 31) / 32);
}

static std::string check_plasma(const axpic_plasma_desc& d, const axpic_params& p) {
  if (d.ncells < 0) return "ncells < 0";
  if (d.nspecies < 1 || d.nspecies > kMaxSpecies) return "nspecies must be in 1..8";
  if (d.cell_index_base < 0 || d.cell_index_base + d.ncells > (int64_t)0xFFFFFFFF)
    return "global cell indices must fit in 32 bits";
  if (d.ncells > 0 && (!d.T_keV || !d.n_ion)) return "T_keV or n_ion is NULL";
  if (!d.Z || !d.A) return "Z or A is NULL";
  if (!(d.cell_volume_cm3 > 0)) return "cell_volume_cm3 must be > 0";
  for (auto sp : {std::make_pair(&d.electrons, "electrons"), std::make_pair(&d.photons, "photons"),
                  std::make_pair(&d.axions, "axions")}) {
    const std::string m = check_species(*sp.first, sp.second);
    if (!m.empty()) return m;
  }
  for (int s = 0; s < d.nspecies; ++s)
    if (!(d.Z[s] > 0) || !(d.A[s] > 0)) return "Z and A must be > 0";
  if (!(p.dt_phys_s > 0) || !(p.w_a > 0)) return "dt_phys_s and w_a must be > 0";
  if (!((float)p.w_a > 0) || !std::isfinite((float)p.w_a)) return "w_a must be representable in binary32";
  if (!(p.relax_r >= 0 && p.relax_r <= 1)) return "relax_r must be in [0, 1]";
  if (!(p.brems_gamma_shape > 0)) return "brems_gamma_shape must be > 0";
  if (p.kappa_mode != 0 && p.kappa_mode != 1) return "kappa_mode must be 0 or 1";
  if (p.kappa_mode == 1 && !(p.kappa_fixed_keV > 0)) return "kappa_fixed_keV must be > 0";
  if (p.eq_stats != 0 && p.eq_stats != 1) return "eq_stats must be 0 or 1";
  if (p.absorb_mode != 0 && p.absorb_mode != 1) return "absorb_mode must be 0 or 1";
  if (p.T_mode < 0 || p.T_mode > 2) return "T_mode must be 0, 1 or 2";
  if (!(p.T_floor_keV <= p.T_ceil_keV)) return "T_floor_keV > T_ceil_keV";
  if (p.tally_nbins < 1 || !(p.tally_Emax_keV > 0)) return "tally_nbins >= 1 and tally_Emax_keV > 0";
  if (!(p.prim_inverse_mult >= 0)) return "prim_inverse_mult must be >= 0";
  if (!(p.axion_mass_keV >= 0) || !std::isfinite(p.axion_mass_keV)) return "axion_mass_keV must be finite and >= 0";
  return "";
}

static double w_gref(const axpic_params& p) { return p.w_gamma_ref > 0 ? p.w_gamma_ref : p.w_a; }

static void fold_constants(axpic_ctx* ctx) {
  const axpic_params& p = ctx->prm;
  CellConst& cc = ctx->cc;
  std::memset(&cc, 0, sizeof(cc));
  cc.nspecies = ctx->desc.nspecies;
  for (int s = 0; s < cc.nspecies; ++s) {
    cc.Z[s] = (float)ctx->desc.Z[s];
    cc.A[s] = (float)ctx->desc.A[s];
    cc.is_h[s] = ctx->desc.Z[s] == 1.0;
  }
  cc.kappa_mode = p.kappa_mode;
  cc.kappa_fixed = (float)p.kappa_fixed_keV;
  cc.prim_targets = p.prim_targets;
  cc.prim_mult = (float)p.prim_inverse_mult;
  cc.brems_ee = p.brems_ee;
  const double z5 = zeta(5.0), z6 = zeta(6.0);
  const double mean_xc = 5.0 * z6 / z5;
  const double a = p.brems_gamma_shape;
  const double wa32 = (double)(float)p.w_a;
  const double hc3 = kHbarcKeVcm * kHbarcKeVcm * kHbarcKeVcm;
  const double gcm = p.g_agg_GeV_inv * kHbarcGeVcm;
  cc.k_kappa2 = (float)(4.0 * kPi * kAlpha * hc3 * 1e24);
  cc.k_rho = (float)(kMu * 1e24);
  cc.k_T7 = (float)(1.0 / (kKb * 1e7));
  cc.afac = (float)(p.g_ae * p.g_ae / (4.0 * kPi * 1.60e-23));
  cc.k_AP = (float)(kAlpha * gcm * gcm / 8.0 * kC * 1e24 * p.dt_phys_s);
  cc.k_CC = (float)(p.dt_phys_s / (wa32 * mean_xc * kKeVerg * 1e24));
  cc.k_CB = (float)(p.dt_phys_s / (wa32 * a * kKeVerg * 1e24));
  cc.k_BC = (float)(2.0 * kPi * kPi * hc3 * p.dt_phys_s / (24.0 * z5 * mean_xc * kKeVerg));
  cc.k_BB = (float)(2.0 * kPi * kPi * hc3 * p.dt_phys_s / (std::tgamma(a) * a * kKeVerg));
}


// The rate models' records and network, as the kernels see them.
static RecordArgs make_record_args(axpic_ctx* ctx) {
  RecordArgs a;
  std::memset(&a, 0, sizeof(a));
  if (!ctx->prm.rate_model) return a;
  a.sr = ctx->sr;
  a.tab = ctx->srtab;
  a.nkt = ctx->sr_nkt;
  a.nne = ctx->sr_nne;
  a.Z = ctx->desc.nspecies > 0 ? (float)ctx->desc.Z[0] : 1.f;
  a.ln_gP = ctx->ln_gP;
  a.ln_gA = ctx->ln_gA;
  a.lnK_CC = ctx->lnK_CC;
  a.lnK_CB = ctx->lnK_CB;
  // the e-e term's weight (1 + X_H) / (2 sqrt 2) of the single ion species
  a.bee_c = (float)((a.Z == 1.f ? 2.0 : 1.0) / (2.0 * std::sqrt(2.0)));
  a.k_T7 = ctx->cc.k_T7;
  // no trusted node: the network is never evaluated (every cell keeps the table)
  a.trust = ctx->sur_set && ctx->sur_any_trusted ? ctx->sur_trust : nullptr;
  a.tnT = ctx->tnT;
  a.tnne = ctx->tnne;
  a.img = ctx->sur_img;
  a.src = ctx->sr_src;
  a.uni = ctx->sur_uni;
  return a;
}

static StepArgs make_args(axpic_ctx* ctx, int64_t step, int mask) {
  const axpic_params& p = ctx->prm;
  StepArgs A;
  std::memset(&A, 0, sizeof(A));
  A.e = to_ptrs(ctx->desc.electrons);
  A.g = to_ptrs(ctx->desc.photons);
  A.a = to_ptrs(ctx->desc.axions);
  A.ncells = ctx->desc.ncells;
  A.cell0 = 0;
  A.cell_base = (uint32_t)ctx->desc.cell_index_base;
  A.step = (uint32_t)(step & 0xFFFFFFFF);
  A.key0 = (uint32_t)(p.seed & 0xFFFFFFFFu);
  A.key1 = (uint32_t)(p.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    A.rk.k0[r] = A.key0 + (uint32_t)r * 0x9E3779B9u;
    A.rk.k1[r] = A.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  A.mask = mask;
  A.w_a = (float)p.w_a;
  A.w_gref = (float)w_gref(p);
  A.inv_w_a = 1.0f / A.w_a;
  A.inv_w_gref = 1.0f / A.w_gref;
  A.lam_cap = p.lambda_cap > 0 ? (float)std::fmin(p.lambda_cap, (double)kLambdaHardCap) : kLambdaHardCap;
  A.brems_am3 = (float)(p.brems_gamma_shape - 3.0);
  A.eq_stats = p.eq_stats;
  A.absorb_mode = p.absorb_mode;
  A.T_mode = p.T_mode;
  A.tally_enable = p.tally_enable;
  A.diag_enable = p.diag_enable;
  A.relax_r = (float)p.relax_r;
  A.T_floor = p.T_floor_keV;
  A.T_ceil = p.T_ceil_keV;
  // widened so that the binary32 test never misses a clamp the FP64 one needs
  A.T_floor_f = (float)p.T_floor_keV * (1.0f + 1e-6f) + 1e-30f;
  A.T_ceil_f = p.T_ceil_keV > 3e38 ? 3e38f : (float)p.T_ceil_keV * (1.0f - 1e-6f);
  A.rec = ctx->rec;
  A.mom = ctx->mom;
  A.T = ctx->desc.T_keV;
  A.n_ion = ctx->desc.n_ion;
  A.xbuf = ctx->xbuf;
  A.res = ctx->res;
  A.diag = ctx->diag;
  A.photon_start = ctx->photon_start;
  A.tables = ctx->tables;
  A.tally = ctx->tally;
  A.nbins = p.tally_nbins;
  A.inv_dE_bin = (float)(p.tally_nbins / p.tally_Emax_keV);
  A.counters = ctx->counters;
  A.err = ctx->err;
  A.Wa = (ctx->desc.axions.capacity + 31) / 32;
  A.Wg = (ctx->desc.photons.capacity + 31) / 32;
  A.We = (ctx->desc.electrons.capacity + 31) / 32;
  A.bitsA = ctx->bits;
  A.bitsG = ctx->bits + (size_t)A.Wa * ctx->desc.ncells;
  A.bitsE = A.bitsG + (size_t)A.Wg * ctx->desc.ncells;
  A.recA = ctx->recA;
  A.recG = ctx->recG;
  A.recE = ctx->recE;
  A.dec_grid = ctx->dec_grid;
  A.dec_chunk = ctx->dec_chunk;
  A.ctr_rows = ctx->ctr_rows;
  A.step_dev = nullptr;
  A.heavy = ctx->heavy;
  A.heavy_n = ctx->heavy_n;
  A.rate_model = ctx->prm.rate_model;
  A.ra = make_record_args(ctx);
  A.mu = (float)(p.axion_mass_keV / kMeC2);
  A.mu2 = A.mu * A.mu;
  A.guard_margin = ctx->prm.rate_model ? 1.05f : 1.0f;
  A.cc = ctx->cc;
  return A;
}

static SrArgs make_sr_args(axpic_ctx* ctx) {
  SrArgs a;
  std::memset(&a, 0, sizeof(a));
  a.ncells = ctx->desc.ncells;
  a.cell0 = 0;
  a.rec = ctx->rec;
  a.ra = make_record_args(ctx);
  a.err = ctx->err;
  return a;
}

// Rebuilds every cell's rate-model record for its current T and composition
// (the cell records' closed-form slots must be current): the table model's
// spectral records; under the surrogate model the network's prefactors
// where it is trusted and the table's records elsewhere.
static cudaError_t build_records(axpic_ctx* ctx, cudaStream_t st) {
  if (!ctx->prm.rate_model) return cudaSuccess;
  return launch_sr_records(ctx->prm.rate_model, make_sr_args(ctx), st);
}

static void free_events(axpic_ctx* ctx) {
  for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
  ctx->prof_events.clear();
  ctx->prof_max = ctx->prof_used = 0;
}

static void free_graphs(axpic_ctx* ctx) {
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.second);
  ctx->graphs.clear();
  for (auto& g : ctx->sgraphs) cudaGraphExecDestroy(g.second);
  ctx->sgraphs.clear();
}

static void free_ctx(axpic_ctx* ctx) {
  free_events(ctx);
  free_graphs(ctx);
  for (cudaEvent_t e : ctx->graph_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->graph_stream) cudaStreamDestroy(ctx->graph_stream);
  for (cudaStream_t b : ctx->br_stream)
    if (b) cudaStreamDestroy(b);
  for (cudaEvent_t b : ctx->br_ev)
    if (b) cudaEventDestroy(b);
  void* bufs[] = {ctx->rec,    ctx->mom,   ctx->xbuf,     ctx->res, ctx->diag,    ctx->photon_start,
                  ctx->tables, ctx->tally, ctx->counters, ctx->err, ctx->scratch, ctx->bits,
                  ctx->recA,   ctx->recG,  ctx->recE,     ctx->step_dev, ctx->sr, ctx->srtab,
                  ctx->sur_P,  ctx->sur_mu, ctx->sur_sigma, ctx->sur_trust, ctx->sur_img, ctx->sur_skip,
                  ctx->sr_src, ctx->sur_uni, ctx->st_dir, ctx->st_cnt, ctx->st_buf, ctx->st_stats, ctx->mg_grp,
                  ctx->mg_removed, ctx->heavy, ctx->heavy_n};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete ctx;
}

extern "C" {

void axpic_default_params(axpic_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->g_agg_GeV_inv = 1e-10;
  p->g_ae = 1e-13;
  p->dt_phys_s = 1.0;
  p->w_a = 1.0;
  p->w_gamma_ref = 0.0;
  p->lambda_cap = 0.0;
  p->kappa_mode = 0;
  p->prim_targets = 0;
  p->prim_inverse_mult = 1.0;
  p->eq_stats = 0;
  p->brems_ee = 1;
  p->absorb_mode = 0;
  p->brems_gamma_shape = 1.70;
  p->relax_r = 0.1;
  p->T_floor_keV = 0.0;
  p->T_ceil_keV = 1e30;
  p->T_mode = 0;
  p->seed = 0;
  p->tally_nbins = 160;
  p->tally_Emax_keV = 80.0;
  p->tally_enable = 1;
  p->diag_enable = 0;
  p->threads_per_block = 0;
  p->decide_chunk = 0;
}

axpic_status axpic_init_plasma(axpic_ctx** out, const axpic_plasma_desc* desc, const axpic_params* params,
                               void* stream) {
  AXPIC_RANGE("axpic_init_plasma");
  if (!out || !desc || !params) return AXPIC_E_INVALID;
  *out = nullptr;
  const axpic_plasma_desc& d = *desc;
  const axpic_params& p = *params;
  auto* ctx = new axpic_ctx();
  ctx->desc = d;
  ctx->prm = p;
  ctx->stream = (cudaStream_t)stream;
  auto bad = [&](const std::string& m) {
    fprintf(stderr, "axpic_init_plasma: %s\n", m.c_str());
    delete ctx;
    return AXPIC_E_INVALID;
  };
  const std::string why = check_plasma(d, p);
  if (!why.empty()) return bad(why);
  for (int s = 0; s < d.nspecies; ++s) {
    ctx->Z.push_back(d.Z[s]);
    ctx->A.push_back(d.A[s]);
  }
  const size_t per_warp = step_smem_per_warp(d.axions.capacity, d.photons.capacity, d.electrons.capacity);
  int warps = p.threads_per_block > 0 ? p.threads_per_block / 32 : kDefaultWarps;
  if (warps < 1 || warps > 4 || (p.threads_per_block > 0 && p.threads_per_block % 32))
    return bad("threads_per_block must be 32..128, a multiple of 32");
  const size_t smem_limit = 227 * 1024 - 128;
  while (warps > 1 && per_warp * warps > smem_limit) --warps;
  if (per_warp > smem_limit) return bad("slab capacities too large for shared-memory scratch");
  ctx->max_warps = 4;
  while (ctx->max_warps > 1 && per_warp * ctx->max_warps > smem_limit) --ctx->max_warps;
  if (p.decide_chunk != 0 && p.decide_chunk != 4 && p.decide_chunk != 8 && p.decide_chunk != 16 &&
      p.decide_chunk != 32)
    return bad("decide_chunk must be 0, 4, 8, 16 or 32");
  if (p.step_branches < 0 || p.step_branches > kMaxBranches || (p.step_branches & (p.step_branches - 1)))
    return bad("step_branches must be 0 or a power of two up to 8");
  if (p.rate_model < 0 || p.rate_model > 2) return bad("rate_model must be 0, 1 or 2");
  if (p.rate_model) {
    if (d.nspecies != 1 || (d.Z[0] != 1.0 && d.Z[0] != 2.0) || p.kappa_mode != 0 || p.prim_targets != 0)
      return bad("rate models 1 and 2 need one ion species with Z 1 or 2, Debye screening and ion targets");
    ctx->sr_nkt = p.sr_table_nkt > 0 ? p.sr_table_nkt : 128;
    ctx->sr_nne = p.sr_table_nne > 0 ? p.sr_table_nne : 64;
    if (ctx->sr_nkt < 2 || ctx->sr_nne < 2 || ctx->sr_nkt > 4096 || ctx->sr_nne > 4096)
      return bad("sr_table_nkt and sr_table_nne must be in [2, 4096]");
    const double hc3 = kHbarcKeVcm * kHbarcKeVcm * kHbarcKeVcm;
    const double gcm = p.g_agg_GeV_inv;  // the records are at g_agg = 1 GeV^-1
    ctx->ln_gP = (float)std::log(gcm * gcm * p.dt_phys_s * kPi * kPi * hc3 / kKeVerg);
    ctx->ln_gA = (float)std::log(p.g_ae * p.g_ae * p.dt_phys_s * 2.0 * kPi * kPi * hc3 / kKeVerg);
    // the network's emission rates per unit electron weight: lambda / w_e =
    // Q dt / (n_e <E> w_a) with Q_C = g_ae^2 e^c_C Gamma(6) zeta(6), <E>_C =
    // 5 zeta(6) / zeta(5) T, Q_B = g_ae^2 e^c_B Gamma(a + 1), <E>_B = a T (the
    // cell divides by n_e / 1e24 and T)
    const double wa32 = (double)(float)p.w_a, a = p.brems_gamma_shape, z6 = zeta(6.0), z5 = zeta(5.0);
    const double gae2 = p.g_ae * p.g_ae;
    ctx->lnK_CC = (float)std::log(gae2 * 120.0 * z6 * p.dt_phys_s / (wa32 * (5.0 * z6 / z5) * kKeVerg * 1e24));
    ctx->lnK_CB = (float)std::log(gae2 * std::tgamma(a + 1.0) * p.dt_phys_s / (wa32 * a * kKeVerg * 1e24));
  }
  ctx->dec_chunk = p.decide_chunk ? p.decide_chunk : kDefaultDecChunk;
  ctx->branches = p.step_branches                    ? p.step_branches
                  : d.ncells <= kBranchCells         ? kDefaultBranches
                                                     : 1;
  ctx->warps = warps;
  ctx->grid = (d.ncells + warps - 1) / warps;
  ctx->ctr_rows = std::max(1, std::min(kCounterRows, (d.ncells + 3) / 4));
  fold_constants(ctx);

  const int n = d.ncells;
  cudaError_t e;
#define ALLOC(ptr, bytes)                                                 \
  if ((e = cudaMalloc((void**)&ptr, (bytes) > 0 ? (bytes) : 16)) != cudaSuccess) { \
    ctx->last_error = cudaGetErrorString(e);                              \
    free_ctx(ctx);                                                        \
    return AXPIC_E_CUDA;                                                  \
  }
  ALLOC(ctx->rec, sizeof(float) * kRecLen * (size_t)n);
  ALLOC(ctx->mom, sizeof(float) * kMomLen * (size_t)n);
  ALLOC(ctx->xbuf, sizeof(double) * 4 * (size_t)n);
  ALLOC(ctx->res, sizeof(double) * 4 * (size_t)n);
  ALLOC(ctx->diag, sizeof(double) * AXPIC_CELL_DIAG_LEN * (size_t)n);
  ALLOC(ctx->photon_start, sizeof(int32_t) * (size_t)n);
  ALLOC(ctx->tables, sizeof(float) * kNumTables * kTableN);
  ALLOC(ctx->tally, sizeof(double) * (3 * (size_t)p.tally_nbins + 6));
  ALLOC(ctx->counters, sizeof(unsigned long long) * kNumCounters * (size_t)ctx->ctr_rows);
  ALLOC(ctx->step_dev, sizeof(uint32_t) * kMaxBranches);
  ALLOC(ctx->heavy, sizeof(int32_t) * (size_t)n);
  ALLOC(ctx->heavy_n, sizeof(int32_t) * kMaxBranches);
  if (p.rate_model) {
    ALLOC(ctx->sr, sizeof(float) * kSrLen * (size_t)n);
    ALLOC(ctx->srtab, sizeof(float) * kSrTabOut * 2 * (size_t)ctx->sr_nkt * ctx->sr_nne);
  }
  if (p.rate_model == 2) {
    ALLOC(ctx->sr_src, (size_t)n);
    ALLOC(ctx->sur_P, sizeof(float) * AXPIC_MLP_PARAMS);
    ALLOC(ctx->sur_mu, sizeof(float) * 96);
    ALLOC(ctx->sur_sigma, sizeof(float) * 96);
    ALLOC(ctx->sur_skip, sizeof(float) * 96 * 4);
    ALLOC(ctx->sur_uni, sizeof(float) * kSrLen);
    ALLOC(ctx->sur_img, kNetImgBytes);
  }
  ALLOC(ctx->err, sizeof(int));
  ALLOC(ctx->scratch, sizeof(double) * (8 + kNumCounters + (size_t)kInfoChunk * AXPIC_CELL_INFO_LEN));
  const size_t bit_words = mask_words(d);
  ALLOC(ctx->bits, sizeof(uint32_t) * bit_words);
  ALLOC(ctx->recA, sizeof(uint4) * (size_t)n * d.axions.capacity);
  ALLOC(ctx->recG, sizeof(uint4) * (size_t)n * d.photons.capacity);
  ALLOC(ctx->recE, sizeof(uint32_t) * (size_t)n * d.electrons.capacity);
#undef ALLOC
  std::vector<float> tab((size_t)kNumTables * kTableN);
  build_tables(p.brems_gamma_shape, tab.data());
  std::vector<float> srtab;
  if (p.rate_model) {
    srtab.resize((size_t)kSrTabOut * 2 * ctx->sr_nkt * ctx->sr_nne);
    build_sr_table(ctx->sr_nkt, ctx->sr_nne, p.brems_gamma_shape, srtab.data());
  }
  cudaStream_t st = ctx->stream;
  if ((e = cudaMemcpyAsync(ctx->tables, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemsetAsync(ctx->xbuf, 0, sizeof(double) * 4 * (size_t)n, st)) ||
      (e = cudaMemsetAsync(ctx->res, 0, sizeof(double) * 4 * (size_t)n, st)) ||
      (e = cudaMemsetAsync(ctx->diag, 0, sizeof(double) * AXPIC_CELL_DIAG_LEN * (size_t)n, st)) ||
      (e = cudaMemsetAsync(ctx->photon_start, 0, sizeof(int32_t) * (size_t)n, st)) ||
      (e = cudaMemsetAsync(ctx->tally, 0, sizeof(double) * (3 * (size_t)p.tally_nbins + 6), st)) ||
      (e = cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * kNumCounters * (size_t)ctx->ctr_rows, st)) ||
      (e = cudaMemsetAsync(ctx->err, 0, sizeof(int), st)) ||
      (e = cudaMemsetAsync(ctx->bits, 0, sizeof(uint32_t) * (bit_words > 0 ? bit_words : 1), st)) ||
      (e = set_step_smem_limits(per_warp * ctx->max_warps)) ||
      (e = decide_shape(p.decide_chunk, n, &ctx->dec_chunk, &ctx->dec_grid)) ||
      (e = launch_records(n, d.nspecies, ctx->cc, d.T_keV, d.n_ion, ctx->rec, ctx->err, st)) ||
      (e = launch_moments(n, to_ptrs(d.electrons), ctx->mom, st)) ||
      (p.rate_model && (e = cudaMemcpyAsync(ctx->srtab, srtab.data(), srtab.size() * sizeof(float),
                                            cudaMemcpyHostToDevice, st))) ||
      (p.rate_model && (e = sr_init_kernels())) || (e = build_records(ctx, st)) || (e = cudaStreamSynchronize(st))) {
    ctx->last_error = cudaGetErrorString(e);
    fprintf(stderr, "axpic_init_plasma: %s\n", ctx->last_error.c_str());
    free_ctx(ctx);
    return AXPIC_E_CUDA;
  }
  *out = ctx;
  return AXPIC_OK;
}

axpic_status axpic_sample_plasma(axpic_ctx* ctx, int32_t n_el, int32_t n_ph, int32_t n_ax) {
  AXPIC_RANGE("axpic_sample_plasma");
  if (!ctx) return AXPIC_E_INVALID;
  const axpic_plasma_desc& d = ctx->desc;
  if (n_el < 0 || n_ph < 0 || n_ax < 0 || n_el > d.electrons.capacity || n_ph > d.photons.capacity ||
      n_ax > d.axions.capacity)
    return fail(ctx, AXPIC_E_INVALID, "axpic_sample_plasma: count outside [0, capacity]");
  SampleArgs S;
  std::memset(&S, 0, sizeof(S));
  S.e = to_ptrs(d.electrons);
  S.g = to_ptrs(d.photons);
  S.a = to_ptrs(d.axions);
  S.ncells = d.ncells;
  S.n_el = n_el;
  S.n_ph = n_ph;
  S.n_ax = n_ax;
  S.cell_base = (uint32_t)d.cell_index_base;
  S.key0 = (uint32_t)(ctx->prm.seed & 0xFFFFFFFFu);
  S.key1 = (uint32_t)(ctx->prm.seed >> 32);
  S.k_we = n_el > 0 ? (float)(d.cell_volume_cm3 * 1e24 / n_el) : 0.f;
  const double hc3 = kHbarcKeVcm * kHbarcKeVcm * kHbarcKeVcm;
  S.k_wg = n_ph > 0 ? (float)(2.0 * zeta(3.0) / (kPi * kPi * hc3) * d.cell_volume_cm3 / n_ph) : 0.f;
  S.w_a = (float)ctx->prm.w_a;
  S.rec = ctx->rec;
  S.tables = ctx->tables;
  CK(launch_sample(S, ctx->stream), "sample");
  CK(launch_moments(d.ncells, to_ptrs(d.electrons), ctx->mom, ctx->stream), "moments");
  CK(build_records(ctx, ctx->stream), "spectral records");
  return AXPIC_OK;
}

axpic_status axpic_update_cells(axpic_ctx* ctx) {
  AXPIC_RANGE("axpic_update_cells");
  if (!ctx) return AXPIC_E_INVALID;
  const axpic_plasma_desc& d = ctx->desc;
  CK(launch_records(d.ncells, d.nspecies, ctx->cc, d.T_keV, d.n_ion, ctx->rec, ctx->err, ctx->stream), "records");
  CK(launch_moments(d.ncells, to_ptrs(d.electrons), ctx->mom, ctx->stream), "moments");
  CK(build_records(ctx, ctx->stream), "spectral records");
  return AXPIC_OK;
}

axpic_status axpic_deposit_composition(axpic_ctx* ctx, int32_t bind_species, const double* mass_frac,
                                       double* n_ion_out) {
  AXPIC_RANGE("axpic_deposit_composition");
  if (!ctx) return AXPIC_E_INVALID;
  const axpic_plasma_desc& d = ctx->desc;
  const int ns = d.nspecies;
  if (!n_ion_out && d.ncells > 0) return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: n_ion_out");
  DepositCoef k;
  std::memset(&k, 0, sizeof(k));
  if (bind_species >= 0) {
    if (bind_species >= ns || !(d.Z[bind_species] > 0.0))
      return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: bound species out of range or Z <= 0");
    k.coef[bind_species] = 1.0 / d.Z[bind_species] / d.cell_volume_cm3;
  } else if (bind_species == -1) {
    if (!mass_frac) return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: mass fractions missing");
    double sum = 0.0, zxa = 0.0;
    for (int i = 0; i < ns; ++i) {
      if (!std::isfinite(mass_frac[i]) || mass_frac[i] < 0.0)
        return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: mass fractions must be finite and >= 0");
      sum += mass_frac[i];
      zxa += d.Z[i] * mass_frac[i] / d.A[i];
    }
    if (std::fabs(sum - 1.0) > 1e-9 || !(zxa > 0.0))
      return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: mass fractions must sum to 1 and carry charge");
    // n_i = X_i (rho / m_u) / A_i with rho / m_u = n_e / sum_i Z_i X_i / A_i
    for (int i = 0; i < ns; ++i) k.coef[i] = mass_frac[i] / d.A[i] / zxa / d.cell_volume_cm3;
  } else {
    return fail(ctx, AXPIC_E_INVALID, "axpic_deposit_composition: bind_species must be -1 or a species");
  }
  CK(launch_deposit(d.ncells, ns, to_ptrs(d.electrons), k, n_ion_out, ctx->stream), "deposit");
  if (n_ion_out == d.n_ion) {
    CK(launch_records(d.ncells, ns, ctx->cc, d.T_keV, d.n_ion, ctx->rec, ctx->err, ctx->stream), "records");
    CK(build_records(ctx, ctx->stream), "spectral records");
  }
  return AXPIC_OK;
}

static axpic_status run_phases(axpic_ctx* ctx, int phases, int64_t step, int32_t mask, const char* name) {
  if (!ctx) return AXPIC_E_INVALID;
  if (step < 0 || step >= (int64_t)0xFFFFFFFF) return fail(ctx, AXPIC_E_INVALID, std::string(name) + ": step out of range");
  if (mask & ~AXPIC_CH_ALL) return fail(ctx, AXPIC_E_INVALID, std::string(name) + ": unknown channel bits");
  StepArgs A = make_args(ctx, step, mask);
  if (phases == PH_EMIT) A.use_snapshot = ctx->last_absorb_step == step;
  cudaEvent_t* ev = nullptr;
  if (phases == PH_ALL && ctx->prof_used < ctx->prof_max)
    ev = ctx->prof_events.data() + (kStepKernels + 1) * (ctx->prof_used++);
  const SrArgs sra = make_sr_args(ctx);
  CK(launch_step(phases, A, ctx->warps, ctx->stream, ev, ctx->prm.rate_model ? &sra : nullptr), name);
  if (phases == PH_ABSORB) ctx->last_absorb_step = step;
  return AXPIC_OK;
}

axpic_status axpic_absorb(axpic_ctx* ctx, int64_t step, int32_t channel_mask) {
  AXPIC_RANGE("axpic_absorb");
  return run_phases(ctx, PH_ABSORB, step, channel_mask, "axpic_absorb");
}

axpic_status axpic_emit(axpic_ctx* ctx, int64_t step, int32_t channel_mask) {
  AXPIC_RANGE("axpic_emit");
  return run_phases(ctx, PH_EMIT, step, channel_mask, "axpic_emit");
}

axpic_status axpic_feedback(axpic_ctx* ctx, int64_t step) {
  AXPIC_RANGE("axpic_feedback");
  return run_phases(ctx, PH_FEEDBACK, step, 0, "axpic_feedback");
}

axpic_status axpic_step(axpic_ctx* ctx, int64_t step, int32_t channel_mask) {
  AXPIC_RANGE("axpic_step");
  return run_phases(ctx, PH_ALL, step, channel_mask, "axpic_step");
}

axpic_status axpic_step_cells(axpic_ctx* ctx, int64_t step, int32_t channel_mask, int32_t first_cell,
                              int32_t ncells) {
  AXPIC_RANGE("axpic_step_cells");
  if (!ctx) return AXPIC_E_INVALID;
  if (step < 0 || step >= (int64_t)0xFFFFFFFF) return fail(ctx, AXPIC_E_INVALID, "axpic_step_cells: step out of range");
  if (channel_mask & ~AXPIC_CH_ALL) return fail(ctx, AXPIC_E_INVALID, "axpic_step_cells: unknown channel bits");
  if (first_cell < 0 || ncells < 0 || first_cell > ctx->desc.ncells - ncells)
    return fail(ctx, AXPIC_E_INVALID, "axpic_step_cells: cell range outside the context");
  if (ncells == 0) return AXPIC_OK;
  StepArgs A = make_args(ctx, step, channel_mask);
  A.cell0 = first_cell;
  A.ncells = ncells;
  SrArgs sra = make_sr_args(ctx);
  sra.cell0 = first_cell;
  sra.ncells = ncells;
  CK(launch_step(PH_ALL, A, ctx->warps, ctx->stream, nullptr, ctx->prm.rate_model ? &sra : nullptr),
     "axpic_step_cells");
  return AXPIC_OK;
}

static axpic_status read_err(axpic_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read error flag");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (h & ERR_CAPACITY) return fail(ctx, AXPIC_E_CAPACITY, "a slab capacity was exceeded; products were dropped");
  if (h & ERR_NUMERIC) return fail(ctx, AXPIC_E_NUMERIC, "a non-finite or non-positive temperature was found");
  if (h & ERR_TIMEOUT)
    return fail(ctx, AXPIC_E_TIMEOUT, "a tensor-core wait of the surrogate network ran out (its cells kept the table)");
  return AXPIC_OK;
}

axpic_status axpic_tally_spectrum(axpic_ctx* ctx, int32_t nbins, double* H_out, double* totals_out) {
  AXPIC_RANGE("axpic_tally_spectrum");
  if (!ctx) return AXPIC_E_INVALID;
  if (nbins != ctx->prm.tally_nbins) return fail(ctx, AXPIC_E_INVALID, "axpic_tally_spectrum: nbins mismatch");
  const axpic_plasma_desc& d = ctx->desc;
  cudaStream_t st = ctx->stream;
  const size_t hn = 3 * (size_t)nbins + 6;
  std::vector<double> h(hn), tot(8 + kNumCounters);
  CK(cudaMemsetAsync(ctx->scratch, 0, sizeof(double) * (8 + kNumCounters), st), "memset");
  CK(launch_totals(d.ncells, to_ptrs(d.electrons), to_ptrs(d.photons), to_ptrs(d.axions), ctx->res, ctx->counters,
                   ctx->ctr_rows, ctx->scratch, ctx->scratch + 8, st),
     "totals");
  CK(cudaMemcpyAsync(h.data(), ctx->tally, hn * sizeof(double), cudaMemcpyDeviceToHost, st), "copy tally");
  CK(cudaMemcpyAsync(tot.data(), ctx->scratch, tot.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
     "copy totals");
  CK(cudaMemsetAsync(ctx->tally, 0, hn * sizeof(double), st), "reset tally");
  CK(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * kNumCounters * (size_t)ctx->ctr_rows, st),
     "reset counters");
  CK(cudaStreamSynchronize(st), "synchronize");
  if (H_out) std::memcpy(H_out, h.data(), 3 * (size_t)nbins * sizeof(double));
  if (totals_out) {
    double* T = totals_out;
    std::memset(T, 0, sizeof(double) * AXPIC_TOTALS_LEN);
    const double* em = h.data() + 3 * (size_t)nbins;
    for (int c = 0; c < 3; ++c) {
      T[AXPIC_T_NEMIT_P + c] = em[c];
      T[AXPIC_T_UEMIT_P + c] = em[3 + c];
    }
    const double* cn = tot.data() + 8;
    T[AXPIC_T_EVENTS_P] = cn[C_EV_P];
    T[AXPIC_T_EVENTS_C] = cn[C_EV_C];
    T[AXPIC_T_EVENTS_B] = cn[C_EV_B];
    T[AXPIC_T_EVENTS_PINV] = cn[C_EV_PINV];
    T[AXPIC_T_ABSORBED_C] = cn[C_ABS_C];
    T[AXPIC_T_ABSORBED_B] = cn[C_ABS_B];
    T[AXPIC_T_CAP_HITS] = cn[C_CAP];
    T[AXPIC_T_CLAMP_HITS] = cn[C_CLAMP];
    T[AXPIC_T_DROPPED] = cn[C_DROP];
    T[AXPIC_T_N_AXIONS] = tot[0];
    T[AXPIC_T_U_AXIONS] = tot[1] * kMeC2;
    T[AXPIC_T_N_PHOTONS] = tot[2];
    T[AXPIC_T_U_PHOTONS] = tot[3] * kMeC2;
    T[AXPIC_T_U_ELECTRONS] = tot[4] * kMeC2;
    T[AXPIC_T_MACRO_AXIONS] = tot[5];
    T[AXPIC_T_MACRO_PHOTONS] = tot[6];
    T[AXPIC_T_RESIDUAL_E] = tot[7];
    T[AXPIC_T_REMAPS] = cn[C_REMAP];
    T[AXPIC_T_PART_E] = cn[C_NE];
    T[AXPIC_T_PART_G] = cn[C_NG];
    T[AXPIC_T_PART_A] = cn[C_NA];
    T[AXPIC_T_REMAP_E] = cn[C_REMAP_E];
    T[AXPIC_T_CALLS] = cn[C_CELLS];
  }
  return read_err(ctx);
}

axpic_status axpic_eval_rates(axpic_ctx* ctx, int32_t cell, const float* E_keV, int32_t n, float* out) {
  if (!ctx) return AXPIC_E_INVALID;
  if (cell < 0 || cell >= ctx->desc.ncells || n < 0 || (n > 0 && (!E_keV || !out)))
    return fail(ctx, AXPIC_E_INVALID, "axpic_eval_rates: bad cell, count or pointer");
  const float mu = (float)(ctx->prm.axion_mass_keV / kMeC2);
  CK(launch_rates(ctx->rec, cell, E_keV, n, ctx->prm.eq_stats, (float)(ctx->prm.brems_gamma_shape - 3.0),
                  ctx->cc.prim_mult, mu * mu, out, ctx->stream),
     "rates");
  return AXPIC_OK;
}

axpic_status axpic_get_cell_info(axpic_ctx* ctx, int32_t first, int32_t count, double* host_out) {
  if (!ctx) return AXPIC_E_INVALID;
  if (first < 0 || count < 0 || first + count > ctx->desc.ncells || (count > 0 && !host_out))
    return fail(ctx, AXPIC_E_INVALID, "axpic_get_cell_info: range outside the cells");
  double* dev = ctx->scratch + 8 + kNumCounters;
  const double k_gamma = (double)(float)ctx->prm.w_a / ctx->prm.dt_phys_s;
  for (int c0 = 0; c0 < count; c0 += kInfoChunk) {
    const int m = std::min(kInfoChunk, count - c0);
    CK(launch_info(first + c0, m, ctx->cc, k_gamma, ctx->rec, dev, ctx->stream), "info");
    CK(cudaMemcpyAsync(host_out + (size_t)c0 * AXPIC_CELL_INFO_LEN, dev, sizeof(double) * m * AXPIC_CELL_INFO_LEN,
                       cudaMemcpyDeviceToHost, ctx->stream),
       "copy info");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    for (int i = 0; i < m; ++i)
      host_out[(size_t)(c0 + i) * AXPIC_CELL_INFO_LEN + AXPIC_CI_GAMMA0_P] /= ctx->prm.dt_phys_s;
  }
  return AXPIC_OK;
}

axpic_status axpic_get_cell_diag(axpic_ctx* ctx, int32_t first, int32_t count, double* host_out) {
  if (!ctx) return AXPIC_E_INVALID;
  if (first < 0 || count < 0 || first + count > ctx->desc.ncells || (count > 0 && !host_out))
    return fail(ctx, AXPIC_E_INVALID, "axpic_get_cell_diag: range outside the cells");
  CK(cudaMemcpyAsync(host_out, ctx->diag + (size_t)first * AXPIC_CELL_DIAG_LEN,
                     sizeof(double) * AXPIC_CELL_DIAG_LEN * (size_t)count, cudaMemcpyDeviceToHost, ctx->stream),
     "copy diag");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_get_residuals(axpic_ctx* ctx, int32_t first, int32_t count, double* host_out) {
  if (!ctx) return AXPIC_E_INVALID;
  if (first < 0 || count < 0 || first + count > ctx->desc.ncells || (count > 0 && !host_out))
    return fail(ctx, AXPIC_E_INVALID, "axpic_get_residuals: range outside the cells");
  CK(cudaMemcpyAsync(host_out, ctx->res + (size_t)first * 4, sizeof(double) * 4 * (size_t)count,
                     cudaMemcpyDeviceToHost, ctx->stream),
     "copy residuals");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_profile_begin(axpic_ctx* ctx, int32_t max_steps) {
  if (!ctx || max_steps < 0 || max_steps > (1 << 20)) return AXPIC_E_INVALID;
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  free_events(ctx);
  ctx->prof_events.resize((kStepKernels + 1) * (size_t)max_steps);
  for (auto& e : ctx->prof_events) CK(cudaEventCreate(&e), "event create");
  ctx->prof_max = max_steps;
  return AXPIC_OK;
}

axpic_status axpic_profile_end(axpic_ctx* ctx, double* ms_out, int32_t* steps_out) {
  if (!ctx || !ms_out) return AXPIC_E_INVALID;
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  static_assert(kStepKernels <= AXPIC_PROFILE_SLOTS, "profile slots");
  for (int k = 0; k < AXPIC_PROFILE_SLOTS; ++k) ms_out[k] = 0.0;
  for (int s = 0; s < ctx->prof_used; ++s) {
    const cudaEvent_t* ev = ctx->prof_events.data() + (kStepKernels + 1) * s;
    for (int k = 0; k < kStepKernels; ++k) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]), "elapsed");
      ms_out[k] += ms;
    }
  }
  if (steps_out) *steps_out = ctx->prof_used;
  free_events(ctx);
  return AXPIC_OK;
}

// The steps a replayed graph holds (nsteps of them). With several branches
// the cells are split into ranges of whole event CTAs (128 cells); each
// range's kernels run nsteps steps on a stream forked from gs, reading and
// advancing their own step counter, and join gs at the end. Cells are
// independent, so the results are those of one launch over all cells.
static cudaError_t capture_steps(axpic_ctx* ctx, StepArgs A, int nsteps, cudaStream_t gs, const SrArgs* sra) {
  const int n = ctx->desc.ncells;
  const int part = ((n + ctx->branches - 1) / ctx->branches + 127) / 128 * 128;
  cudaError_t e;
  if (ctx->branches == 1 || part >= n) {
    for (int k = 0; k < nsteps; ++k)
      if ((e = launch_step(PH_ALL, A, ctx->warps, gs, nullptr, sra))) return e;
    return cudaSuccess;
  }
  for (int b = 0; b < kMaxBranches; ++b) {
    if (!ctx->br_stream[b] && (e = cudaStreamCreateWithFlags(&ctx->br_stream[b], cudaStreamNonBlocking))) return e;
  }
  for (int b = 0; b <= kMaxBranches; ++b) {
    if (!ctx->br_ev[b] && (e = cudaEventCreateWithFlags(&ctx->br_ev[b], cudaEventDisableTiming))) return e;
  }
  if ((e = cudaEventRecord(ctx->br_ev[kMaxBranches], gs))) return e;
  int nb = 0;
  for (int c0 = 0; c0 < n; c0 += part, ++nb) {
    StepArgs B = A;
    B.cell0 = c0;
    B.ncells = std::min(part, n - c0);
    B.step_dev = ctx->step_dev + nb;
    B.heavy_n = ctx->heavy_n + nb;
    SrArgs Bsr;
    if (sra) {  // the branch's records, rebuilt after its temperature update
      Bsr = *sra;
      Bsr.cell0 = B.cell0;
      Bsr.ncells = B.ncells;
    }
    cudaStream_t bs = ctx->br_stream[nb];
    if ((e = cudaStreamWaitEvent(bs, ctx->br_ev[kMaxBranches], 0))) return e;
    for (int k = 0; k < nsteps; ++k)
      if ((e = launch_step(PH_ALL, B, ctx->warps, bs, nullptr, sra ? &Bsr : nullptr))) return e;
    if ((e = cudaEventRecord(ctx->br_ev[nb], bs))) return e;
  }
  for (int b = 0; b < nb; ++b)
    if ((e = cudaStreamWaitEvent(gs, ctx->br_ev[b], 0))) return e;
  return cudaSuccess;
}

// The graph of nsteps steps for channel_mask, captured on first use.
static axpic_status stream_setup(axpic_ctx* ctx, int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_s,
                                 double mass_keV, int32_t boundary, StreamArgs* out);

static axpic_status step_graph(axpic_ctx* ctx, int64_t first_step, int nsteps, int32_t channel_mask,
                               cudaGraphExec_t* out, const StreamArgs* sa = nullptr) {
  const int key = channel_mask * 1024 + nsteps;
  std::map<int, cudaGraphExec_t>& cache = sa ? ctx->sgraphs : ctx->graphs;
  auto it = cache.find(key);
  if (it == cache.end()) {
    StepArgs A = make_args(ctx, first_step, channel_mask);
    A.step_dev = ctx->step_dev;
    cudaStream_t gs = ctx->graph_stream;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture");
    const SrArgs sra = make_sr_args(ctx);
    cudaError_t le = cudaSuccess;
    if (!sa) {
      le = capture_steps(ctx, A, nsteps, gs, ctx->prm.rate_model ? &sra : nullptr);
    } else {
      // each step (its branches joined: migration crosses them), then the
      // axions' streaming over all cells
      for (int k = 0; k < nsteps && le == cudaSuccess; ++k) {
        le = capture_steps(ctx, A, 1, gs, ctx->prm.rate_model ? &sra : nullptr);
        if (le == cudaSuccess) le = launch_stream(*sa, gs);
      }
    }
    const cudaError_t ce = cudaStreamEndCapture(gs, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, le != cudaSuccess ? le : ce, "axpic_run_steps: capture");
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(ctx, ie, "axpic_run_steps: instantiate");
    it = cache.emplace(key, ex).first;
  }
  *out = it->second;
  return AXPIC_OK;
}

axpic_status axpic_run_steps(axpic_ctx* ctx, int64_t first_step, int32_t nsteps, int32_t channel_mask) {
  AXPIC_RANGE("axpic_run_steps");
  if (!ctx) return AXPIC_E_INVALID;
  if (nsteps < 0 || first_step < 0 || first_step + (int64_t)nsteps >= (int64_t)0xFFFFFFFF)
    return fail(ctx, AXPIC_E_INVALID, "axpic_run_steps: step range outside [0, 2^32 - 1)");
  if (channel_mask & ~AXPIC_CH_ALL) return fail(ctx, AXPIC_E_INVALID, "axpic_run_steps: unknown channel bits");
  if (nsteps == 0 || ctx->desc.ncells == 0) return AXPIC_OK;
  if (!ctx->graph_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking), "stream create");
    CK(cudaEventCreateWithFlags(&ctx->graph_ev[0], cudaEventDisableTiming), "event create");
    CK(cudaEventCreateWithFlags(&ctx->graph_ev[1], cudaEventDisableTiming), "event create");
  }
  cudaStream_t gs = ctx->graph_stream;
  // ordered after the work already queued on the context's stream
  CK(cudaEventRecord(ctx->graph_ev[0], ctx->stream), "event record");
  CK(cudaStreamWaitEvent(gs, ctx->graph_ev[0], 0), "stream wait");
  // both graphs (32 steps and one) are captured on the first call for a mask,
  // so that later calls of any length launch without capturing
  cudaGraphExec_t many = nullptr, one = nullptr;
  axpic_status st;
  if ((st = step_graph(ctx, first_step, kGraphSteps, channel_mask, &many))) return st;
  if ((st = step_graph(ctx, first_step, 1, channel_mask, &one))) return st;
  CK(launch_set_step(ctx->step_dev, (uint32_t)first_step, kMaxBranches, gs), "set step");
  for (int32_t k = 0; k < nsteps / kGraphSteps; ++k) CK(cudaGraphLaunch(many, gs), "graph launch");
  for (int32_t k = 0; k < nsteps % kGraphSteps; ++k) CK(cudaGraphLaunch(one, gs), "graph launch");
  CK(cudaEventRecord(ctx->graph_ev[1], gs), "event record");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->graph_ev[1], 0), "stream wait");
  return AXPIC_OK;
}

axpic_status axpic_run_steps_streamed(axpic_ctx* ctx, int64_t first_step, int32_t nsteps, int32_t channel_mask,
                                      int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_stream_s,
                                      double mass_keV, int32_t boundary) {
  AXPIC_RANGE("axpic_run_steps_streamed");
  if (!ctx) return AXPIC_E_INVALID;
  if (nsteps < 0 || first_step < 0 || first_step + (int64_t)nsteps >= (int64_t)0xFFFFFFFF)
    return fail(ctx, AXPIC_E_INVALID, "axpic_run_steps_streamed: step range outside [0, 2^32 - 1)");
  if (channel_mask & ~AXPIC_CH_ALL)
    return fail(ctx, AXPIC_E_INVALID, "axpic_run_steps_streamed: unknown channel bits");
  StreamArgs sa;
  axpic_status st = stream_setup(ctx, nx, ny, nz, h_cm, dt_stream_s, mass_keV, boundary, &sa);
  if (st != AXPIC_OK) return st;
  if (nsteps == 0 || ctx->desc.ncells == 0) return AXPIC_OK;
  // graphs captured for other streaming parameters are dropped
  int32_t kbits, mbits;
  std::memcpy(&kbits, &sa.kappa, 4);
  std::memcpy(&mbits, &sa.mu, 4);
  const std::vector<int64_t> sig = {nx, ny, nz, kbits, mbits, sa.periodic};
  if (sig != ctx->stream_sig) {
    for (auto& g : ctx->sgraphs) cudaGraphExecDestroy(g.second);
    ctx->sgraphs.clear();
    ctx->stream_sig = sig;
  }
  if (!ctx->graph_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking), "stream create");
    CK(cudaEventCreateWithFlags(&ctx->graph_ev[0], cudaEventDisableTiming), "event create");
    CK(cudaEventCreateWithFlags(&ctx->graph_ev[1], cudaEventDisableTiming), "event create");
  }
  cudaStream_t gs = ctx->graph_stream;
  CK(cudaEventRecord(ctx->graph_ev[0], ctx->stream), "event record");
  CK(cudaStreamWaitEvent(gs, ctx->graph_ev[0], 0), "stream wait");
  cudaGraphExec_t many = nullptr, one = nullptr;
  if ((st = step_graph(ctx, first_step, kGraphSteps, channel_mask, &many, &sa))) return st;
  if ((st = step_graph(ctx, first_step, 1, channel_mask, &one, &sa))) return st;
  CK(launch_set_step(ctx->step_dev, (uint32_t)first_step, kMaxBranches, gs), "set step");
  for (int32_t k = 0; k < nsteps / kGraphSteps; ++k) CK(cudaGraphLaunch(many, gs), "graph launch");
  for (int32_t k = 0; k < nsteps % kGraphSteps; ++k) CK(cudaGraphLaunch(one, gs), "graph launch");
  CK(cudaEventRecord(ctx->graph_ev[1], gs), "event record");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->graph_ev[1], 0), "stream wait");
  return AXPIC_OK;
}

// The context's device state, as (pointer, bytes) pairs: what a step reads or
// writes. The autotuner saves and restores exactly this.
static std::vector<std::pair<void*, size_t>> state_buffers(axpic_ctx* ctx, bool with_caller = true) {
  const axpic_plasma_desc& d = ctx->desc;
  const size_t n = (size_t)d.ncells;
  std::vector<std::pair<void*, size_t>> b;
  if (with_caller) {  // the caller's slabs and T
    for (const axpic_species* s : {&d.electrons, &d.photons, &d.axions}) {
      const size_t slots = n * (size_t)s->capacity * sizeof(float);
      b.emplace_back(s->wp, 4 * slots);
      b.emplace_back(s->xyz, 4 * slots);
      b.emplace_back(s->count, n * sizeof(int32_t));
    }
    b.emplace_back(d.T_keV, n * sizeof(double));
  }
  const size_t bit_words = mask_words(d);
  b.emplace_back(ctx->rec, n * kRecLen * sizeof(float));
  b.emplace_back(ctx->mom, n * kMomLen * sizeof(float));
  b.emplace_back(ctx->xbuf, n * 4 * sizeof(double));
  b.emplace_back(ctx->res, n * 4 * sizeof(double));
  b.emplace_back(ctx->diag, n * AXPIC_CELL_DIAG_LEN * sizeof(double));
  b.emplace_back(ctx->photon_start, n * sizeof(int32_t));
  b.emplace_back(ctx->tally, (3 * (size_t)ctx->prm.tally_nbins + 6) * sizeof(double));
  b.emplace_back(ctx->counters, sizeof(unsigned long long) * kNumCounters * (size_t)ctx->ctr_rows);
  b.emplace_back(ctx->err, sizeof(int));
  b.emplace_back(ctx->bits, bit_words * sizeof(uint32_t));
  if (ctx->sr) b.emplace_back(ctx->sr, n * kSrLen * sizeof(float));
  if (ctx->sr_src) b.emplace_back(ctx->sr_src, n);
  return b;
}

static cudaError_t copy_state(axpic_ctx* ctx, unsigned char* save, bool to_save) {
  size_t off = 0;
  for (auto& b : state_buffers(ctx)) {
    if (b.second == 0) continue;
    void* dst = to_save ? (void*)(save + off) : b.first;
    const void* src = to_save ? (const void*)b.first : (const void*)(save + off);
    const cudaError_t e = cudaMemcpyAsync(dst, src, b.second, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    off += (b.second + 255) & ~size_t(255);
  }
  return cudaSuccess;
}

static void set_shape(axpic_ctx* ctx, int chunk, int warps, int dec_grid) {
  ctx->dec_chunk = chunk;
  ctx->dec_grid = dec_grid;
  ctx->warps = warps;
  ctx->grid = (ctx->desc.ncells + warps - 1) / warps;
}

axpic_status axpic_launch_shape(const axpic_ctx* ctx, int32_t* decide_chunk, int32_t* event_warps,
                                int32_t* step_branches) {
  if (!ctx) return AXPIC_E_INVALID;
  if (decide_chunk) *decide_chunk = ctx->dec_chunk;
  if (event_warps) *event_warps = ctx->warps;
  if (step_branches) {
    const int n = ctx->desc.ncells;
    const int part = ((n + ctx->branches - 1) / ctx->branches + 127) / 128 * 128;
    *step_branches = (ctx->branches == 1 || part >= n) ? 1 : (n + part - 1) / part;
  }
  return AXPIC_OK;
}

axpic_status axpic_autotune(axpic_ctx* ctx, int64_t step, int32_t trial_steps, int32_t channel_mask,
                            double* best_ms_out, int32_t* chunk_out, int32_t* warps_out) {
  AXPIC_RANGE("axpic_autotune");
  if (!ctx) return AXPIC_E_INVALID;
  if (trial_steps < 1 || step < 0 || step + (int64_t)trial_steps >= (int64_t)0xFFFFFFFF)
    return fail(ctx, AXPIC_E_INVALID, "axpic_autotune: trial_steps < 1 or step range outside [0, 2^32 - 1)");
  if (channel_mask & ~AXPIC_CH_ALL) return fail(ctx, AXPIC_E_INVALID, "axpic_autotune: unknown channel bits");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  size_t total = 0;
  for (auto& b : state_buffers(ctx)) total += (b.second + 255) & ~size_t(255);
  unsigned char* save = nullptr;
  CK(cudaMalloc((void**)&save, total > 0 ? total : 256), "autotune scratch");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int keep_chunk = ctx->dec_chunk, keep_warps = ctx->warps, keep_grid = ctx->dec_grid;
  int best_chunk = keep_chunk, best_warps = keep_warps, best_grid = keep_grid;
  double best = -1.0;
  cudaError_t e = copy_state(ctx, save, true);
  if (!e) e = cudaEventCreate(&e0);
  if (!e) e = cudaEventCreate(&e1);
  for (int chunk : {4, 8, 16, 32}) {
    int dgrid = 1;
    if (!e) e = decide_resident_ctas(chunk, &dgrid);
    for (int warps : {2, 4}) {
      if (e) break;
      if (warps > ctx->max_warps) continue;
      set_shape(ctx, chunk, warps, dgrid);
      // one untimed step, then trial_steps timed ones, from the saved state
      StepArgs A = make_args(ctx, step, channel_mask);
      const SrArgs sra = make_sr_args(ctx);
      const SrArgs* sp = ctx->prm.rate_model ? &sra : nullptr;
      if ((e = launch_step(PH_ALL, A, ctx->warps, ctx->stream, nullptr, sp)) || (e = cudaEventRecord(e0, ctx->stream)))
        break;
      for (int32_t k = 0; k < trial_steps && !e; ++k) {
        A = make_args(ctx, step + 1 + k, channel_mask);
        e = launch_step(PH_ALL, A, ctx->warps, ctx->stream, nullptr, sp);
      }
      float ms = 0.f;
      if (e || (e = cudaEventRecord(e1, ctx->stream)) || (e = cudaEventSynchronize(e1)) ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) || (e = copy_state(ctx, save, false)))
        break;
      const double per = ms / trial_steps;
      if (best < 0.0 || per < best) {
        best = per;
        best_chunk = chunk;
        best_warps = warps;
        best_grid = dgrid;
      }
    }
  }
  if (!e) e = cudaStreamSynchronize(ctx->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(save);
  if (e) {
    set_shape(ctx, keep_chunk, keep_warps, keep_grid);
    return cuda_fail(ctx, e, "axpic_autotune");
  }
  set_shape(ctx, best_chunk, best_warps, best_grid);
  free_graphs(ctx);
  if (best_ms_out) *best_ms_out = best;
  if (chunk_out) *chunk_out = best_chunk;
  if (warps_out) *warps_out = best_warps;
  return AXPIC_OK;
}

axpic_status axpic_set_surrogate(axpic_ctx* ctx, axpic_mlp* m, const float* err_map, int32_t nT, int32_t nne,
                                 float tol_rate, float tol_quantile) {
  AXPIC_RANGE("axpic_set_surrogate");
  if (!ctx || !m || !err_map) return AXPIC_E_INVALID;
  if (ctx->prm.rate_model != 2) return fail(ctx, AXPIC_E_INVALID, "axpic_set_surrogate: rate_model is not 2");
  if (nT < 2 || nne < 2 || nT > 4096 || nne > 4096) return fail(ctx, AXPIC_E_INVALID, "axpic_set_surrogate: grid");
  if (!(tol_rate >= 0.f) || !(tol_quantile >= 0.f))
    return fail(ctx, AXPIC_E_INVALID, "axpic_set_surrogate: tolerances must be >= 0");
  std::vector<float> P(AXPIC_MLP_PARAMS), mu(96), sigma(96), skip(96 * 4);
  axpic_status s;
  if ((s = axpic_mlp_get_params(m, P.data())) != AXPIC_OK || (s = axpic_mlp_get_norm(m, mu.data(), sigma.data())) ||
      (s = axpic_mlp_get_skip(m, skip.data())))
    return fail(ctx, s, "axpic_set_surrogate: reading the network");
  // the step samples emission energies from the Compton-like and
  // bremsstrahlung quantiles of the model, which must not depend on the cell
  std::vector<float> uni(kSrLen, 0.f);
  for (int ch = 1; ch < 3; ++ch)
    for (int j = 1; j < 32; ++j) {
      const int o = 32 * ch + j;
      if (sigma[o] != 0.f || skip[o * 4 + 1] != 0.f || skip[o * 4 + 2] != 0.f || skip[o * 4 + 3] != 0.f)
        return fail(ctx, AXPIC_E_INVALID,
                    "axpic_set_surrogate: the Compton-like and bremsstrahlung quantiles must not depend on the cell "
                    "(their sigma and S zero, as axpic_surrogate_fit leaves them)");
      uni[96 + 31 * ch + j - 1] = mu[o];
    }
  // nodes that pass, then trusted nodes: those whose 3 x 3 neighbourhood
  // (within the grid, per Z) passes
  std::vector<uint8_t> pass((size_t)2 * nT * nne), trust(pass.size());
  for (size_t i = 0; i < pass.size(); ++i)
    pass[i] = err_map[3 * i] <= tol_rate && err_map[3 * i + 1] <= tol_quantile ? 1 : 0;
  int any = 0;
  for (int z = 0; z < 2; ++z)
    for (int j = 0; j < nne; ++j)
      for (int i = 0; i < nT; ++i) {
        uint8_t t = 1;
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            const int jj = j + dj, ii = i + di;
            if (jj >= 0 && jj < nne && ii >= 0 && ii < nT) t &= pass[((size_t)z * nne + jj) * nT + ii];
          }
        trust[((size_t)z * nne + j) * nT + i] = t;
        any |= t;
      }
  cudaStream_t st = ctx->stream;
  CK(cudaStreamSynchronize(st), "synchronize");
  if (ctx->sur_trust) cudaFree(ctx->sur_trust);
  ctx->sur_trust = nullptr;
  CK(cudaMalloc((void**)&ctx->sur_trust, trust.size()), "trust map");
  CK(cudaMemcpyAsync(ctx->sur_P, P.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice, st), "params");
  CK(cudaMemcpyAsync(ctx->sur_mu, mu.data(), sizeof(float) * 96, cudaMemcpyHostToDevice, st), "norm");
  CK(cudaMemcpyAsync(ctx->sur_sigma, sigma.data(), sizeof(float) * 96, cudaMemcpyHostToDevice, st), "norm");
  CK(cudaMemcpyAsync(ctx->sur_skip, skip.data(), sizeof(float) * 96 * 4, cudaMemcpyHostToDevice, st), "skip");
  CK(cudaMemcpyAsync(ctx->sur_uni, uni.data(), sizeof(float) * kSrLen, cudaMemcpyHostToDevice, st), "quantiles");
  CK(cudaMemcpyAsync(ctx->sur_trust, trust.data(), trust.size(), cudaMemcpyHostToDevice, st), "trust map");
  CK(launch_net_image(ctx->sur_P, ctx->sur_mu, ctx->sur_sigma, ctx->sur_skip, ctx->sur_img, st), "network image");
  ctx->tnT = nT;
  ctx->tnne = nne;
  ctx->sur_set = 1;
  ctx->sur_any_trusted = any;
  free_graphs(ctx);
  const axpic_plasma_desc& d = ctx->desc;
  CK(launch_records(d.ncells, d.nspecies, ctx->cc, d.T_keV, d.n_ion, ctx->rec, ctx->err, st), "records");
  CK(build_records(ctx, st), "rate-model records");
  CK(cudaStreamSynchronize(st), "synchronize");
  return read_err(ctx);
}

axpic_status axpic_get_cell_records(axpic_ctx* ctx, int32_t first, int32_t count, float* rec_out, uint8_t* src_out) {
  if (!ctx || first < 0 || count < 0 || first + count > ctx->desc.ncells || (count > 0 && !rec_out))
    return AXPIC_E_INVALID;
  if (count == 0) return AXPIC_OK;
  CK(cudaMemcpyAsync(rec_out, ctx->rec + (size_t)first * kRecLen, sizeof(float) * kRecLen * count,
                     cudaMemcpyDeviceToHost, ctx->stream),
     "copy records");
  if (src_out) {
    if (ctx->sr_src) {
      CK(cudaMemcpyAsync(src_out, ctx->sr_src + first, (size_t)count, cudaMemcpyDeviceToHost, ctx->stream),
         "copy sources");
    } else {
      std::memset(src_out, ctx->prm.rate_model == 1 ? 1 : 0, (size_t)count);
    }
  }
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

// Validates the streaming parameters, makes the scratch on first use and fills
// the kernels' arguments (nothing is launched).
static axpic_status stream_setup(axpic_ctx* ctx, int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_s,
                                 double mass_keV, int32_t boundary, StreamArgs* out) {
  const axpic_plasma_desc& d = ctx->desc;
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz != d.ncells)
    return fail(ctx, AXPIC_E_INVALID, "axpic_stream_axions: nx ny nz must give the context's cells");
  if (!(h_cm > 0) || !std::isfinite(h_cm) || !(dt_s >= 0) || !std::isfinite(dt_s) || !(mass_keV >= 0) ||
      !std::isfinite(mass_keV) || (boundary != 0 && boundary != 1))
    return fail(ctx, AXPIC_E_INVALID, "axpic_stream_axions: h, dt, mass or boundary");
  const float kappa = (float)(2.99792458e10 * dt_s / h_cm);
  if (!(kappa < 1.0f - 0x1p-20f))
    return fail(ctx, AXPIC_E_INVALID, "axpic_stream_axions: c dt must stay below the cell edge");
  const size_t slots = (size_t)d.ncells * d.axions.capacity;
  if (!ctx->st_dir) {
    CK(cudaMalloc((void**)&ctx->st_dir, std::max<size_t>(slots, 1)), "streaming scratch");
    CK(cudaMalloc((void**)&ctx->st_cnt, sizeof(int32_t) * 2 * kStreamDirs * (size_t)d.ncells), "streaming scratch");
    CK(cudaMalloc((void**)&ctx->st_buf, sizeof(float) * 8 * std::max<size_t>(slots, 1)), "streaming scratch");
    CK(cudaMalloc((void**)&ctx->st_stats, sizeof(double) * 4), "streaming scratch");
    CK(cudaMemsetAsync(ctx->st_stats, 0, sizeof(double) * 4, ctx->stream), "memset");
  }
  StreamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s = to_ptrs(d.axions);
  a.ncells = d.ncells;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.kappa = kappa;
  a.mu = (float)(mass_keV / kMeC2);
  a.periodic = boundary == 0;
  a.dir = ctx->st_dir;
  a.cnt = ctx->st_cnt;
  a.goff = ctx->st_cnt + (size_t)kStreamDirs * d.ncells;
  a.buf = ctx->st_buf;
  a.stats = ctx->st_stats;
  a.err = ctx->err;
  *out = a;
  return AXPIC_OK;
}

axpic_status axpic_stream_axions(axpic_ctx* ctx, int32_t nx, int32_t ny, int32_t nz, double h_cm, double dt_s,
                                 double mass_keV, int32_t boundary) {
  AXPIC_RANGE("axpic_stream_axions");
  if (!ctx) return AXPIC_E_INVALID;
  StreamArgs a;
  const axpic_status st = stream_setup(ctx, nx, ny, nz, h_cm, dt_s, mass_keV, boundary, &a);
  if (st != AXPIC_OK) return st;
  CK(launch_stream(a, ctx->stream), "stream kernels");
  return AXPIC_OK;
}

axpic_status axpic_state_bytes(axpic_ctx* ctx, uint64_t* bytes) {
  if (!ctx || !bytes) return AXPIC_E_INVALID;
  uint64_t t = 0;
  for (auto& b : state_buffers(ctx, false)) t += b.second;
  *bytes = t;
  return AXPIC_OK;
}

axpic_status axpic_save_state(axpic_ctx* ctx, void* host_out, uint64_t bytes) {
  AXPIC_RANGE("axpic_save_state");
  uint64_t need = 0;
  if (!ctx || !host_out || axpic_state_bytes(ctx, &need) != AXPIC_OK || bytes != need)
    return ctx ? fail(ctx, AXPIC_E_INVALID, "axpic_save_state: buffer size") : AXPIC_E_INVALID;
  unsigned char* p = static_cast<unsigned char*>(host_out);
  for (auto& b : state_buffers(ctx, false)) {
    CK(cudaMemcpyAsync(p, b.first, b.second, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    p += b.second;
  }
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_load_state(axpic_ctx* ctx, const void* host_in, uint64_t bytes) {
  AXPIC_RANGE("axpic_load_state");
  uint64_t need = 0;
  if (!ctx || !host_in || axpic_state_bytes(ctx, &need) != AXPIC_OK || bytes != need)
    return ctx ? fail(ctx, AXPIC_E_INVALID, "axpic_load_state: buffer size") : AXPIC_E_INVALID;
  const unsigned char* p = static_cast<const unsigned char*>(host_in);
  for (auto& b : state_buffers(ctx, false)) {
    CK(cudaMemcpyAsync(b.first, p, b.second, cudaMemcpyHostToDevice, ctx->stream), "copy");
    p += b.second;
  }
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_merge_axions(axpic_ctx* ctx, int32_t n_target, int32_t nedges, const float* edges_p2) {
  AXPIC_RANGE("axpic_merge_axions");
  if (!ctx) return AXPIC_E_INVALID;
  if (n_target < 0 || nedges < 0 || nedges > kMergeMaxEdges || (nedges > 0 && !edges_p2))
    return fail(ctx, AXPIC_E_INVALID, "axpic_merge_axions: n_target or thresholds");
  for (int k = 0; k < nedges; ++k)
    if (!std::isfinite(edges_p2[k]) || edges_p2[k] < 0.f || (k > 0 && !(edges_p2[k] > edges_p2[k - 1])))
      return fail(ctx, AXPIC_E_INVALID, "axpic_merge_axions: thresholds must be finite, >= 0 and ascending");
  const axpic_plasma_desc& d = ctx->desc;
  if (!ctx->mg_grp) {
    CK(merge_init_kernels(), "merge kernel attributes");
    CK(cudaMalloc((void**)&ctx->mg_grp, std::max<size_t>((size_t)d.ncells * d.axions.capacity, 1)), "merge scratch");
    CK(cudaMalloc((void**)&ctx->mg_removed, sizeof(double)), "merge scratch");
    CK(cudaMemsetAsync(ctx->mg_removed, 0, sizeof(double), ctx->stream), "memset");
  }
  MergeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s = to_ptrs(d.axions);
  a.ncells = d.ncells;
  a.n_target = n_target;
  a.nedges = nedges;
  for (int k = 0; k < nedges; ++k) a.edges[k] = edges_p2[k];
  a.grp = ctx->mg_grp;
  a.removed = ctx->mg_removed;
  CK(launch_merge(a, ctx->stream), "merge kernel");
  return AXPIC_OK;
}

axpic_status axpic_merge_stats(axpic_ctx* ctx, double* removed) {
  if (!ctx || !removed) return AXPIC_E_INVALID;
  *removed = 0.0;
  if (!ctx->mg_removed) return AXPIC_OK;
  CK(cudaMemcpyAsync(removed, ctx->mg_removed, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_stream_stats(axpic_ctx* ctx, double* out) {
  if (!ctx || !out) return AXPIC_E_INVALID;
  for (int i = 0; i < 4; ++i) out[i] = 0.0;
  if (!ctx->st_stats) return AXPIC_OK;
  CK(cudaMemcpyAsync(out, ctx->st_stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

axpic_status axpic_get_spectral_records(axpic_ctx* ctx, int32_t first, int32_t count, float* out) {
  if (!ctx || !out || first < 0 || count < 0 || first + count > ctx->desc.ncells) return AXPIC_E_INVALID;
  if (!ctx->sr) return fail(ctx, AXPIC_E_INVALID, "axpic_get_spectral_records: rate_model 0 keeps no records");
  if (count == 0) return AXPIC_OK;
  CK(cudaMemcpyAsync(out, ctx->sr + (size_t)first * kSrLen, sizeof(float) * kSrLen * count, cudaMemcpyDeviceToHost,
                     ctx->stream),
     "copy");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return AXPIC_OK;
}

const char* axpic_step_kernel_names(const axpic_ctx* ctx) {
  return ctx ? step_kernel_names(ctx->prm.rate_model, ctx->prm.T_mode) : "";
}

axpic_status axpic_sync(axpic_ctx* ctx) {
  if (!ctx) return AXPIC_E_INVALID;
  return read_err(ctx);
}

axpic_status axpic_destroy(axpic_ctx* ctx) {
  if (!ctx) return AXPIC_E_INVALID;
  axpic_status s = read_err(ctx);
  free_ctx(ctx);
  return s;
}


// ---------------------------------------------------------------- no-alloc step
// Scratch of axpic_step_noalloc: a file-scope device array, so the call
// allocates nothing. Every GPU that loads the library holds it until exit.
// Layout: rate records, electron moments, sampling tables, per-CTA counters,
// error flag.
namespace {
constexpr int kNoAllocMaxCells = 16384;
constexpr int kNoAllocWarps = 4;
constexpr int kNoAllocMaxGrid = kNoAllocMaxCells / kNoAllocWarps;
constexpr size_t kNaRec = 0;
constexpr size_t kNaMom = kNaRec + sizeof(float) * kRecLen * kNoAllocMaxCells;
constexpr size_t kNaTables = kNaMom + sizeof(float) * kMomLen * kNoAllocMaxCells;
constexpr size_t kNaCounters = kNaTables + sizeof(float) * kNumTables * kTableN;
constexpr size_t kNaErr = kNaCounters + sizeof(unsigned long long) * kNumCounters * kNoAllocMaxGrid;
constexpr size_t kNaXbuf = kNaErr + 256;
constexpr size_t kNaStart = kNaXbuf + sizeof(double) * 4 * kNoAllocMaxCells;
constexpr size_t kNaBitsBytes = 4u << 20;  // decision bit masks: cells * (acap + gcap + ecap) / 8 bytes
constexpr size_t kNaBits = kNaStart + sizeof(int32_t) * kNoAllocMaxCells;
constexpr size_t kNaRecBytes = 16u << 20;  // decision records: cells * (16 (acap + gcap) + 4 ecap) bytes
constexpr size_t kNaRecs = kNaBits + kNaBitsBytes;
constexpr size_t kNaHeavy = kNaRecs + kNaRecBytes;  // cells left to the warp-path event kernel
constexpr size_t kNaHeavyN = kNaHeavy + sizeof(int32_t) * kNoAllocMaxCells;
constexpr size_t kNaUnused = kNaHeavyN + 256;  // diagnostic/tally slots never touched
constexpr size_t kNoAllocBytes = kNaUnused + 256;
// the event kernel copies exchange buffers by 16-byte cp.async
static_assert(kNaXbuf % 16 == 0, "exchange buffers 16-byte aligned");
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_na_mu;
unsigned char* g_na_base[kNoAllocMaxDevices] = {};
double g_na_brems[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

axpic_status axpic_step_noalloc(const axpic_plasma_desc* desc, const axpic_params* params, int64_t step,
                                int32_t channel_mask, double* carry, void* stream) {
  AXPIC_RANGE("axpic_step_noalloc");
  if (!desc || !params || !carry) return AXPIC_E_INVALID;
  const axpic_plasma_desc& d = *desc;
  const axpic_params& p = *params;
  auto bad = [](const char* m) {
    fprintf(stderr, "axpic_step_noalloc: %s\n", m);
    return AXPIC_E_INVALID;
  };
  if (d.ncells > kNoAllocMaxCells) return bad("ncells above 16384, the scratch maximum");
  const std::string why = check_plasma(d, p);
  if (!why.empty()) return bad(why.c_str());
  if (step < 0 || step >= (int64_t)0xFFFFFFFF || (channel_mask & ~AXPIC_CH_ALL)) return bad("bad step or mask");
  if (p.rate_model != 0) return bad("rate_model must be 0 (the records need a context)");
  const size_t per_warp = step_smem_per_warp(d.axions.capacity, d.photons.capacity, d.electrons.capacity);
  if (per_warp * kNoAllocWarps > 227 * 1024 - 128) return bad("slab capacities too large");
  const size_t bit_bytes = sizeof(uint32_t) * mask_words(d);
  if (bit_bytes > kNaBitsBytes) return bad("ncells * (capacities) / 8 above the 4 MiB mask scratch");
  const size_t rec_bytes = (size_t)d.ncells * (16 * ((size_t)d.axions.capacity + d.photons.capacity) +
                                               4 * (size_t)d.electrons.capacity);
  if (rec_bytes > kNaRecBytes) return bad("ncells * (16 (acap + gcap) + 4 ecap) above the 16 MiB record scratch");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return AXPIC_E_CUDA;
  unsigned char* base = nullptr;
  {
    // set-up, once per device and with that device current: the device
    // address of the scratch array (its name is only a host stand-in here)
    // and the sampling tables for the requested bremsstrahlung shape
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_base[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return AXPIC_E_CUDA;
      g_na_base[dev] = static_cast<unsigned char*>(ptr);
      g_na_brems[dev] = -1.0;
    }
    base = g_na_base[dev];
    if (g_na_brems[dev] != p.brems_gamma_shape) {
      static float tab[kNumTables * kTableN];
      build_tables(p.brems_gamma_shape, tab);
      if (cudaMemcpyAsync(base + kNaTables, tab, sizeof(tab), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return AXPIC_E_CUDA;
      g_na_brems[dev] = p.brems_gamma_shape;
    }
  }
  // a context on the stack that points into the scratch (no member allocates)
  axpic_ctx c;
  c.desc = d;
  c.prm = p;
  c.prm.diag_enable = 0;
  c.prm.tally_enable = 0;
  c.stream = st;
  c.rec = reinterpret_cast<float*>(base + kNaRec);
  c.mom = reinterpret_cast<float*>(base + kNaMom);
  c.tables = reinterpret_cast<float*>(base + kNaTables);
  c.counters = reinterpret_cast<unsigned long long*>(base + kNaCounters);
  c.err = reinterpret_cast<int*>(base + kNaErr);
  c.xbuf = reinterpret_cast<double*>(base + kNaXbuf);
  c.photon_start = reinterpret_cast<int32_t*>(base + kNaStart);
  c.diag = reinterpret_cast<double*>(base + kNaUnused);
  c.tally = reinterpret_cast<double*>(base + kNaUnused);
  c.bits = reinterpret_cast<uint32_t*>(base + kNaBits);
  c.recA = reinterpret_cast<uint4*>(base + kNaRecs);
  c.heavy = reinterpret_cast<int32_t*>(base + kNaHeavy);
  c.heavy_n = reinterpret_cast<int32_t*>(base + kNaHeavyN);
  c.recG = c.recA + (size_t)d.ncells * d.axions.capacity;
  c.recE = reinterpret_cast<uint32_t*>(c.recG + (size_t)d.ncells * d.photons.capacity);
  c.res = carry;
  c.warps = kNoAllocWarps;
  c.grid = (d.ncells + kNoAllocWarps - 1) / kNoAllocWarps;
  c.ctr_rows = std::max(1, std::min(kCounterRows, (d.ncells + 3) / 4));
  c.dec_chunk = kDefaultDecChunk;
  fold_constants(&c);
  cudaError_t e = decide_shape(p.decide_chunk, d.ncells, &c.dec_chunk, &c.dec_grid);
  if (e) {
    fprintf(stderr, "axpic_step_noalloc: %s\n", cudaGetErrorString(e));
    return AXPIC_E_CUDA;
  }
  const StepArgs A = make_args(&c, step, channel_mask);
  int h_err = 0;
  if ((e = cudaMemsetAsync(c.err, 0, sizeof(int), st)) ||
      (e = cudaMemsetAsync(c.counters, 0, sizeof(unsigned long long) * kNumCounters * (size_t)c.ctr_rows, st)) ||
      (e = cudaMemsetAsync(c.xbuf, 0, sizeof(double) * 4 * (size_t)d.ncells, st)) ||
      (e = cudaMemsetAsync(c.bits, 0, bit_bytes > 0 ? bit_bytes : 4, st)) ||
      (e = set_step_smem_limits(per_warp * kNoAllocWarps)) ||
      (e = launch_records(d.ncells, d.nspecies, c.cc, d.T_keV, d.n_ion, c.rec, c.err, st)) ||
      (e = launch_moments(d.ncells, to_ptrs(d.electrons), c.mom, st)) ||
      (e = launch_step(PH_ALL, A, kNoAllocWarps, st)) ||
      (e = cudaMemcpyAsync(&h_err, c.err, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st))) {
    fprintf(stderr, "axpic_step_noalloc: %s\n", cudaGetErrorString(e));
    return AXPIC_E_CUDA;
  }
  if (h_err & ERR_CAPACITY) return AXPIC_E_CAPACITY;
  if (h_err & ERR_NUMERIC) return AXPIC_E_NUMERIC;
  return AXPIC_OK;
}

const char* axpic_last_error(const axpic_ctx* ctx) { return ctx ? ctx->last_error.c_str() : kNoCtxMsg; }

const char* axpic_version(void) { return "axpic 0.1.0 (sm_103a)"; }

}  // extern "C"
