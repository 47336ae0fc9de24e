// The per-cell step: absorb -> emit -> feedback (Sec. II.D-II.J).
//
// A step is three kernels:
//  * decide_kernel: persistent warps over chunks of consecutive cells, lane
//    per quad of consecutive slots (float4 loads from the SoA slabs, one
//    Philox4x32-10 block per quad and stream, word j for slot 4q+j). Each
//    slot gets a cheap exact test that proves "no event this step"; slots it
//    cannot clear are flagged in a per-cell bit mask and their full decision
//    is taken from per-warp lists, 32 at a time, into slot-indexed records.
//    This kernel carries almost all the per-particle work.
//  * event_kernel: one warp per cell. It reads the bit masks and the records
//    of the flagged slots, writes products and refills removed slots at
//    offsets from warp prefix sums, so the output order is the deterministic
//    one of the method's definition, and accumulates the FP64 exchange
//    (Delta E, Delta P).
//  * feedback_kernel: thread per cell for the temperature update; the rare
//    cells whose exchange needs an affine remap are remapped by the CTA's
//    warps side by side.
// The separate API calls run the same kernels with a subset of the passes;
// the exchange passes through an FP64 per-cell buffer in the same summation
// order, so results do not depend on how a step is called.
#include <mutex>

#include "common.cuh"
#include "sr.h"
#include "step.h"

namespace axpic {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int warp_excl_scan(int v, int* total) {
  const int lane = lane_id();
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += t;
  }
  *total = __shfl_sync(kFull, x, 31);
  return x - v;
}

// Plain (coherent) 128-bit load: slabs are also written by this kernel.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

__device__ __forceinline__ bool bit(const uint32_t* b, int i) { return (b[i >> 5] >> (i & 31)) & 1u; }


// Lane-local FP64 exchange (Delta E keV, Delta P m_e c) and a flag that avoids
// FP64 zero tests on the common path.
struct Lane64 {
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0;
  bool any = false;
  __device__ void add(double w, float om, float px, float py, float pz) {
    dE += w * (double)om;
    dPx += w * (double)px;
    dPy += w * (double)py;
    dPz += w * (double)pz;
    any = true;
  }
};

// Per-CTA counters live in shared memory; events are rare, so they are
// counted with shared-memory atomics where they happen instead of holding a
// register per counter for the whole kernel.
struct Cnt {
  unsigned long long* c;
  __device__ void add(int i, unsigned v) const {
    if (v) atomicAdd(c + i, (unsigned long long)v);
  }
};

__device__ __forceinline__ void write_particle(const SpeciesPtrs& s, long idx, float w, float px, float py,
                                               float pz, float x, float y, float z) {
  s.wp[idx] = make_float4(w, px, py, pz);
  s.xyz[idx] = make_float4(x, y, z, 0.f);
}

// A slot's weight alone (the first word of its record).
__device__ __forceinline__ float& slot_w(const SpeciesPtrs& s, long idx) {
  return reinterpret_cast<float*>(s.wp + idx)[0];
}

__device__ __noinline__ void tally_add(const StepArgs& A, int ch, float w, float E) {
  const int k = (int)floorf(E * A.inv_dE_bin);
  const double wE = (double)w * (double)E;
  if (k >= 0 && k < A.nbins) atomicAdd(A.tally + ch * A.nbins + k, wE);
  atomicAdd(A.tally + 3 * A.nbins + ch, (double)w);
  atomicAdd(A.tally + 3 * A.nbins + 3 + ch, wE);
}

// ---------------------------------------------------------------- spectral records
// Rates from a cell's spectral record (table or surrogate rate model): the
// record holds ln(dQ_c/dx) + x at unit coupling on 32 points of ln x (step
// ln(400)/29, one beyond each end of [0.05, 20]); a Catmull-Rom spline in
// ln x interpolates it, the closed factors of Eqs. prim_rate and gamma_abs
// turn it into a rate.
__device__ __forceinline__ bool sr_in_range(float x) { return x >= 0.05f && x <= 20.0f; }

__device__ __forceinline__ float sr_lnL(const float* sr, int ch, float lnx) {
  float u = (lnx - kSrLnXLo) * (1.0f / kSrH) + 1.0f;
  u = fminf(fmaxf(u, 1.f), 30.f);
  const int k = min((int)u, 29);
  const float f = u - (float)k;
  const float* g = sr + ch * kSrGrid;
  const float p0 = g[k - 1], p1 = g[k], p2 = g[k + 1], p3 = g[k + 2];
  const float s = p1 + 0.5f * f * (p2 - p0 + f * (2.f * p0 - 5.f * p1 + 4.f * p2 - p3 + f * (3.f * (p1 - p2) + p3 - p0)));
  return s - fminf(fmaxf(__expf(lnx), 0.05f), 20.0f);  // the stored values are ln(dQ/dx) + x
}

// Gamma_{gamma->a} dt at the cell's couplings (multiplicity 1).
__device__ __forceinline__ float sr_prim_gdt(const float* sr, float x) {
  const float lx = logf(x);
  return expf((sr_lnL(sr, 0, lx) + sr[SR_LNKP]) - 3.f * lx) * expm1f(x);
}

// Absorption tau_c = Gamma_abs,c dt (c = 1 Compton-like, 2 bremsstrahlung).
__device__ __forceinline__ float sr_tau(const float* sr, int ch, float x, int eq_stats) {
  const float lx = logf(x);
  const float b = expf((sr_lnL(sr, ch, lx) + sr[SR_LNKA]) - 3.f * lx);
  return eq_stats ? b * expm1f(x) : b * expf(x);
}

// x from the record's 31 quantiles of channel c (end points 0.05 and 20),
// linear between quantiles.
__device__ __forceinline__ float sr_sample_x(const float* sr, int ch, float u) {
  const float t = u * 32.f;
  const int j = min((int)t, 31);
  const float f = t - (float)j;
  const float* q = sr + 96 + ch * kSrKnots;
  const float x0 = j == 0 ? 0.05f : q[j - 1];
  const float x1 = j == 31 ? 20.0f : q[j];
  return fmaf(f, x1 - x0, x0);
}

// ---------------------------------------------------------------- decisions
// One axion at the start of the step: a->gamma conversion (Sec. II.F.1, last
// paragraph) then detailed-balance absorption of the thermal-bath channels
// (Sec. II.I).
struct AxionDecision {
  int K;
  float wprod, wnew, om, w;
  bool keep, absorbed, capped, over, abs_c;
};

__device__ __forceinline__ AxionDecision axion_decide(const float* rec, const float* sr, const StepArgs& A, int mask,
                                                      float w, float px, float py, float pz, uint32_t wP,
                                                      uint32_t wA) {
  AxionDecision d;
  d.om = sqrtf((px * px + py * py + pz * pz) + A.mu2) * kMeC2f;  // the total energy E
  d.K = 0;
  d.wprod = 0.f;
  d.capped = false;
  d.over = false;
  d.absorbed = false;
  d.abs_c = false;
  float wrem = w;
  const float xr = d.om * rec[R_INVT];
  const bool use_sr = sr && sr_in_range(xr);
  if (mask & AXPIC_CH_PRIMAKOFF) {
    const float P = use_sr ? -expm1f(-A.cc.prim_mult * sr_prim_gdt(sr, xr))
                           : prim_prob(rec, d.om, A.cc.prim_mult * rec[R_AP]);
    float fac;
    const float le = cap_lambda(w * P * A.inv_w_gref, A.lam_cap, &fac, &d.capped);
    d.K = poisson_inv(u23(wP), le);
    if (d.K > 0) d.wprod = deplete(w, d.K, d.capped ? A.w_gref * fac : A.w_gref, &wrem, &d.over);
  }
  d.keep = wrem > 0.f;
  d.wnew = wrem;
  if (d.keep && (mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS))) {
    const float x = xr;
    const float tc = !(mask & AXPIC_CH_COMPTON) ? 0.f
                     : use_sr                   ? sr_tau(sr, 1, x, A.eq_stats)
                                                : tau_compton(rec, x, A.eq_stats);
    const float tb = !(mask & AXPIC_CH_BREMS) ? 0.f
                     : use_sr                 ? sr_tau(sr, 2, x, A.eq_stats)
                                              : tau_brems(rec, x, A.brems_am3, A.eq_stats);
    const float tau = tc + tb;
    if (A.absorb_mode == 0) {
      const float P = -expm1f(-tau);
      const float u = u23(wA);
      if (u < P) {
        d.absorbed = true;
        d.keep = false;
        d.abs_c = u / P < tc / tau;
      }
    } else {
      d.wnew = wrem * expf(-tau);
      d.keep = d.wnew > 0.f;
    }
  }
  return d;
}

// The spectral record a cell's full decisions and emission energies take
// their rates from: every cell's under the table model, the cells the
// network is not trusted for under the surrogate model; NULL otherwise (the
// closed forms with the cell record's prefactors).
__device__ __forceinline__ const float* cell_sr(const StepArgs& A, int cell) {
  if (A.rate_model == 1 || (A.rate_model == 2 && A.ra.src[cell])) return A.ra.sr + (size_t)cell * kSrLen;
  return nullptr;
}

__device__ __forceinline__ void load_rec(const StepArgs& A, int cell, float* rec) {
  const float4* r4 = reinterpret_cast<const float4*>(A.rec + (size_t)cell * kRecLen);
#pragma unroll
  for (int i = 0; i < kRecLen / 4; ++i) {
    const float4 v = r4[i];
    rec[4 * i] = v.x;
    rec[4 * i + 1] = v.y;
    rec[4 * i + 2] = v.z;
    rec[4 * i + 3] = v.w;
  }
}

// Out-of-line full decisions of slot idx: they load the slot's record and
// the cell's record together (one round trip), so that the caller's cell
// constants stay in registers.
__device__ __noinline__ AxionDecision axion_decide_slow(const StepArgs& A, int cell, int mask, long idx, uint32_t wP,
                                                        uint32_t wA) {
  const float4 v = A.a.wp[idx];
  float rec[kRecLen];
  load_rec(A, cell, rec);
  AxionDecision d = axion_decide(rec, cell_sr(A, cell), A, mask, v.x, v.y, v.z, v.w, wP, wA);
  d.w = v.x;
  return d;
}

// One photon at the start of the step: gamma->a conversion (Sec. II.F,
// Eqs. prim_rate, prim_prob, lambda_P, depletion).
struct PhotonDecision {
  int K;
  float wprod, wrem, om;
  bool capped, over;
};

__device__ __forceinline__ PhotonDecision photon_decide(const float* rec, const float* sr, const StepArgs& A, float w,
                                                        float px, float py, float pz, uint32_t wd) {
  PhotonDecision d;
  const float pm = sqrtf(px * px + py * py + pz * pz);
  d.om = pm * kMeC2f;
  const float xr = d.om * rec[R_INVT];
  // a massive axion: the rate times beta(omega), zero at and below m_a
  const float beta = A.mu > 0.f ? axion_beta(pm, A.mu2) : 1.0f;
  const float P = sr && sr_in_range(xr) ? -expm1f(-(beta * sr_prim_gdt(sr, xr))) : prim_prob(rec, d.om, beta * rec[R_AP]);
  float fac;
  const float le = cap_lambda(w * P * A.inv_w_a, A.lam_cap, &fac, &d.capped);
  d.K = poisson_inv(u23(wd), le);
  d.wrem = w;
  d.wprod = 0.f;
  d.over = false;
  if (d.K > 0) d.wprod = deplete(w, d.K, d.capped ? A.w_a * fac : A.w_a, &d.wrem, &d.over);
  return d;
}

__device__ __noinline__ PhotonDecision photon_decide_slow(const StepArgs& A, int cell, long idx, uint32_t wd) {
  const float4 v = A.g.wp[idx];
  float rec[kRecLen];
  load_rec(A, cell, rec);
  return photon_decide(rec, cell_sr(A, cell), A, v.x, v.y, v.z, v.w, wd);
}

// Guards: cheap upper bounds that prove, without the transcendental chain,
// that a particle has no event this step. Whenever a guard answers true the
// full decision would give the same answer (the bounds carry margins far
// above the binary32 rounding of the full path), so results are unchanged.
//
// Conversion: P = 1 - exp(-A F(s)) <= A F(s) and F(s) <= min(s/2, ln(1+s)),
// so lambda <= w A min(s/2, ln(1+s)) / w_ref = lb, and K = 0 whenever
// u <= 1 - lb <= exp(-lambda).
// A bound at or above the Poisson-mean cap also sends the slot to the full
// decision, so that cap hits are counted exactly.
// kb is the cell's A / w_ref with the margin 1.0001 (times the rate model's
// guard margin) folded in.
__device__ __forceinline__ bool no_conversion(float w, float p2, float c_s, float kb, float u, float lam_cap) {
  const float s = p2 * c_s;
  const float Fb = s < 2.5f ? 0.5f * s : __logf(1.0f + s);
  const float lb = w * kb * Fb;
  return (lb < lam_cap) & (u <= 1.0f - lb - 1e-6f);
}
__device__ __forceinline__ float conversion_kb(float Acoef, float inv_wref, float gm) {
  return Acoef * inv_wref * (1.0001f * gm);
}

// Absorption: P_abs <= tau; x/(1-e^-x) <= 1 + x bounds the Compton-like
// factor, (1 - e^-x) <= 1 the Bose-Einstein one. b_c, b_b: the cell's
// coefficients with the margin 1.001 (times the guard margin) folded in; x
// = |p| m_e c^2 / T from p2 by a reciprocal square root (p2 = 0 gives NaN,
// which clears nothing).
__device__ __forceinline__ bool no_absorption(float b_c, float b_b, const StepArgs& A, int mask, float x, float u) {
  float tb = 0.f;
  if (mask & AXPIC_CH_COMPTON) tb += b_c * x * (1.0f + x);
  if (mask & AXPIC_CH_BREMS) tb += b_b * __expf(A.brems_am3 * __logf(x));
  return u >= tb + 1e-6f;
}

// ---------------------------------------------------------------- feedback
struct RemapOut {
  double applied_E, apx, apy, apz;
  float mW, mPx, mPy, mPz, mU2;
};

// p' = p + (s1 p + b) over the cell's electrons (Eq. affine_map with S = 1 + s1),
// measuring in FP64 what the binary32 momenta actually received.
__device__ __noinline__ RemapOut remap_electrons(const StepArgs& A, long ebase, int ne, float s1, float fbx, float fby,
                                                 float fbz) {
  const int lane = lane_id();
  float aE = 0.f, aPx = 0.f, aPy = 0.f, aPz = 0.f;
  float mW = 0.f, mPx = 0.f, mPy = 0.f, mPz = 0.f, mU2 = 0.f;
  const int nqe = (ne + 3) >> 2;
  // two quads per lane and pass, both loaded before either is stored; each
  // lane still sums its quads in ascending order
  for (int q0 = lane; q0 < nqe; q0 += 64) {
    float4 v[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = q0 + 32 * h;
      if (q < nqe) {
        const long b = ebase + 4 * q;
#pragma unroll
        for (int j = 0; j < 4; ++j) v[h][j] = A.e.wp[b + j];
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = q0 + 32 * h;
      if (q >= nqe) break;
      const long b = ebase + 4 * q;
      const int nj = min(4, ne - 4 * q);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= nj) break;
        const float w = v[h][j].x, px = v[h][j].y, py = v[h][j].z, pz = v[h][j].w;
        const float nx = px + fmaf(s1, px, fbx);
        const float ny = py + fmaf(s1, py, fby);
        const float nz = pz + fmaf(s1, pz, fbz);
        const float ddx = nx - px, ddy = ny - py, ddz = nz - pz;
        aE += w * (ddx * (2.f * px + ddx) + ddy * (2.f * py + ddy) + ddz * (2.f * pz + ddz));
        aPx += w * ddx;
        aPy += w * ddy;
        aPz += w * ddz;
        mW += w;
        mPx += w * nx;
        mPy += w * ny;
        mPz += w * nz;
        mU2 += w * (nx * nx + ny * ny + nz * nz);
        A.e.wp[b + j] = make_float4(w, nx, ny, nz);
      }
    }
  }
  RemapOut o;
  o.applied_E = warp_sum_d((double)aE) * 0.5 * kMeC2;
  o.apx = warp_sum_d((double)aPx);
  o.apy = warp_sum_d((double)aPy);
  o.apz = warp_sum_d((double)aPz);
  o.mW = warp_sum_f(mW);
  o.mPx = warp_sum_f(mPx);
  o.mPy = warp_sum_f(mPy);
  o.mPz = warp_sum_f(mPz);
  o.mU2 = warp_sum_f(mU2);
  return o;
}

__device__ __forceinline__ bool nz64(double v) { return (__double_as_longlong(v) << 1) != 0; }

// ---------------------------------------------------------------- decision records
// A flagged slot's full decision, written by the decision kernels and read by
// the event kernel (slot-indexed arrays, touched only for flagged slots):
// x = K | flags << 8, y = product weight, z = new weight (axions) or the
// remaining weight (photons).
enum : uint32_t {
  DF_KEEP = 1u << 8, DF_ABSORBED = 1u << 9, DF_ABS_C = 1u << 10, DF_CAPPED = 1u << 11, DF_OVER = 1u << 12,
  DF_CAPPED_B = 1u << 13
};

// ---------------------------------------------------------------- decision kernels
// Bit masks: word (cell * W + s / 32), bit s % 32 flags slot s. Words are
// set by atomicOr (rare: electrons whose draw passes, axions and photons
// whose full decision changes something) and cleared by the event kernel
// after reading.

__device__ __forceinline__ void flag_quad(uint32_t* bits, int W, int cell, int q, uint32_t nib) {
  if (nib) atomicOr(bits + (size_t)cell * W + ((4 * q) >> 5), nib << ((4 * q) & 31));
}

// A persistent grid of warps. Warp i owns the chunks i, i + nwarps, ... of
// C consecutive cells and, per chunk and species, gives the chunk's quads
// to its lanes as one flat range (lane per quad, cell-major), so uneven counts
// still fill the lanes. Slots that the guards cannot clear go to the warp's
// own list in shared memory, which carries over from chunk to chunk and is
// decided 32 at a time: the out-of-line chain runs with full lanes and no CTA
// barrier is needed. List order does not matter: records are indexed by slot.
constexpr int kDecThreads = 256;
constexpr int kDecWarps = kDecThreads / 32;
// Cells per chunk: a launch-shape choice (4, 8, 16 or 32), picked per context. With
// 32 every lane holds one cell's constants.
constexpr int kChunkDefault = AXPIC_DEC_CHUNK;
static_assert(kChunkDefault == 4 || kChunkDefault == 8 || kChunkDefault == 16 || kChunkDefault == 32,
              "cells per decision chunk");
constexpr int kListCap = 32 + 4 * 32;  // < 32 pending + one pass of flags

// Per-warp lists: {cell, slot, decision word(s)}.
struct DecLists {
  uint4 a[kDecWarps][kListCap];
  uint4 g[kDecWarps][kListCap];
};

// Flat quad range of a chunk: lanes < nc hold their cell's slot count n; on
// return lanes < nc hold their cell's first quad (qoff; the lanes beyond
// hold INT_MAX) and every lane the total. The starts stay in the lanes: a
// quad's cell is found by shuffles, which keeps the per-chunk state to two
// registers.
template <int C>
struct QuadRange {
  int qoff, total;
};

template <int C>
__device__ __forceinline__ QuadRange<C> quad_range(int n, int lane, int nc) {
  QuadRange<C> R;
  const int nq = lane < nc ? (n + 3) >> 2 : 0;
  R.qoff = warp_excl_scan(nq, &R.total);
  if (lane >= nc) R.qoff = 0x7fffffff;
  return R;
}

// Cell (in the chunk) of flat quad g: the last cell whose first quad is at
// or before g (binary search over the lanes' starts).
template <int C>
__device__ __forceinline__ int quad_cell(const QuadRange<C>& R, int g) {
  int lc = 0;
#pragma unroll
  for (int s = C / 2; s >= 1; s >>= 1) lc += g >= __shfl_sync(kFull, R.qoff, lc + s) ? s : 0;
  return lc;
}

// Appends this lane's flagged slots (bits of nib; words w0/w1 rotate with the
// slot) to a warp list of current length pend; returns the new length.
__device__ __forceinline__ int list_append(uint4* L, int pend, int cell, int slot0, uint32_t nib, uint4 w0, uint4 w1) {
  if (!__any_sync(kFull, nib != 0)) return pend;  // the common pass: nothing flagged
  int tot;
  int o = pend + warp_excl_scan(__popc(nib), &tot);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if ((nib >> j) & 1u) L[o++] = make_uint4((uint32_t)cell, (uint32_t)(slot0 + j), word(w0, j), word(w1, j));
  __syncwarp();
  return pend + tot;
}

// A full decision that changes nothing (no event, no cap hit, weight kept
// unchanged) leaves its slot unflagged: the event kernel never sees it.
__device__ __forceinline__ void axion_full(const StepArgs& A, uint4 it) {
  const int cell = (int)it.x;
  const long idx = (long)cell * A.a.cap + it.y;
  const AxionDecision d = axion_decide_slow(A, cell, A.mask, idx, it.z, it.w);
  const float w = d.w;
  uint32_t f = (uint32_t)d.K;
  if (d.keep) f |= DF_KEEP;
  if (d.absorbed) f |= DF_ABSORBED;
  if (d.abs_c) f |= DF_ABS_C;
  if (d.capped) f |= DF_CAPPED;
  if (d.over) f |= DF_OVER;
  const bool reduce = A.absorb_mode == 1 && (A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS));
  if (f == DF_KEEP && d.wnew == w && !reduce) return;
  A.recA[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wnew), 0u);
  atomicOr(A.bitsA + (size_t)cell * A.Wa + (it.y >> 5), 1u << (it.y & 31));
}

__device__ __forceinline__ void photon_full(const StepArgs& A, uint4 it) {
  const int cell = (int)it.x;
  const long idx = (long)cell * A.g.cap + it.y;
  const PhotonDecision d = photon_decide_slow(A, cell, idx, it.z);
  uint32_t f = (uint32_t)d.K;
  if (d.wrem > 0.f) f |= DF_KEEP;
  if (d.capped) f |= DF_CAPPED;
  if (d.over) f |= DF_OVER;
  if (f == DF_KEEP) return;
  A.recG[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wrem), 0u);
  atomicOr(A.bitsG + (size_t)cell * A.Wg + (it.y >> 5), 1u << (it.y & 31));
}

// Decides full batches of 32 from the top of a list; returns what is left.
template <bool AX>
__device__ __forceinline__ int list_drain(const StepArgs& A, const uint4* L, int pend, int lane) {
  while (pend >= 32) {
    pend -= 32;
    const uint4 it = L[pend + lane];
    if (AX) axion_full(A, it);
    else photon_full(A, it);
  }
  __syncwarp();
  return pend;
}

// Electrons of a chunk (thermal-bath emission). With a common weight the
// decision is u > exp(-lambda) with lambda shared by the cell; the full
// decision of a flagged electron is a short Poisson inversion, taken here.
template <int C>
__device__ __forceinline__ void electron_chunk(const StepArgs& A, uint32_t step, int c0, int nc, int lane) {
  const int mask = A.mask;
  const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
  int n = 0, thr = 0;
  float wu = 0.f, lsum = 0.f, rcc = 0.f, rcb = 0.f;
  if (lane < nc) {
    const int c = c0 + lane;
    const float* rec = A.rec + (size_t)c * kRecLen;
    n = min(max(A.e.count[c], 0), A.e.cap);
    rcc = __ldg(rec + R_CC);
    rcb = __ldg(rec + R_CB);
    wu = __ldg(A.mom + (size_t)c * kMomLen + M_WU);
    if (wu > 0.f) {
      float fac;
      bool cc = false, cb = false;
      const float lc = eC ? cap_lambda(wu * rcc, A.lam_cap, &fac, &cc) : 0.f;
      const float lb = eB ? cap_lambda(wu * rcb, A.lam_cap, &fac, &cb) : 0.f;
      lsum = lc + lb;
      // every electron of the cell has the capped mean (rare: counted here,
      // where the cap is found)
      if (cc || cb)
        atomicAdd(A.counters + (size_t)(blockIdx.x % A.ctr_rows) * kNumCounters + C_CAP,
                  (unsigned long long)n * ((unsigned)cc + (unsigned)cb));
      // u23(w) > F0 exactly when (w >> 9) > floor(F0 2^23 - 1/2): the
      // scaling and the subtraction are exact in binary32
      thr = (int)floorf(__fsub_rn(__fmul_rn(expf(-lsum), 8388608.0f), 0.5f));
    }
  }
  if (__all_sync(kFull, lane >= nc || (wu > 0.f && (((n + 3) >> 2) & 63) == 0))) {
    // every cell of the chunk has a common weight and whole passes of 64
    // quads: cell by cell, two quads per lane and pass (two independent
    // Philox chains in flight), the decision the integer compare alone
    for (int lc = 0; lc < nc; ++lc) {
      const int nn = __shfl_sync(kFull, n, lc);
      const int cthr = __shfl_sync(kFull, thr, lc);
      const float cls = __shfl_sync(kFull, lsum, lc);
      const int cell = c0 + lc;
      const uint32_t gcell = A.cell_base + (uint32_t)cell;
      const long cb = (long)cell * A.e.cap;
      const int nq = (nn + 3) >> 2;
      for (int q0 = 0; q0 < nq; q0 += 64) {
        uint4 r[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
          r[h] = philox4x32_10(make_uint4(step, gcell, (uint32_t)(q0 + 32 * h + lane), S_EMIT_E << 24), A.rk);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = q0 + 32 * h + lane;
          const uint32_t m = max(max(r[h].x, r[h].y), max(r[h].z, r[h].w));
          if ((int)(m >> 9) <= cthr) continue;  // no slot of the quad emits
          const int nj = min(4, nn - 4 * q);
          uint32_t nib = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t wj = word(r[h], j);
            if (j < nj && (int)(wj >> 9) > cthr) {
              A.recE[cb + 4 * q + j] = (uint32_t)poisson_inv(u23(wj), cls);
              nib |= 1u << j;
            }
          }
          flag_quad(A.bitsE, A.We, cell, q, nib);
        }
      }
    }
    return;
  }
  const QuadRange<C> R = quad_range<C>(n, lane, nc);
  if (__all_sync(kFull, lane >= nc || wu > 0.f)) {
    // every cell of the chunk has a common weight: the decision is the
    // integer compare alone. Two quads per lane and pass, so that two
    // independent Philox chains are in flight.
    for (int g0 = 0; g0 < R.total; g0 += 64) {
      int lc[2], q[2];
      uint4 r[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        lc[h] = quad_cell(R, g0 + 32 * h + lane);
        q[h] = g0 + 32 * h + lane - __shfl_sync(kFull, R.qoff, lc[h]);
        r[h] = philox4x32_10(make_uint4(step, A.cell_base + (uint32_t)(c0 + lc[h]), (uint32_t)q[h], S_EMIT_E << 24), A.rk);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int nn = __shfl_sync(kFull, n, lc[h]);
        const int cthr = __shfl_sync(kFull, thr, lc[h]);
        const float cls = __shfl_sync(kFull, lsum, lc[h]);
        const uint32_t m = max(max(r[h].x, r[h].y), max(r[h].z, r[h].w));
        if (g0 + 32 * h + lane >= R.total || (int)(m >> 9) <= cthr) continue;  // no slot of the quad emits
        const int cell = c0 + lc[h];
        const int nj = min(4, nn - 4 * q[h]);
        const long b = (long)cell * A.e.cap + 4 * q[h];
        uint32_t nib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t wj = word(r[h], j);
          if (j < nj && (int)(wj >> 9) > cthr) {
            A.recE[b + j] = (uint32_t)poisson_inv(u23(wj), cls);
            nib |= 1u << j;
          }
        }
        flag_quad(A.bitsE, A.We, cell, q[h], nib);
      }
    }
    return;
  }
  for (int g0 = 0; g0 < R.total; g0 += 32) {
    const int g = g0 + lane;
    const int lc = quad_cell(R, g);
    const int qb = __shfl_sync(kFull, R.qoff, lc);
    const int nn = __shfl_sync(kFull, n, lc);
    const float cwu = __shfl_sync(kFull, wu, lc);
    const int cthr = __shfl_sync(kFull, thr, lc);
    const float cls = __shfl_sync(kFull, lsum, lc);
    const float ccc = __shfl_sync(kFull, rcc, lc);
    const float ccb = __shfl_sync(kFull, rcb, lc);
    if (g >= R.total) continue;
    const int cell = c0 + lc;
    const int q = g - qb;
    const int nj = min(4, nn - 4 * q);
    const uint4 r = philox4x32_10(make_uint4(step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_EMIT_E << 24), A.rk);
    const long b = (long)cell * A.e.cap + 4 * q;
    uint32_t nib = 0;
    if (cwu > 0.f) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t wj = word(r, j);
        if (j < nj && (int)(wj >> 9) > cthr) {
          A.recE[b + j] = (uint32_t)poisson_inv(u23(wj), cls);
          nib |= 1u << j;
        }
      }
    } else {
      const float rsum = ((eC ? ccc : 0.f) + (eB ? ccb : 0.f)) * 1.0001f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float wj = slot_w(A.e, b + j);
        const float lbnd = wj * rsum;
        if (j < nj && !(lbnd < A.lam_cap && u23(word(r, j)) <= 1.0f - lbnd - 1e-6f)) {
          float fac;
          bool cc = false, cb = false;
          const float l1 = eC ? cap_lambda(wj * ccc, A.lam_cap, &fac, &cc) : 0.f;
          const float l2 = eB ? cap_lambda(wj * ccb, A.lam_cap, &fac, &cb) : 0.f;
          uint32_t f = (uint32_t)poisson_inv(u23(word(r, j)), l1 + l2);
          if (cc) f |= DF_CAPPED;
          if (cb) f |= DF_CAPPED_B;
          A.recE[b + j] = f;
          nib |= 1u << j;
        }
      }
    }
    flag_quad(A.bitsE, A.We, cell, q, nib);
  }
}

// Photons of a chunk present at the start of the step (gamma->a).
template <int C>
__device__ __forceinline__ int photon_chunk(const StepArgs& A, uint32_t step, int c0, int nc, int lane, uint4* L,
                                            int pend) {
  int n = 0;
  float c_s = 0.f, ap = 0.f;
  if (lane < nc) {
    const int c = c0 + lane;
    const float* rec = A.rec + (size_t)c * kRecLen;
    const int cnt = min(max(A.g.count[c], 0), A.g.cap);
    n = A.use_snapshot ? min(A.photon_start[c], cnt) : cnt;
    c_s = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    ap = conversion_kb(__ldg(rec + R_AP), A.inv_w_a, A.guard_margin);
  }
  const QuadRange<C> R = quad_range<C>(n, lane, nc);
  for (int g0 = 0; g0 < R.total; g0 += 32) {
    const int g = g0 + lane;
    const int lc = quad_cell(R, g);
    const int qb = __shfl_sync(kFull, R.qoff, lc);
    const int nn = __shfl_sync(kFull, n, lc);
    const float cs = __shfl_sync(kFull, c_s, lc);
    const float ca = __shfl_sync(kFull, ap, lc);
    const int cell = c0 + lc;
    const int q = g - qb;
    uint32_t nib = 0;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (g < R.total) {
      const int nj = min(4, nn - 4 * q);
      const long b = (long)cell * A.g.cap + 4 * q;
      float4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = A.g.wp[b + j];
      r = philox4x32_10(make_uint4(step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_PRIM_FWD << 24), A.rk);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float px = v[j].y, py = v[j].z, pz = v[j].w;
        const float p2 = px * px + py * py + pz * pz;
        nib |= (uint32_t)((j < nj) & !no_conversion(v[j].x, p2, cs, ca, u23(word(r, j)), A.lam_cap)) << j;
      }
    }
    pend = list_append(L, pend, cell, 4 * q, nib, r, r);
    pend = list_drain<false>(A, L, pend, lane);
  }
  return pend;
}

// Axions of a chunk present at the start of the step: a->gamma and absorption.
template <int C>
__device__ __forceinline__ int axion_chunk(const StepArgs& A, uint32_t step, int c0, int nc, int lane, uint4* L,
                                           int pend) {
  const int mask = A.mask;
  const bool prim = mask & AXPIC_CH_PRIMAKOFF;
  const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const bool all = A.absorb_mode == 1 && bath;  // weight reduction changes every axion
  int n = 0;
  float c_s = 0.f, apinv = 0.f, invT = 0.f, r_bc = 0.f, r_bb = 0.f;
  if (lane < nc) {
    const int c = c0 + lane;
    const float* rec = A.rec + (size_t)c * kRecLen;
    n = min(max(A.a.count[c], 0), A.a.cap);
    c_s = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    apinv = conversion_kb(A.cc.prim_mult * __ldg(rec + R_AP), A.inv_w_gref, A.guard_margin);
    invT = kMeC2f * __ldg(rec + R_INVT);
    r_bc = __ldg(rec + R_BC) * (1.001f * A.guard_margin);
    r_bb = __ldg(rec + R_BB) * (1.001f * A.guard_margin);
  }
  const QuadRange<C> R = quad_range<C>(n, lane, nc);
  for (int g0 = 0; g0 < R.total; g0 += 32) {
    const int g = g0 + lane;
    const int lc = quad_cell(R, g);
    const int qb = __shfl_sync(kFull, R.qoff, lc);
    const int nn = __shfl_sync(kFull, n, lc);
    const float cs = __shfl_sync(kFull, c_s, lc);
    const float cap_inv = __shfl_sync(kFull, apinv, lc);
    const float cinvT = __shfl_sync(kFull, invT, lc);
    const float cbc = __shfl_sync(kFull, r_bc, lc);
    const float cbb = __shfl_sync(kFull, r_bb, lc);
    const int cell = c0 + lc;
    const int q = g - qb;
    uint32_t nib = 0;
    uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
    if (g < R.total) {
      const int nj = min(4, nn - 4 * q);
      const uint32_t gcell = A.cell_base + (uint32_t)cell;
      const long b = (long)cell * A.a.cap + 4 * q;
      if (prim) rP = philox4x32_10(make_uint4(step, gcell, (uint32_t)q, S_PRIM_INV << 24), A.rk);
      if (bath) rA = philox4x32_10(make_uint4(step, gcell, (uint32_t)q, S_ABSORB << 24), A.rk);
      float4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = A.a.wp[b + j];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float px = v[j].y, py = v[j].z, pz = v[j].w;
        const float p2 = (px * px + py * py + pz * pz) + A.mu2;  // E^2 (m_e c^2 units)
        bool fast = !all;
        if (prim) fast &= no_conversion(v[j].x, p2, cs, cap_inv, u23(word(rP, j)), A.lam_cap);
        if (bath) fast &= no_absorption(cbc, cbb, A, mask, p2 * rsqrtf(p2) * cinvT, u23(word(rA, j)));
        nib |= (uint32_t)((j < nj) & !fast) << j;
      }
    }
    pend = list_append(L, pend, cell, 4 * q, nib, rP, rA);
    pend = list_drain<true>(A, L, pend, lane);
  }
  return pend;
}

// All decisions of a call in one launch. The photon decisions read the
// photons present at the start of the step: the absorb phase appends a->gamma
// products only in the event kernel.
enum : int { DK_ELECTRON = 1, DK_PHOTON = 2, DK_AXION = 4 };

#ifndef AXPIC_DEC_MIN_CTAS
#define AXPIC_DEC_MIN_CTAS 4
#endif

// The step index of this call: from the device counter when the step runs
// inside a replayed graph, else the launch argument.
__device__ __forceinline__ uint32_t step_of(const StepArgs& A) { return A.step_dev ? *A.step_dev : A.step; }

template <int C>
__global__ void __launch_bounds__(kDecThreads, AXPIC_DEC_MIN_CTAS) decide_kernel(StepArgs A, int kinds) {
  __shared__ DecLists L;
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  const uint32_t step = step_of(A);
  const int nwarps = gridDim.x * kDecWarps;
  const int nchunks = (A.ncells + C - 1) / C;
  const int cend = A.cell0 + A.ncells;
  int pa = 0, pg = 0;
  for (int ch = blockIdx.x * kDecWarps + wid; ch < nchunks; ch += nwarps) {
    const int c0 = A.cell0 + ch * C;
    const int nc = min(C, cend - c0);
    if (kinds & DK_ELECTRON) electron_chunk<C>(A, step, c0, nc, lane);
    if (kinds & DK_PHOTON) pg = photon_chunk<C>(A, step, c0, nc, lane, L.g[wid], pg);
    if (kinds & DK_AXION) pa = axion_chunk<C>(A, step, c0, nc, lane, L.a[wid], pa);
  }
  if (lane < pg) photon_full(A, L.g[wid][lane]);
  if (lane < pa) axion_full(A, L.a[wid][lane]);
}

// ---------------------------------------------------------------- feedback kernel
// Per cell: the exchange of this step plus the carried part; when it is
// representable in binary32 momenta the cell's electrons get the affine remap
// (Eqs. delta_def to b_def, affine_map) by a whole warp, measuring what was
// applied; then the temperature update (Eqs. Te_est, Te_relax) and the
// record's temperature half.

struct FbCell {
  double dE, dPx, dPy, dPz;  // this step's exchange
  double rE, rPx, rPy, rPz;  // carried exchange
  double T;
  double qE, qPx, qPy, qPz, s1d, bx, by, bz, vnd;
  float W, Px, Py, Pz, U2, var;
  float4 rc[4];
  int ne;
  bool has_x, has_res, need;
};

// What the feedback of a cell reads besides the exchange.
__device__ __forceinline__ void fb_load(const StepArgs& A, int cell, FbCell& f) {
  const double* rs = A.res + (size_t)cell * 4;
  f.rE = rs[0];
  f.rPx = rs[1];
  f.rPy = rs[2];
  f.rPz = rs[3];
  const float* mom = A.mom + (size_t)cell * kMomLen;
  f.W = mom[M_W];
  f.Px = mom[M_PX];
  f.Py = mom[M_PY];
  f.Pz = mom[M_PZ];
  f.U2 = mom[M_U2];
  f.var = mom[M_VAR];
  f.ne = min(max(A.e.count[cell], 0), A.e.cap);
  f.T = 0.0;
  f.rc[0] = f.rc[1] = f.rc[2] = f.rc[3] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (A.T_mode == 2) {
    f.T = A.T[cell];
    const float4* r4 = reinterpret_cast<const float4*>(A.rec + (size_t)cell * kRecLen);
    f.rc[0] = r4[0];
    f.rc[1] = r4[1];
    f.rc[2] = r4[2];
    f.rc[3] = r4[3];
  }
}

// The pending exchange and, when it needs a remap now, the map's s - 1 and b.
__device__ __forceinline__ void fb_prepare(FbCell& f) {
  f.has_x = nz64(f.dE) || nz64(f.dPx) || nz64(f.dPy) || nz64(f.dPz);
  f.has_res = nz64(f.rE) || nz64(f.rPx) || nz64(f.rPy) || nz64(f.rPz);
  f.need = false;
  f.qE = f.qPx = f.qPy = f.qPz = f.s1d = f.bx = f.by = f.bz = f.vnd = 0.0;
  if (!(f.has_x || f.has_res)) return;
  f.qE = f.dE + f.rE;
  f.qPx = f.dPx + f.rPx;
  f.qPy = f.dPy + f.rPy;
  f.qPz = f.dPz + f.rPz;
  // Exchanges below 2^-22 of the cell's kinetic energy (or momentum spread)
  // cannot be represented by binary32 momenta; they stay pending.
  const float ekin = 0.5f * f.U2 * kMeC2f;
  const float prms = sqrtf(fmaxf(f.U2 * f.W, 0.f));
  f.need = f.W > 0.f && (fabsf((float)f.qE) >= 2.384185791015625e-07f * ekin ||
                         sqrtf((float)(f.qPx * f.qPx + f.qPy * f.qPy + f.qPz * f.qPz)) >=
                             2.384185791015625e-07f * prms);
  if (!f.need) return;
  // Eqs. delta_def, dE_bulk, dE_th, var_new, s_def, b_def (mu = 1). Three
  // FP64 divisions and one square root (FP64 runs at a small fraction of the
  // FP32 rate): 1/W once, and S - 1 = t / (S + 1) with t = var_new / var - 1
  // formed from 2 dE_th without cancellation.
  const double Wd = f.W;
  const double iW = 1.0 / Wd;
  const double dx = f.qPx * iW, dy = f.qPy * iW, dz = f.qPz * iW;
  const double dEb = (2.0 * (dx * f.Px + dy * f.Py + dz * f.Pz) + Wd * (dx * dx + dy * dy + dz * dz)) * 0.5;
  const double dEth = f.qE * (1.0 / kMeC2) - dEb;
  f.vnd = f.var;
  if (f.var > 0.f) {
    const double var = f.var;
    f.vnd = fmax(0.0, var + 2.0 * dEth);
    const double t = (f.vnd > 0.0 ? 2.0 * dEth : -var) / var;
    const double S = sqrt(1.0 + t);
    f.s1d = t / (S + 1.0);
  }
  f.bx = -f.s1d * f.Px * iW + dx;
  f.by = -f.s1d * f.Py * iW + dy;
  f.bz = -f.s1d * f.Pz * iW + dz;
}

// Carry, moments, diagnostics, temperature and record once the remap (r;
// null when the cell was not remapped) is done. The record gets the
// closed-form prefactors of the new temperature; under the surrogate rate
// model the network's kernel, launched next, replaces them where it is
// trusted.
__device__ __forceinline__ void fb_finish(const StepArgs& A, int cell, const FbCell& f, const RemapOut* r) {
  double nrE = f.qE, nrPx = f.qPx, nrPy = f.qPy, nrPz = f.qPz, applied_E = 0.0;
  float var_new = f.var;
  if (r) {
    applied_E = r->applied_E;
    nrE = f.qE - r->applied_E;
    nrPx = f.qPx - r->apx;
    nrPy = f.qPy - r->apy;
    nrPz = f.qPz - r->apz;
    var_new = (float)f.vnd;
    float* mom = A.mom + (size_t)cell * kMomLen;
    mom[M_W] = r->mW;
    mom[M_PX] = r->mPx;
    mom[M_PY] = r->mPy;
    mom[M_PZ] = r->mPz;
    mom[M_U2] = r->mU2;
    mom[M_VAR] = fmaxf(0.f, r->mU2 - (r->mPx * r->mPx + r->mPy * r->mPy + r->mPz * r->mPz) / r->mW);
  }
  if (f.has_x || f.has_res) {
    double* rs = A.res + (size_t)cell * 4;
    rs[0] = nrE;
    rs[1] = nrPx;
    rs[2] = nrPy;
    rs[3] = nrPz;
  }
  if (A.diag_enable) {
    double* dg = A.diag + (size_t)cell * AXPIC_CELL_DIAG_LEN;
    dg[AXPIC_CD_DE] = f.dE;
    dg[AXPIC_CD_DPX] = f.dPx;
    dg[AXPIC_CD_DPY] = f.dPy;
    dg[AXPIC_CD_DPZ] = f.dPz;
    dg[AXPIC_CD_S_MINUS_1] = f.s1d;
    dg[AXPIC_CD_BX] = f.bx;
    dg[AXPIC_CD_BY] = f.by;
    dg[AXPIC_CD_BZ] = f.bz;
    dg[AXPIC_CD_VAR] = f.var;
    dg[AXPIC_CD_VAR_NEW] = f.need ? f.vnd : (double)f.var;
    dg[AXPIC_CD_W] = f.W;
    dg[AXPIC_CD_APPLIED_E] = applied_E;
    dg[AXPIC_CD_RES_E] = f.has_x || f.has_res ? nrE : 0.0;
    dg[AXPIC_CD_RES_PX] = f.has_x || f.has_res ? nrPx : 0.0;
    dg[AXPIC_CD_RES_PY] = f.has_x || f.has_res ? nrPy : 0.0;
    dg[AXPIC_CD_RES_PZ] = f.has_x || f.has_res ? nrPz : 0.0;
  }
  // temperature (Eqs. Te_est, Te_relax), then the record's temperature half;
  // T stays FP64, the relaxation step is formed in binary32 and added once
  if (A.T_mode == 2 && f.W > 0.f) {
    const float Tf = (float)f.T;
    const float Test = (kMeC2f / 3.0f) * var_new / f.W;
    const float dT = A.relax_r * (Test - Tf);
    double Tn = f.T + (double)dT;
    const float Tnf = Tf + dT;
    if (Tnf <= A.T_floor_f || Tnf >= A.T_ceil_f) Tn = fmin(fmax(Tn, A.T_floor), A.T_ceil);
    float rec[kRecLen];
    const float4* rc = f.rc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      rec[4 * i] = rc[i].x;
      rec[4 * i + 1] = rc[i].y;
      rec[4 * i + 2] = rc[i].z;
      rec[4 * i + 3] = rc[i].w;
    }
    compute_temperature(A.cc, (float)Tn, rec);
    A.T[cell] = Tn;
    // the closed-form Primakoff prefactor (the network's may be there)
    if (A.rate_model == 2) rec[R_AP] = A.cc.k_AP * rec[R_SZ];
    float4* r4 = reinterpret_cast<float4*>(A.rec + (size_t)cell * kRecLen);
    r4[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
    r4[1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
  }
}

// Thread per cell, every load issued first; a warp remaps the cells among
// its 32 whose exchange needs an affine remap, one at a time with all lanes
// (about one warp in twelve has one), then each thread finishes its cell. No
// CTA barrier: the warps of a CTA never wait for one another's remaps. Five
// CTAs an SM (96 registers; the remap path spills a little).
constexpr int kFeedbackThreads = 128;

__global__ void __launch_bounds__(kFeedbackThreads, 5) feedback_kernel(StepArgs A) {
  // a replayed graph takes its step index from the device counter: the last
  // kernel of the step advances it (no kernel of this launch reads it)
  if (A.step_dev && blockIdx.x == 0 && threadIdx.x == 0) *A.step_dev += 1u;
  const int lane = threadIdx.x & 31;
  const int cell = A.cell0 + blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < A.cell0 + A.ncells;
  FbCell f = {};
  if (valid) {
    double* xb = A.xbuf + (size_t)cell * 4;
    f.dE = xb[0];
    f.dPx = xb[1];
    f.dPy = xb[2];
    f.dPz = xb[3];
    fb_load(A, cell, f);
    fb_prepare(f);
    if (f.has_x) {
      xb[0] = 0.0;
      xb[1] = 0.0;
      xb[2] = 0.0;
      xb[3] = 0.0;
    }
  }
  // the warp remaps its cells that need it one by one, all lanes together
  RemapOut mine;
  for (unsigned m = __ballot_sync(kFull, f.need); m; m &= m - 1u) {
    const int j = __ffs(m) - 1;
    const int c = __shfl_sync(kFull, cell, j);
    const RemapOut r = remap_electrons(A, (long)c * A.e.cap, __shfl_sync(kFull, f.ne, j),
                                       __shfl_sync(kFull, (float)f.s1d, j), __shfl_sync(kFull, (float)f.bx, j),
                                       __shfl_sync(kFull, (float)f.by, j), __shfl_sync(kFull, (float)f.bz, j));
    if (lane == j) mine = r;
  }
  if (valid) {
    fb_finish(A, cell, f, f.need ? &mine : nullptr);
    if (f.need) {
      atomicAdd(A.counters + C_REMAP, 1ull);
      atomicAdd(A.counters + C_REMAP_E, (unsigned long long)f.ne);
    }
  }
}


// ---------------------------------------------------------------- event kernel
// Warp w takes cells [32 w, 32 w + 32), lane l cell 32 w + l. Most cells
// have a handful of flagged slots: the lane then takes the cell alone, so the
// per-cell scans, counts and stores are shared by 32 cells per instruction.
// A cell with more flagged slots in a phase than a lane takes is done by the
// whole warp for that phase.
//
// Per-warp shared scratch:
//   flagged-slot lists of one heavy cell (u16, full capacities; the removed
//   lists reuse them) and its removed-slot bits;
//   the lanes' lists: kLight entries per species and lane, entry i of lane l
//   at [32 i + l] (the removed list reuses it in place);
//   the 32 cells' mask rows, copied in by cp.async (row stride W | 1 words,
//   so that lanes reading their own rows hit distinct banks).

// Flagged slots per species up to which one lane takes a cell's phase
// (electrons: kLightE, each event with its own Philox block).
constexpr int kLight = 8;
constexpr int kLightE = 4;
// Flagged slots and tail movers per species whose loads go out together
// (one: more in flight cost registers, and occupancy gained more).
constexpr int kLoad = 1;
constexpr size_t kLaneListBytes = 3 * kLight * 32 * sizeof(uint16_t);

struct EvScratch {
  uint16_t *flA, *flG, *flE, *rmA, *rmG;
  uint32_t *rbA, *rbG;
  uint16_t* lt;
  uint32_t *rowA, *rowG, *rowE;  // null when some row is longer than 32 words
  double2* xs;                    // the lanes' exchange buffers, copied in by cp.async
  int sA, sG, sE;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline int row_words(int cap) { return (cap + 31) / 32; }
__host__ __device__ inline bool rows_staged(int acap, int gcap, int ecap) {
  return row_words(acap) <= 32 && row_words(gcap) <= 32 && row_words(ecap) <= 32;
}

__host__ __device__ inline size_t ev_scratch_bytes(int acap, int gcap, int ecap) {
  size_t b = align16(2 * ((size_t)acap + (size_t)gcap + (size_t)ecap));
  b = align16(b + 4 * (size_t)(row_words(acap) + row_words(gcap)));
  b += kLaneListBytes;
  if (rows_staged(acap, gcap, ecap))
    b += align16(4 * 32 * (size_t)((row_words(acap) | 1) + (row_words(gcap) | 1) + (row_words(ecap) | 1)));
  return b + 32 * 2 * sizeof(double2);
}

__device__ inline EvScratch ev_carve(unsigned char* base, int acap, int gcap, int ecap) {
  EvScratch s;
  uint16_t* h = reinterpret_cast<uint16_t*>(base);
  s.flA = h; h += acap;
  s.flG = h; h += gcap;
  s.flE = h; h += ecap;
  s.rmA = s.flA;
  s.rmG = s.flG;
  size_t off = align16(2 * ((size_t)acap + gcap + ecap));
  uint32_t* u = reinterpret_cast<uint32_t*>(base + off);
  s.rbA = u; u += row_words(acap);
  s.rbG = u;
  off = align16(off + 4 * (size_t)(row_words(acap) + row_words(gcap)));
  s.lt = reinterpret_cast<uint16_t*>(base + off);
  off += kLaneListBytes;
  s.sA = row_words(acap) | 1;
  s.sG = row_words(gcap) | 1;
  s.sE = row_words(ecap) | 1;
  if (rows_staged(acap, gcap, ecap)) {
    s.rowA = reinterpret_cast<uint32_t*>(base + off);
    s.rowG = s.rowA + 32 * s.sA;
    s.rowE = s.rowG + 32 * s.sG;
    off += align16(4 * 32 * (size_t)(s.sA + s.sG + s.sE));
  } else {
    s.rowA = s.rowG = s.rowE = nullptr;
  }
  s.xs = reinterpret_cast<double2*>(base + off);
  return s;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// Waits for this thread's copies; the warp then synchronises to see all.
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Turns one bit-mask word per lane (words [w0, w0 + 32) of a row covering
// [0, n)) into the ascending list of flagged slots; returns the new length.
__device__ __forceinline__ int list_flags(uint32_t v, int wi, int nw, int n, uint16_t* list, int total) {
  if (wi == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;  // bits beyond n never count
  int tot;
  int at = total + warp_excl_scan(__popc(v), &tot);
  while (v) {
    const int bpos = __ffs(v) - 1;
    v &= v - 1u;
    list[at++] = (uint16_t)(32 * wi + bpos);
  }
  return total + tot;
}

// Writes the flagged slots of a mask row covering [0, n) to `list` in
// ascending order (warp-wide) and returns their number. The row is the
// staged copy, or the global row itself, which is then cleared (clr).
__device__ __noinline__ int gather_row(const uint32_t* row, uint32_t* clr, int n, uint16_t* list) {
  const int lane = lane_id();
  const int nw = (n + 31) >> 5;
  int total = 0;
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int wi = w0 + lane;
    const uint32_t v = wi < nw ? row[wi] : 0u;
    if (clr && v) clr[wi] = 0u;
    total = list_flags(v, wi, nw, n, list, total);
  }
  return total;
}

// Tail fill by the warp with the ascending removed list: holes are the
// removed slots below n_surv, movers the kept slots at or beyond it, matched
// in order.
__device__ __noinline__ void compact_tail(const SpeciesPtrs& s, long base, const uint16_t* rm, const uint32_t* rb,
                                          int n_surv, int n) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  int run = 0;
  for (int b0 = n_surv; b0 < n; b0 += 32) {
    const int i = b0 + lane;
    const bool mv = i < n && !bit(rb, i);
    const unsigned m = __ballot_sync(kFull, mv);
    if (mv) {
      const long src = base + i;
      const long dst = base + rm[run + __popc(m & lt)];
      s.wp[dst] = s.wp[src];
      s.xyz[dst] = s.xyz[src];
    }
    run += __popc(m);
  }
}

// A flagged slot with its decision record and the fields its outcome may
// need, loaded in one round trip.
struct AxItem {
  uint4 r;
  float w, px, py, pz, x, y, z;
  int slot;
};
struct PhItem {
  uint4 r;
  float px, py, pz, x, y, z;
  int slot;
};
struct ElItem {
  uint32_t f;
  float w, x, y, z;
  int slot;
};

__device__ __forceinline__ AxItem ax_load(const StepArgs& A, long base, int slot) {
  AxItem t;
  t.slot = slot;
  t.r = make_uint4(0, 0, 0, 0);
  t.w = t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (slot >= 0) {
    const long src = base + slot;
    t.r = A.recA[src];
    const float4 v = A.a.wp[src];
    t.w = v.x;
    t.px = v.y;
    t.py = v.z;
    t.pz = v.w;
    const float4 r = A.a.xyz[src];
    t.x = r.x;
    t.y = r.y;
    t.z = r.z;
  }
  return t;
}

__device__ __forceinline__ PhItem ph_load(const StepArgs& A, long base, int slot) {
  PhItem t;
  t.slot = slot;
  t.r = make_uint4(0, 0, 0, 0);
  t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (slot >= 0) {
    const long src = base + slot;
    t.r = A.recG[src];
    const float4 v = A.g.wp[src];
    t.px = v.y;
    t.py = v.z;
    t.pz = v.w;
    const float4 r = A.g.xyz[src];
    t.x = r.x;
    t.y = r.y;
    t.z = r.z;
  }
  return t;
}

__device__ __forceinline__ ElItem el_load(const StepArgs& A, long base, int slot, float wu) {
  ElItem t;
  t.slot = slot;
  t.f = 0u;
  t.w = wu;
  t.x = t.y = t.z = 0.f;
  if (slot >= 0) {
    const long src = base + slot;
    t.f = A.recE[src];
    const float4 r = A.e.xyz[src];
    t.x = r.x;
    t.y = r.y;
    t.z = r.z;
    if (wu <= 0.f) t.w = slot_w(A.e, src);
  }
  return t;
}

// ---------------------------------------------------------------- per-slot outcomes
// Shared by the lane and warp paths. Output order is the method's: photon
// products of a->gamma after the photons present, axion products of gamma->a
// after the surviving axions, then the thermal-bath products in electron then
// event order; removed slots are refilled from the tail.

// A flagged axion: counters, exchange, new weight. Returns K; *removed tells
// whether the slot leaves the slab.
// The momentum of an a->gamma photon: the axion's direction with the axion's
// total energy E (its own momentum when massless).
__device__ __forceinline__ float3 photon_from_axion(const StepArgs& A, float px, float py, float pz) {
  if (A.mu <= 0.f) return make_float3(px, py, pz);
  const float p2 = px * px + py * py + pz * pz;
  const float f = __fdiv_rn(sqrtf(p2 + A.mu2), sqrtf(p2));
  return make_float3(px * f, py * f, pz * f);
}

__device__ __forceinline__ int axion_outcome(const StepArgs& A, const AxItem& t, long abase, bool bath,
                                             const Cnt& cnt, Lane64& x64, bool* removed) {
  const int K = t.r.x & 0xFF;
  const float wprod = __uint_as_float(t.r.y);
  const float wnew = __uint_as_float(t.r.z);
  const float om = sqrtf((t.px * t.px + t.py * t.py + t.pz * t.pz) + A.mu2) * kMeC2f;  // E
  cnt.add(C_CAP, (t.r.x & DF_CAPPED) ? 1u : 0u);
  cnt.add(C_CLAMP, (t.r.x & DF_OVER) ? 1u : 0u);
  cnt.add(C_EV_PINV, (unsigned)K);
  if (t.r.x & DF_ABSORBED) {
    x64.add((double)wnew, om, t.px, t.py, t.pz);
    cnt.add((t.r.x & DF_ABS_C) ? C_ABS_C : C_ABS_B, 1);
  } else if (A.absorb_mode == 1 && bath) {
    // weight reduction: the lost weight's energy goes to the plasma
    float wrem = t.w;
    if (K > 0) wrem = (t.r.x & DF_OVER) ? 0.f : __fsub_rn(t.w, __fmul_rn((float)K, wprod));
    x64.add((double)wrem - (double)wnew, om, t.px, t.py, t.pz);
  }
  *removed = !(t.r.x & DF_KEEP);
  if (!*removed && wnew != t.w) slot_w(A.a, abase + t.slot) = wnew;
  return K;
}

// A flagged photon: counters and the remaining weight. Returns K.
__device__ __forceinline__ int photon_outcome(const StepArgs& A, const PhItem& t, long gbase, const Cnt& cnt,
                                              bool* removed) {
  const int K = t.r.x & 0xFF;
  cnt.add(C_CAP, (t.r.x & DF_CAPPED) ? 1u : 0u);
  cnt.add(C_CLAMP, (t.r.x & DF_OVER) ? 1u : 0u);
  cnt.add(C_EV_P, (unsigned)K);
  *removed = !(t.r.x & DF_KEEP);
  if (K && !*removed) slot_w(A.g, gbase + t.slot) = __uint_as_float(t.r.z);
  return K;
}

// Slot of the i-th new axion of an emit phase: the freed slots holes[0,
// nholes) (ascending, entries `stride` apart) first, then from base on. A
// separate emit call has no freed slots (base: the axion count); a full step
// reuses the slots its absorb phase freed (base: the count at its start).
struct AxDest {
  const uint16_t* holes;
  int nholes, stride, base;
  __device__ __forceinline__ int at(int i) const {
    return i < nholes ? (int)holes[stride * i] : base + (i - nholes);
  }
};

// The K axion products of a gamma->a event, new axions i0 .. i0 + K - 1.
__device__ __forceinline__ void gamma_products(const StepArgs& A, const PhItem& t, long abase, const AxDest& D,
                                               int i0, int K, const Cnt& cnt) {
  const float wprod = __uint_as_float(t.r.y);
  const float pm = sqrtf(t.px * t.px + t.py * t.py + t.pz * t.pz);
  const float om = pm * kMeC2f;
  // a massive axion takes E = omega and momentum beta p_gamma
  const float beta = A.mu > 0.f ? axion_beta(pm, A.mu2) : 1.0f;
  const float ax = A.mu > 0.f ? t.px * beta : t.px, ay = A.mu > 0.f ? t.py * beta : t.py,
              az = A.mu > 0.f ? t.pz * beta : t.pz;
  for (int k = 0; k < K; ++k) {
    const int dst = D.at(i0 + k);
    if (dst < A.a.cap) {
      write_particle(A.a, abase + dst, wprod, ax, ay, az, t.x, t.y, t.z);
      if (A.tally_enable) tally_add(A, 0, wprod, om);
    } else {
      cnt.add(C_DROP, 1);
    }
  }
}

// The events of a flagged electron (thermal-bath emission), new axions i0
// on: event k takes cos theta, phi, energy and channel from one Philox
// block. A massive axion's event is kept when the channel uniform, rescaled
// inside its channel's interval, is below beta(E) (thinning; every event is
// kept when massless). Returns the kept events; WRITE = false only counts
// them (the warp path's offsets need the counts first).
template <bool WRITE>
__device__ __forceinline__ int electron_events(const StepArgs& A, uint32_t step, int cell, const ElItem& t,
                                               long abase, const AxDest& D, int i0, float r_cc, float r_cb,
                                               float r_T, float wu, const Cnt& cnt, Lane64& x64) {
  const int K = t.f & 0xFF;
  if (WRITE && wu <= 0.f) cnt.add(C_CAP, ((t.f & DF_CAPPED) ? 1u : 0u) + ((t.f & DF_CAPPED_B) ? 1u : 0u));
  if (!K) return 0;
  const bool eC = A.mask & AXPIC_CH_COMPTON, eB = A.mask & AXPIC_CH_BREMS;
  float facC = 1.f, facB = 1.f;
  bool cc = false, cb = false;
  const float lc = eC ? cap_lambda(t.w * r_cc, A.lam_cap, &facC, &cc) : 0.f;
  const float lb = eB ? cap_lambda(t.w * r_cb, A.lam_cap, &facB, &cb) : 0.f;
  const float fracC = lc / (lc + lb);
  const float wvC = cc ? A.w_a * facC : A.w_a;
  const float wvB = cb ? A.w_a * facB : A.w_a;
  const uint32_t gcell = A.cell_base + (uint32_t)cell;
  // the energies: the exact inverse CDFs (closed forms), the cell's spectral
  // record, or the network's cell-independent quantiles
  const float* q = nullptr;
  if (A.rate_model) {
    q = cell_sr(A, cell);
    if (!q) q = A.ra.uni;
  }
  int kept = 0;
  for (int k = 0; k < K; ++k) {
    const uint4 r = philox4x32_10(make_uint4(step, gcell, (uint32_t)t.slot, (S_EV_E << 24) | (uint32_t)k), A.rk);
    const float uc = u23(r.w);
    const bool isC = uc < fracC;
    const float E = (q ? sr_sample_x(q, isC ? 1 : 2, u23(r.z))
                       : icdf_lookup(A.tables + (isC ? TAB_COMPTON : TAB_BREMS) * kTableN, u23(r.z))) *
                    r_T;
    float pm = E * kInvMeC2f;
    if (A.mu > 0.f) {
      const float ut = isC ? __fdiv_rn(uc, fracC) : __fdiv_rn(__fsub_rn(uc, fracC), __fsub_rn(1.0f, fracC));
      const float beta = axion_beta(pm, A.mu2);
      if (!(ut < beta)) continue;  // thinned: below the threshold always
      pm = pm * beta;               // |p| = sqrt(E^2 - m_a^2)
    }
    if (WRITE) {
      const float3 dv = iso_dir(u23(r.x), u23(r.y));
      const float wv = isC ? wvC : wvB;
      const float px = pm * dv.x, py = pm * dv.y, pz = pm * dv.z;
      const int dst = D.at(i0 + kept);
      if (dst < A.a.cap) {
        write_particle(A.a, abase + dst, wv, px, py, pz, t.x, t.y, t.z);
        if (A.tally_enable) tally_add(A, isC ? 1 : 2, wv, E);
      } else {
        cnt.add(C_DROP, 1);
      }
      x64.add(-(double)wv, E, px, py, pz);
      cnt.add(isC ? C_EV_C : C_EV_B, 1);
    }
    ++kept;
  }
  return kept;
}

// ---------------------------------------------------------------- warp path
struct PhaseOut {
  int na, ng, np;  // axion and photon counts, new axions
  double x[4];
  bool any;
};

__device__ __forceinline__ void reduce_out(const Lane64& x64, PhaseOut* out) {
  out->any = __any_sync(kFull, x64.any);
  out->x[0] = out->x[1] = out->x[2] = out->x[3] = 0.0;
  if (out->any) {
    out->x[0] = warp_sum_d(x64.dE);
    out->x[1] = warp_sum_d(x64.dPx);
    out->x[2] = warp_sum_d(x64.dPy);
    out->x[3] = warp_sum_d(x64.dPz);
  }
}

// Absorb phase of one cell by the warp: a->gamma products, absorption and
// weight reduction, then (fill) the axion tail fill; without it the freed
// slots stay listed, ascending, in S.rmA (marked in S.rbA). sb is the warp's
// scratch, carved here again: a scratch descriptor passed by reference to an
// out-of-line call would live in local memory, written by every thread of
// the kernel.
__device__ __noinline__ void absorb_warp(const StepArgs& A, int cell, unsigned char* sb, const uint32_t* row,
                                         uint32_t* clr, const Cnt cnt, int na_start, int ng_start, bool fill,
                                         PhaseOut* out) {
  const EvScratch S = ev_carve(sb, A.a.cap, A.g.cap, A.e.cap);
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const bool bath = A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const int nfl = gather_row(row, clr, na_start, S.flA);
  for (int i = lane; i < (na_start + 31) / 32; i += 32) S.rbA[i] = 0u;
  __syncwarp();
  Lane64 x64;
  int run = 0, nrm = 0;
  for (int i0 = 0; i0 < nfl; i0 += 32) {
    const AxItem t = ax_load(A, abase, i0 + lane < nfl ? (int)S.flA[i0 + lane] : -1);
    int K = 0;
    bool removed = false;
    if (t.slot >= 0) K = axion_outcome(A, t, abase, bath, cnt, x64, &removed);
    int tot;
    int off = run + warp_excl_scan(K, &tot);
    const float wprod = __uint_as_float(t.r.y);
    const float3 pg = photon_from_axion(A, t.px, t.py, t.pz);
    for (int k = 0; k < K; ++k, ++off) {
      const int dst = ng_start + off;
      if (dst < A.g.cap) write_particle(A.g, gbase + dst, wprod, pg.x, pg.y, pg.z, t.x, t.y, t.z);
      else cnt.add(C_DROP, 1);
    }
    run += tot;
    const unsigned m = __ballot_sync(kFull, removed);
    if (removed) {
      S.rmA[nrm + __popc(m & lt)] = (uint16_t)t.slot;
      atomicOr(&S.rbA[t.slot >> 5], 1u << (t.slot & 31));
    }
    nrm += __popc(m);
  }
  reduce_out(x64, out);
  __syncwarp();
  if (fill && nrm > 0) compact_tail(A.a, abase, S.rmA, S.rbA, na_start - nrm, na_start);
  out->na = na_start - nrm;
  out->ng = min(ng_start + run, A.g.cap);
  out->np = 0;
}

// Emit phase of one cell by the warp: gamma->a, the thermal-bath events (new
// axions placed by D), then the photon tail fill (a->gamma products
// included).
__device__ __noinline__ void emit_warp(const StepArgs& A, uint32_t step, int cell, unsigned char* sb,
                                       const uint32_t* rowG, uint32_t* clrG, const uint32_t* rowE, uint32_t* clrE,
                                       const Cnt cnt, AxDest D, int ng_tot, int ng0, int ne, float wu, float r_cc,
                                       float r_cb, float r_T, PhaseOut* out) {
  const EvScratch S = ev_carve(sb, A.a.cap, A.g.cap, A.e.cap);
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  const int nflG = rowG ? gather_row(rowG, clrG, ng0, S.flG) : 0;
  const int nflE = rowE ? gather_row(rowE, clrE, ne, S.flE) : 0;
  for (int i = lane; i < (ng_tot + 31) / 32; i += 32) S.rbG[i] = 0u;
  __syncwarp();
  int run = 0, nrm = 0;
  for (int i0 = 0; i0 < nflG; i0 += 32) {
    const PhItem t = ph_load(A, gbase, i0 + lane < nflG ? (int)S.flG[i0 + lane] : -1);
    int K = 0;
    bool removed = false;
    if (t.slot >= 0) K = photon_outcome(A, t, gbase, cnt, &removed);
    int tot;
    const int off = run + warp_excl_scan(K, &tot);
    if (K) gamma_products(A, t, abase, D, off, K, cnt);
    run += tot;
    const unsigned m = __ballot_sync(kFull, removed);
    if (removed) {
      S.rmG[nrm + __popc(m & lt)] = (uint16_t)t.slot;
      atomicOr(&S.rbG[t.slot >> 5], 1u << (t.slot & 31));
    }
    nrm += __popc(m);
  }
  Lane64 x64;
  for (int i0 = 0; i0 < nflE; i0 += 32) {
    const ElItem t = el_load(A, ebase, i0 + lane < nflE ? (int)S.flE[i0 + lane] : -1, wu);
    int K = t.slot >= 0 ? (int)(t.f & 0xFF) : 0;
    if (A.mu > 0.f && K > 0)  // massive axions: the kept events, before the offsets
      K = electron_events<false>(A, step, cell, t, abase, D, 0, r_cc, r_cb, r_T, wu, cnt, x64);
    int tot;
    const int off = run + warp_excl_scan(K, &tot);
    if (t.slot >= 0) electron_events<true>(A, step, cell, t, abase, D, off, r_cc, r_cb, r_T, wu, cnt, x64);
    run += tot;
  }
  reduce_out(x64, out);
  __syncwarp();
  if (nrm > 0) compact_tail(A.g, gbase, S.rmG, S.rbG, ng_tot - nrm, ng_tot);
  out->na = min(D.base - D.nholes + run, A.a.cap);
  out->ng = ng_tot - nrm;
  out->np = run;
}

// ---------------------------------------------------------------- lane path
// Counts the flagged slots of a staged mask row in [0, n) and lists the
// first kLight of them (ascending, stride 32); *nz gets the nonzero words.
__device__ __forceinline__ int scan_row(const uint32_t* row, int n, uint16_t* list, uint32_t* nz) {
  const int nw = (n + 31) >> 5;
  int c = 0;
  uint32_t m = 0u;
  for (int w = 0; w < nw; ++w) {
    uint32_t v = row[w];
    if (v) {
      m |= 1u << w;
      if (w == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;
      while (v) {
        if (c < kLight) list[32 * c] = (uint16_t)(32 * w + __ffs(v) - 1);
        ++c;
        v &= v - 1u;
      }
    }
  }
  *nz = m;
  return c;
}

// Clears the nonzero words of a cell's global mask row.
__device__ __forceinline__ void clear_row(uint32_t* bits, int W, int cell, uint32_t nz) {
  uint32_t* row = bits + (size_t)cell * W;
  while (nz) {
    row[__ffs(nz) - 1] = 0u;
    nz &= nz - 1u;
  }
}

// Tail fill by one lane: the removed slots rm[0, nrm) (ascending) below
// n_surv are refilled, in order, by the kept slots of [n_surv, n). The first
// kLoad movers can be loaded ahead (fill_load) and written later
// (fill_store); fill_rest moves the others.
struct FillIt {
  int h, j, i, m;  // holes, next removed entry at or past the scan, scan position, movers done
};
struct Mover {
  float w, px, py, pz, x, y, z;
  int dst;
};

__device__ __forceinline__ FillIt fill_begin(const uint16_t* rm, int nrm, int n_surv) {
  FillIt it;
  it.h = 0;
  while (it.h < nrm && rm[32 * it.h] < n_surv) ++it.h;
  it.j = it.h;
  it.i = n_surv;
  it.m = 0;
  return it;
}

// Source slot of the next mover (the caller checks it.m < it.h).
__device__ __forceinline__ int fill_next(const uint16_t* rm, int nrm, FillIt& it) {
  while (it.j < nrm && rm[32 * it.j] == it.i) {
    ++it.j;
    ++it.i;
  }
  return it.i++;
}

__device__ __forceinline__ Mover mover_load(const SpeciesPtrs& sp, long base, int src, int dst) {
  Mover v;
  v.dst = dst;
  if (dst >= 0) {
    const long q = base + src;
    const float4 r = sp.wp[q];
    v.w = r.x;
    v.px = r.y;
    v.py = r.z;
    v.pz = r.w;
    const float4 u = sp.xyz[q];
    v.x = u.x;
    v.y = u.y;
    v.z = u.z;
  }
  return v;
}

__device__ __forceinline__ void mover_store(const SpeciesPtrs& sp, long base, const Mover& v) {
  if (v.dst >= 0) write_particle(sp, base + v.dst, v.w, v.px, v.py, v.pz, v.x, v.y, v.z);
}

// Loads the next kLoad movers.
__device__ __forceinline__ void fill_load(const SpeciesPtrs& sp, long base, const uint16_t* rm, int nrm, FillIt& it,
                                          Mover* v) {
#pragma unroll
  for (int t = 0; t < kLoad; ++t) {
    int src = 0, dst = -1;
    if (it.m < it.h) {
      src = fill_next(rm, nrm, it);
      dst = rm[32 * it.m++];
    }
    v[t] = mover_load(sp, base, src, dst);
  }
}

__device__ __forceinline__ void fill_rest(const SpeciesPtrs& sp, long base, const uint16_t* rm, int nrm, FillIt& it) {
  while (it.m < it.h) {
    Mover v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int src = 0, dst = -1;
      if (it.m < it.h) {
        src = fill_next(rm, nrm, it);
        dst = rm[32 * it.m++];
      }
      v[t] = mover_load(sp, base, src, dst);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) mover_store(sp, base, v[t]);
  }
}

// One cell by one lane: its absorb phase (doA), its emit phase (doE) or the
// full step (both: the new axions of the emit phase reuse the axion slots the
// absorb phase freed). Round trips: the first kLoad flagged axions and
// photons together; the first kLoad tail movers together; then the stores.
// Longer lists take further round trips. Every flagged axion is read before
// a new axion is written over a freed slot, and axion movers before any new
// axion is written.
struct LaneCell {
  int na, ng;       // in: counts at the start of the phase(s); out: final counts
  int ng0, ne;      // photons eligible for gamma->a, electrons
  int nflA, nflG, nflE;
  float wu, r_cc, r_cb, r_T;
};

__device__ __forceinline__ void cell_lane(const StepArgs& A, uint32_t step, int cell, bool doA, bool doE,
                                          uint16_t* lA, uint16_t* lG, const uint16_t* lE, LaneCell& L,
                                          const Cnt& cnt, Lane64& xa, Lane64& xe) {
  const bool bath = A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  const int nA = doA ? L.nflA : 0;
  const int nG = doE ? L.nflG : 0;
  const int nE = doE ? L.nflE : 0;
  AxItem ta[kLoad];
  PhItem tg[kLoad];
#pragma unroll
  for (int j = 0; j < kLoad; ++j) ta[j] = ax_load(A, abase, j < nA ? (int)lA[32 * j] : -1);
#pragma unroll
  for (int j = 0; j < kLoad; ++j) tg[j] = ph_load(A, gbase, j < nG ? (int)lG[32 * j] : -1);

  // absorb: a->gamma products after the photons present
  int na = L.na, ng = L.ng, nrmA = 0;
  if (doA) {
    int run = 0;
#pragma unroll
    for (int j = 0; j < kLoad; ++j) {
      if (ta[j].slot < 0) break;
      bool removed;
      const int K = axion_outcome(A, ta[j], abase, bath, cnt, xa, &removed);
      const float wprod = __uint_as_float(ta[j].r.y);
      const float3 pg = photon_from_axion(A, ta[j].px, ta[j].py, ta[j].pz);
      for (int k = 0; k < K; ++k) {
        const int dst = L.ng + run + k;
        if (dst < A.g.cap) write_particle(A.g, gbase + dst, wprod, pg.x, pg.y, pg.z, ta[j].x, ta[j].y, ta[j].z);
        else cnt.add(C_DROP, 1);
      }
      run += K;
      if (removed) lA[32 * nrmA++] = (uint16_t)ta[j].slot;
    }
    for (int i = kLoad; i < nA; ++i) {
      const AxItem t = ax_load(A, abase, lA[32 * i]);
      bool removed;
      const int K = axion_outcome(A, t, abase, bath, cnt, xa, &removed);
      const float wprod = __uint_as_float(t.r.y);
      const float3 pg = photon_from_axion(A, t.px, t.py, t.pz);
      for (int k = 0; k < K; ++k) {
        const int dst = L.ng + run + k;
        if (dst < A.g.cap) write_particle(A.g, gbase + dst, wprod, pg.x, pg.y, pg.z, t.x, t.y, t.z);
        else cnt.add(C_DROP, 1);
      }
      run += K;
      if (removed) lA[32 * nrmA++] = (uint16_t)t.slot;
    }
    na = L.na - nrmA;
    ng = min(L.ng + run, A.g.cap);
  }

  // emit: gamma->a decisions of the loaded photons (products after the fill)
  int nrmG = 0, Kg[kLoad];
#pragma unroll
  for (int j = 0; j < kLoad; ++j) {
    Kg[j] = 0;
    if (tg[j].slot >= 0) {
      bool removed;
      Kg[j] = photon_outcome(A, tg[j], gbase, cnt, &removed);
      if (removed) lG[32 * nrmG++] = (uint16_t)tg[j].slot;
    }
  }

  // tail movers, loaded together: the axions' unless the step reuses the
  // freed slots, the photons' when every photon removal is known
  const bool reuse = doA && doE;
  FillIt fa = fill_begin(lA, reuse ? 0 : nrmA, na);
  Mover ma[kLoad], mg[kLoad];
  fill_load(A.a, abase, lA, reuse ? 0 : nrmA, fa, ma);
  const bool gFill = nG <= kLoad;
  FillIt fg = fill_begin(lG, nrmG, ng - nrmG);
  if (gFill) fill_load(A.g, gbase, lG, nrmG, fg, mg);
  if (!reuse) {
#pragma unroll
    for (int t = 0; t < kLoad; ++t) mover_store(A.a, abase, ma[t]);
    fill_rest(A.a, abase, lA, nrmA, fa);
  }

  if (doE) {
    // new axions: gamma->a products, then thermal-bath events
    const AxDest D{lA, reuse ? nrmA : 0, 32, reuse ? L.na : na};
    int NP = 0;
#pragma unroll
    for (int j = 0; j < kLoad; ++j) {
      if (Kg[j]) gamma_products(A, tg[j], abase, D, NP, Kg[j], cnt);
      NP += Kg[j];
    }
    for (int i = kLoad; i < nG; ++i) {
      const PhItem t = ph_load(A, gbase, lG[32 * i]);
      bool removed;
      const int K = photon_outcome(A, t, gbase, cnt, &removed);
      if (K) gamma_products(A, t, abase, D, NP, K, cnt);
      NP += K;
      if (removed) lG[32 * nrmG++] = (uint16_t)t.slot;
    }
    for (int i = 0; i < nE; ++i) {
      const ElItem t = el_load(A, ebase, lE[32 * i], L.wu);
      NP += electron_events<true>(A, step, cell, t, abase, D, NP, L.r_cc, L.r_cb, L.r_T, L.wu, cnt, xe);
    }
    na = min(D.base - D.nholes + NP, A.a.cap);
    if (reuse && NP < nrmA) {
      // freed slots left over: closed from the tail (their movers lie beyond
      // every slot a new axion took)
      FillIt fr = fill_begin(lA + 32 * NP, nrmA - NP, na);
      fill_rest(A.a, abase, lA + 32 * NP, nrmA - NP, fr);
    }
    // photon tail fill (a->gamma products included)
    if (gFill) {
#pragma unroll
      for (int t = 0; t < kLoad; ++t) mover_store(A.g, gbase, mg[t]);
    } else {
      fg = fill_begin(lG, nrmG, ng - nrmG);
    }
    fill_rest(A.g, gbase, lG, nrmG, fg);
    ng -= nrmG;
  }
  L.na = na;
  L.ng = ng;
}

#ifndef AXPIC_EVENT_MIN_CTAS
#define AXPIC_EVENT_MIN_CTAS 4
#endif
// the full-step kernel, without the warp paths (event_heavy_kernel takes
// them), fits more CTAs an SM
#ifndef AXPIC_EVENT_FULL_MIN_CTAS
#define AXPIC_EVENT_FULL_MIN_CTAS 6
#endif

// Round trip 1: counts and the mask rows (staged by cp.async; cleared for
// the next step as soon as they are read). Only the cells that have an
// electron event read the cell constants; only those with a flagged slot
// read their exchange buffer (while their events run), and only those with
// an exchange write it. Each phase runs first in the lanes whose cell is
// light for it, then warp-wide for the heavy cells one by one (in a full
// step, by event_heavy_kernel: without the warp paths, and with one load of
// each kind in flight, this kernel holds 6 CTAs an SM instead of 4); a
// cell's absorb phase ends before its emit phase starts. The absorb and emit
// exchanges are added to the cell's buffer in that order, whichever way the
// step was called.
template <int PH>
__global__ void __launch_bounds__(128, PH == 3 ? AXPIC_EVENT_FULL_MIN_CTAS : AXPIC_EVENT_MIN_CTAS)
    event_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long warp_cnt[4][kNumCounters];
  const int wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cell = A.cell0 + (blockIdx.x * nw + wid) * 32 + lane;
  const bool valid = cell < A.cell0 + A.ncells;
  if (lane < kNumCounters) warp_cnt[wid][lane] = 0ull;
  __syncwarp();
  const Cnt cnt{warp_cnt[wid]};
  unsigned char* const sbase = smem + wid * ev_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
  const EvScratch S = ev_carve(sbase, A.a.cap, A.g.cap, A.e.cap);
  uint16_t* lA = S.lt + lane;
  uint16_t* lG = lA + 32 * kLight;
  uint16_t* lE = lG + 32 * kLight;
  const uint32_t step = step_of(A);
  const int mask = A.mask;
  const bool emitG = (PH & PH_EMIT) && (mask & AXPIC_CH_PRIMAKOFF);
  const bool emitE = (PH & PH_EMIT) && (mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS));
  const bool staged = S.rowA != nullptr;
  uint32_t* rA = staged ? S.rowA + lane * S.sA : nullptr;
  uint32_t* rG = staged ? S.rowG + lane * S.sG : nullptr;
  uint32_t* rE = staged ? S.rowE + lane * S.sE : nullptr;

  // ------------------------------------------------------------ round trip 1
  LaneCell L;
  L.na = L.ng = L.ng0 = L.ne = 0;
  L.nflA = L.nflG = L.nflE = 0;
  L.wu = L.r_cc = L.r_cb = L.r_T = 0.f;
  int pstart = 0;
  double xb[4] = {0.0, 0.0, 0.0, 0.0};
  bool xload = false;
  if (valid) {
    if (staged) {
      if (PH & PH_ABSORB)
        for (int w = 0; w < A.Wa; ++w) cp_async4(rA + w, A.bitsA + (size_t)cell * A.Wa + w);
      if (emitG)
        for (int w = 0; w < A.Wg; ++w) cp_async4(rG + w, A.bitsG + (size_t)cell * A.Wg + w);
      if (emitE)
        for (int w = 0; w < A.We; ++w) cp_async4(rE + w, A.bitsE + (size_t)cell * A.We + w);
    }
    L.ne = min(max(A.e.count[cell], 0), A.e.cap);
    L.ng = min(max(A.g.count[cell], 0), A.g.cap);
    L.na = min(max(A.a.count[cell], 0), A.a.cap);
    if (!(PH & PH_ABSORB) && A.use_snapshot) pstart = A.photon_start[cell];
  }
  const int ne = L.ne, ng_start = L.ng, na_start = L.na;
  L.ng0 = (PH & PH_ABSORB) ? ng_start : (A.use_snapshot ? min(pstart, ng_start) : ng_start);
  // particles present at the start of the step: counted by the absorb phase,
  // or by the emit phase when no absorb ran this step
  if ((PH & PH_ABSORB) || ((PH & PH_EMIT) && !A.use_snapshot)) {
    const int sne = warp_sum_i(ne), sng = warp_sum_i(ng_start), sna = warp_sum_i(na_start);
    const unsigned nv = __popc(__ballot_sync(kFull, valid));
    if (lane == 0) {
      cnt.add(C_NE, (unsigned)sne);
      cnt.add(C_NG, (unsigned)sng);
      cnt.add(C_NA, (unsigned)sna);
      cnt.add(C_CELLS, nv);
    }
  }
  if (staged) cp_async_wait_all();
  __syncwarp();

  bool hA = false, hE = false;
  // a full step leaves a cell heavy in either phase, rows uncleared, to
  // event_heavy_kernel
  bool defer = false;
  if (valid) {
    if (staged) {
      uint32_t nzA = 0u, nzG = 0u, nzE = 0u;
      if (PH & PH_ABSORB) L.nflA = scan_row(rA, na_start, lA, &nzA);
      if (emitG) L.nflG = scan_row(rG, L.ng0, lG, &nzG);
      if (emitE) L.nflE = scan_row(rE, ne, lE, &nzE);
      hA = L.nflA > kLight;
      hE = L.nflG > kLight || L.nflE > kLightE;
      defer = PH == (PH_ABSORB | PH_EMIT) && (hA || hE);
      if (!defer) {
        if (PH & PH_ABSORB) clear_row(A.bitsA, A.Wa, cell, nzA);
        if (emitG) clear_row(A.bitsG, A.Wg, cell, nzG);
        if (emitE) clear_row(A.bitsE, A.We, cell, nzE);
      }
    } else {
      hA = (PH & PH_ABSORB) != 0;
      hE = (PH & PH_EMIT) != 0;
      defer = PH == (PH_ABSORB | PH_EMIT);
    }
    if (PH == PH_ABSORB) A.photon_start[cell] = ng_start;  // read by the emit call of this step
    // the cell constants of the thermal-bath events, for the cells that
    // have one (the capped means of common-weight cells are counted by the
    // decision kernel)
    if (!defer && emitE && (!staged || L.nflE > 0)) {
      const float* rec = A.rec + (size_t)cell * kRecLen;
      L.wu = A.mom[(size_t)cell * kMomLen + M_WU];
      L.r_cc = rec[R_CC];
      L.r_cb = rec[R_CB];
      L.r_T = rec[R_T];
    }
    // the exchange buffer of a cell with an event, loaded while its events run
    if (!defer && (!staged || (L.nflA | L.nflG | L.nflE))) {
      xload = true;
      const double2* x2 = reinterpret_cast<const double2*>(A.xbuf + (size_t)cell * 4);
      cp_async16(S.xs + 2 * lane, x2);
      cp_async16(S.xs + 2 * lane + 1, x2 + 1);
    }
  }

  Lane64 xa, xe;
  if (PH == (PH_ABSORB | PH_EMIT)) {
    // full step: a cell light in both phases is taken by its lane, any other
    // by event_heavy_kernel after this kernel (a warp per cell); either way
    // the new axions reuse the freed slots
    if (valid && !defer && (L.nflA | L.nflG | L.nflE))
      cell_lane(A, step, cell, true, true, lA, lG, lE, L, cnt, xa, xe);
    // the heavy cells are listed for event_heavy_kernel, from index cell0
    const unsigned hm = __ballot_sync(kFull, defer);
    if (hm) {
      int base = 0;
      if (lane == 0) base = atomicAdd(A.heavy_n, __popc(hm));
      base = __shfl_sync(kFull, base, 0);
      if (defer) A.heavy[A.cell0 + base + __popc(hm & ((1u << lane) - 1u))] = cell;
    }
  } else if (PH == PH_ABSORB) {
    if (valid && !hA && L.nflA) cell_lane(A, step, cell, true, false, lA, lG, lE, L, cnt, xa, xe);
    __syncwarp();
    for (unsigned hm = __ballot_sync(kFull, valid && hA); hm; hm &= hm - 1u) {
      const int j = __ffs(hm) - 1;
      const int c = __shfl_sync(kFull, cell, j);
      PhaseOut o;
      absorb_warp(A, c, sbase, staged ? S.rowA + j * S.sA : A.bitsA + (size_t)c * A.Wa,
                  staged ? nullptr : A.bitsA + (size_t)c * A.Wa, cnt, __shfl_sync(kFull, na_start, j),
                  __shfl_sync(kFull, ng_start, j), true, &o);
      if (lane == j) {
        L.na = o.na;
        L.ng = o.ng;
        xa.dE = o.x[0];
        xa.dPx = o.x[1];
        xa.dPy = o.x[2];
        xa.dPz = o.x[3];
        xa.any = o.any;
      }
    }
  } else {
    if (valid && !hE && (L.nflG | L.nflE)) cell_lane(A, step, cell, false, true, lA, lG, lE, L, cnt, xa, xe);
    __syncwarp();
    for (unsigned hm = __ballot_sync(kFull, valid && hE); hm; hm &= hm - 1u) {
      const int j = __ffs(hm) - 1;
      const int c = __shfl_sync(kFull, cell, j);
      PhaseOut o;
      const uint32_t* gG = emitG ? (staged ? S.rowG + j * S.sG : A.bitsG + (size_t)c * A.Wg) : nullptr;
      const uint32_t* gE = emitE ? (staged ? S.rowE + j * S.sE : A.bitsE + (size_t)c * A.We) : nullptr;
      emit_warp(A, step, c, sbase, gG, (emitG && !staged) ? A.bitsG + (size_t)c * A.Wg : nullptr, gE,
                (emitE && !staged) ? A.bitsE + (size_t)c * A.We : nullptr, cnt,
                AxDest{nullptr, 0, 1, __shfl_sync(kFull, L.na, j)}, __shfl_sync(kFull, L.ng, j),
                __shfl_sync(kFull, L.ng0, j), __shfl_sync(kFull, ne, j), __shfl_sync(kFull, L.wu, j),
                __shfl_sync(kFull, L.r_cc, j), __shfl_sync(kFull, L.r_cb, j), __shfl_sync(kFull, L.r_T, j), &o);
      if (lane == j) {
        L.na = o.na;
        L.ng = o.ng;
        xe.dE = o.x[0];
        xe.dPx = o.x[1];
        xe.dPy = o.x[2];
        xe.dPz = o.x[3];
        xe.any = o.any;
      }
    }
  }
  if (valid && !defer) {
    A.a.count[cell] = L.na;
    A.g.count[cell] = L.ng;
    if (xa.any || xe.any) {
      {
        const double2* x2 = xload ? S.xs + 2 * lane : reinterpret_cast<const double2*>(A.xbuf + (size_t)cell * 4);
        if (xload) cp_async_wait_all();
        const double2 a = x2[0], b = x2[1];
        xb[0] = a.x;
        xb[1] = a.y;
        xb[2] = b.x;
        xb[3] = b.y;
      }
      if (xa.any) {
        xb[0] += xa.dE;
        xb[1] += xa.dPx;
        xb[2] += xa.dPy;
        xb[3] += xa.dPz;
      }
      if (xe.any) {
        xb[0] += xe.dE;
        xb[1] += xe.dPx;
        xb[2] += xe.dPy;
        xb[3] += xe.dPz;
      }
      double2* xo = reinterpret_cast<double2*>(A.xbuf + (size_t)cell * 4);
      xo[0] = make_double2(xb[0], xb[1]);
      xo[1] = make_double2(xb[2], xb[3]);
    }
  }
  __syncwarp();
  if (lane < kNumCounters) {
    const unsigned long long v = warp_cnt[wid][lane];
    if (v) atomicAdd(A.counters + (size_t)(blockIdx.x % A.ctr_rows) * kNumCounters + lane, v);
    if (lane == C_DROP && v) atomicOr(A.err, ERR_CAPACITY);
  }
}


// The full step of the cells the event kernel listed as heavy (more flagged
// slots in a phase than a lane takes): a warp per cell, persistent over the
// list, with the mask rows read and cleared in global memory. Cells are
// independent within a step, so each gets what the warp path inside the
// event kernel gave it; the list order does not matter.
constexpr int kHeavyGrid = 152;  // one CTA on each of the 152 SMs

__global__ void __launch_bounds__(128) event_heavy_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long warp_cnt[4][kNumCounters];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  if (lane < kNumCounters) warp_cnt[wid][lane] = 0ull;
  __syncwarp();
  const Cnt cnt{warp_cnt[wid]};
  unsigned char* const sbase = smem + wid * ev_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
  const EvScratch S = ev_carve(sbase, A.a.cap, A.g.cap, A.e.cap);
  const uint32_t step = step_of(A);
  const bool emitG = (A.mask & AXPIC_CH_PRIMAKOFF) != 0;
  const bool emitE = (A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS)) != 0;
  const int n = *A.heavy_n;
  for (int k = blockIdx.x * nw + wid; k < n; k += gridDim.x * nw) {
    const int c = A.heavy[A.cell0 + k];
    const int na0 = min(max(A.a.count[c], 0), A.a.cap);
    const int ng0 = min(max(A.g.count[c], 0), A.g.cap);
    const int ne = min(max(A.e.count[c], 0), A.e.cap);
    float wu = 0.f, r_cc = 0.f, r_cb = 0.f, r_T = 0.f;
    if (emitE) {
      const float* rec = A.rec + (size_t)c * kRecLen;
      wu = A.mom[(size_t)c * kMomLen + M_WU];
      r_cc = rec[R_CC];
      r_cb = rec[R_CB];
      r_T = rec[R_T];
    }
    uint32_t* rowA = A.bitsA + (size_t)c * A.Wa;
    uint32_t* rowG = emitG ? A.bitsG + (size_t)c * A.Wg : nullptr;
    uint32_t* rowE = emitE ? A.bitsE + (size_t)c * A.We : nullptr;
    PhaseOut oa, oe;
    absorb_warp(A, c, sbase, rowA, rowA, cnt, na0, ng0, false, &oa);
    const int nrmA = na0 - oa.na;
    emit_warp(A, step, c, sbase, rowG, rowG, rowE, rowE, cnt, AxDest{S.rmA, nrmA, 1, na0}, oa.ng, ng0, ne, wu, r_cc,
              r_cb, r_T, &oe);
    // freed slots left over: closed from the tail
    if (oe.np < nrmA) compact_tail(A.a, (long)c * A.a.cap, S.rmA + oe.np, S.rbA, oe.na, na0);
    if (lane == 0) {
      A.a.count[c] = oe.na;
      A.g.count[c] = oe.ng;
      if (oa.any || oe.any) {
        double* xb = A.xbuf + (size_t)c * 4;
        double x0 = xb[0], x1 = xb[1], x2 = xb[2], x3 = xb[3];
        if (oa.any) {
          x0 += oa.x[0];
          x1 += oa.x[1];
          x2 += oa.x[2];
          x3 += oa.x[3];
        }
        if (oe.any) {
          x0 += oe.x[0];
          x1 += oe.x[1];
          x2 += oe.x[2];
          x3 += oe.x[3];
        }
        xb[0] = x0;
        xb[1] = x1;
        xb[2] = x2;
        xb[3] = x3;
      }
    }
    __syncwarp();
  }
  __syncwarp();
  if (lane < kNumCounters) {
    const unsigned long long v = warp_cnt[wid][lane];
    if (v) atomicAdd(A.counters + (size_t)(blockIdx.x % A.ctr_rows) * kNumCounters + lane, v);
    if (lane == C_DROP && v) atomicOr(A.err, ERR_CAPACITY);
  }
}

// ---------------------------------------------------------------- launchers
size_t step_smem_per_warp(int acap, int gcap, int ecap) { return ev_scratch_bytes(acap, gcap, ecap); }

int resident_ctas(const void* fn, int threads, size_t dyn_smem, int max_per_sm) {
  int dev = 0, sms = 0, regs_sm = 0, smem_sm = 0, reserved = 0, threads_sm = 0, blocks_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) ||
      cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) ||
      cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) ||
      cudaFuncGetAttributes(&fa, fn))
    return 0;
  const int warps = (threads + 31) / 32;
  const int regs_cta = warps * ((max(1, fa.numRegs) * 32 + 255) / 256 * 256);
  const int smem_cta = (int)((fa.sharedSizeBytes + dyn_smem + reserved + 127) / 128 * 128);
  const int nb = min(min(regs_sm / regs_cta, smem_sm / smem_cta), min(threads_sm / (warps * 32), blocks_sm));
  return max(1, min(nb, max_per_sm)) * max(1, sms);
}

template <int PH>
static cudaError_t launch_events(const StepArgs& A, int warps, cudaStream_t st) {
  const size_t per = ev_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
  const int grid = (A.ncells + 32 * warps - 1) / (32 * warps);
  if (PH == (PH_ABSORB | PH_EMIT)) {
    cudaError_t e = cudaMemsetAsync(A.heavy_n, 0, sizeof(int32_t), st);
    if (e) return e;
  }
  event_kernel<PH><<<grid, warps * 32, per * warps, st>>>(A);
  if (PH == (PH_ABSORB | PH_EMIT)) {
    // persistent over the heavy list: a warp per cell, at most one warp per
    // cell of the launch and kHeavyGrid CTAs
    const int hgrid = max(1, min((A.ncells + warps - 1) / warps, kHeavyGrid));
    event_heavy_kernel<<<hgrid, warps * 32, per * warps, st>>>(A);
  }
  return cudaGetLastError();
}

// Persistent decision grid: A.dec_grid CTAs (what the device holds at once
// for this chunk size), at most one warp per chunk.
static int dec_blocks(const StepArgs& A) {
  const int nchunks = (A.ncells + A.dec_chunk - 1) / A.dec_chunk;
  const int need = (nchunks + kDecWarps - 1) / kDecWarps;
  return max(1, min(need, A.dec_grid));
}

// The decision passes a phase set needs, as DK_* bits.
static int decide_kinds(const StepArgs& A, int phases) {
  int k = 0;
  if ((phases & PH_EMIT) && (A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS)) && A.e.cap > 0) k |= DK_ELECTRON;
  if ((phases & PH_EMIT) && (A.mask & AXPIC_CH_PRIMAKOFF) && A.g.cap > 0) k |= DK_PHOTON;
  if ((phases & PH_ABSORB) && A.a.cap > 0) k |= DK_AXION;
  return k;
}

static cudaError_t launch_decide(const StepArgs& A, int phases, cudaStream_t st) {
  const int kinds = decide_kinds(A, phases);
  if (kinds == 0) return cudaSuccess;
  switch (A.dec_chunk) {
    case 4:
      decide_kernel<4><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
    case 8:
      decide_kernel<8><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
    case 16:
      decide_kernel<16><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
    default:
      decide_kernel<32><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_feedback(const StepArgs& A, cudaStream_t st) {
  const int grid = (A.ncells + kFeedbackThreads - 1) / kFeedbackThreads;
  feedback_kernel<<<grid, kFeedbackThreads, 0, st>>>(A);
  return cudaGetLastError();
}

const char* step_kernel_names(int rate_model, int T_mode) {
  if (T_mode == 2 && rate_model == 1) return "decide_kernel,event_kernel,feedback_kernel,sr_table_kernel";
  if (T_mode == 2 && rate_model == 2) return "decide_kernel,event_kernel,feedback_kernel,sr_cells_kernel";
  return "decide_kernel,event_kernel,feedback_kernel";
}

__global__ void set_step_kernel(uint32_t* p, uint32_t v, int n) {
  for (int i = 0; i < n; ++i) p[i] = v;
}

cudaError_t launch_set_step(uint32_t* p, uint32_t v, int n, cudaStream_t st) {
  set_step_kernel<<<1, 1, 0, st>>>(p, v, n);
  return cudaGetLastError();
}

cudaError_t decide_shape(int requested, int ncells, int* chunk, int* grid) {
  int c = requested;
  if (c == 0) {
    int g = 1;
    const cudaError_t e = decide_resident_ctas(32, &g);
    if (e) return e;
    const long warps = (long)g * kDecWarps;
    c = 4;
    for (int k : {32, 16, 8}) {
      if ((long)ncells / k >= warps) {
        c = k;
        break;
      }
    }
  }
  *chunk = c;
  return decide_resident_ctas(c, grid);
}

cudaError_t decide_resident_ctas(int chunk, int* out) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return e;
  if (chunk == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<4>, kDecThreads, 0);
  else if (chunk == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<8>, kDecThreads, 0);
  else if (chunk == 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<16>, kDecThreads, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<32>, kDecThreads, 0);
  if (e) return e;
  *out = max(1, nb) * max(1, sms);
  return cudaSuccess;
}

// After the temperature update of an evolved-T step the rate model's records
// follow the new T: the table model's spectral records, or the surrogate
// network's prefactors (the table's records where it is not trusted).
static cudaError_t launch_records_update(const StepArgs& A, const SrArgs* sra, cudaStream_t st) {
  if (!sra || A.T_mode != 2) return cudaSuccess;
  return launch_sr_records(A.rate_model, *sra, st);
}

cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st, cudaEvent_t* ev,
                        const SrArgs* sra) {
  if (A.ncells == 0) return cudaSuccess;
  cudaError_t e;
  // optional measurement: events between the kernels of a full step
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], st) : cudaSuccess; };
  switch (phases) {
    case PH_ABSORB:
      if ((e = launch_decide(A, PH_ABSORB, st))) return e;
      return launch_events<PH_ABSORB>(A, warps, st);
    case PH_EMIT:
      if ((e = launch_decide(A, PH_EMIT, st))) return e;
      return launch_events<PH_EMIT>(A, warps, st);
    case PH_FEEDBACK:
      if ((e = launch_feedback(A, st))) return e;
      return launch_records_update(A, sra, st);
    case PH_ALL:
      if ((e = mark(0)) || (e = launch_decide(A, PH_ABSORB | PH_EMIT, st)) || (e = mark(1))) return e;
      if ((e = launch_events<PH_ABSORB | PH_EMIT>(A, warps, st)) || (e = mark(2))) return e;
      if ((e = launch_feedback(A, st)) || (e = mark(3)) || (e = launch_records_update(A, sra, st)) || (e = mark(4)))
        return e;
      return cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

// The dynamic shared-memory limit of the event kernels is a process-wide
// attribute of each function: contexts with smaller slabs share it with
// larger ones, so it is only ever raised (per device, under a lock), never
// lowered under a context that needs more.
cudaError_t set_step_smem_limits(size_t bytes) {
  static std::mutex mu;
  static size_t set_for[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t* cur = dev >= 0 && dev < 64 ? &set_for[dev] : nullptr;
  if (cur && bytes <= *cur) return cudaSuccess;
  const int b = (int)bytes;
  if ((e = cudaFuncSetAttribute(event_kernel<PH_ABSORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) ||
      (e = cudaFuncSetAttribute(event_kernel<PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) ||
      (e = cudaFuncSetAttribute(event_kernel<PH_ABSORB | PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) ||
      (e = cudaFuncSetAttribute(event_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  if (cur) *cur = bytes;
  return cudaSuccess;
}

}  // namespace axpic
