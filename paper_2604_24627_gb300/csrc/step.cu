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
  s.w[idx] = w;
  s.px[idx] = px;
  s.py[idx] = py;
  s.pz[idx] = pz;
  s.x[idx] = x;
  s.y[idx] = y;
  s.z[idx] = z;
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
  float wprod, wnew, om;
  bool keep, absorbed, capped, over, abs_c;
};

__device__ __forceinline__ AxionDecision axion_decide(const float* rec, const float* sr, const StepArgs& A, int mask,
                                                      float w, float px, float py, float pz, uint32_t wP,
                                                      uint32_t wA) {
  AxionDecision d;
  d.om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
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
    const float P = use_sr ? -expm1f(-A.cc.prim_mult * sr_prim_gdt(sr, xr)) : prim_prob(rec, d.om, rec[R_APINV]);
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

// Out-of-line full decisions: they reload the cell's record themselves so
// that the caller's record stays in registers.
__device__ __noinline__ AxionDecision axion_decide_slow(const StepArgs& A, int cell, int mask, float w, float px,
                                                        float py, float pz, uint32_t wP, uint32_t wA) {
  float rec[kRecLen];
  load_rec(A, cell, rec);
  return axion_decide(rec, A.rate_model ? A.sr + (size_t)cell * kSrLen : nullptr, A, mask, w, px, py, pz, wP, wA);
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
  d.om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
  const float xr = d.om * rec[R_INVT];
  const float P = sr && sr_in_range(xr) ? -expm1f(-sr_prim_gdt(sr, xr)) : prim_prob(rec, d.om, rec[R_AP]);
  float fac;
  const float le = cap_lambda(w * P * A.inv_w_a, A.lam_cap, &fac, &d.capped);
  d.K = poisson_inv(u23(wd), le);
  d.wrem = w;
  d.wprod = 0.f;
  d.over = false;
  if (d.K > 0) d.wprod = deplete(w, d.K, d.capped ? A.w_a * fac : A.w_a, &d.wrem, &d.over);
  return d;
}

__device__ __noinline__ PhotonDecision photon_decide_slow(const StepArgs& A, int cell, float w, float px, float py,
                                                          float pz, uint32_t wd) {
  float rec[kRecLen];
  load_rec(A, cell, rec);
  return photon_decide(rec, A.rate_model ? A.sr + (size_t)cell * kSrLen : nullptr, A, w, px, py, pz, wd);
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
__device__ __forceinline__ bool no_conversion(float w, float p2, float c_s, float Acoef, float inv_wref, float u,
                                              float lam_cap, float gm) {
  const float s = p2 * c_s;
  const float Fb = s < 2.5f ? 0.5f * s : __logf(1.0f + s);
  const float lb = w * Acoef * Fb * inv_wref * (1.0001f * gm);
  return lb < lam_cap && u <= 1.0f - lb - 1e-6f;
}

// Absorption: P_abs <= tau; x/(1-e^-x) <= 1 + x bounds the Compton-like
// factor, (1 - e^-x) <= 1 the Bose-Einstein one.
__device__ __forceinline__ bool no_absorption(float r_bc, float r_bb, const StepArgs& A, int mask, float x, float u) {
  float tb = 0.f;
  if (mask & AXPIC_CH_COMPTON) tb += r_bc * x * (1.0f + x);
  if (mask & AXPIC_CH_BREMS) tb += r_bb * __expf(A.brems_am3 * __logf(x));
  return u >= tb * (1.001f * A.guard_margin) + 1e-6f;
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
  for (int q = lane; q < nqe; q += 32) {
    const long b = ebase + 4 * q;
    const float4 w4 = ld4(A.e.w + b);
    float4 x4 = ld4(A.e.px + b), y4 = ld4(A.e.py + b), z4 = ld4(A.e.pz + b);
    float* xs = reinterpret_cast<float*>(&x4);
    float* ys = reinterpret_cast<float*>(&y4);
    float* zs = reinterpret_cast<float*>(&z4);
    const float* ws = reinterpret_cast<const float*>(&w4);
    const int nj = min(4, ne - 4 * q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= nj) break;
      const float w = ws[j];
      const float nx = xs[j] + fmaf(s1, xs[j], fbx);
      const float ny = ys[j] + fmaf(s1, ys[j], fby);
      const float nz = zs[j] + fmaf(s1, zs[j], fbz);
      const float ddx = nx - xs[j], ddy = ny - ys[j], ddz = nz - zs[j];
      aE += w * (ddx * (2.f * xs[j] + ddx) + ddy * (2.f * ys[j] + ddy) + ddz * (2.f * zs[j] + ddz));
      aPx += w * ddx;
      aPy += w * ddy;
      aPz += w * ddz;
      mW += w;
      mPx += w * nx;
      mPy += w * ny;
      mPz += w * nz;
      mU2 += w * (nx * nx + ny * ny + nz * nz);
      xs[j] = nx;
      ys[j] = ny;
      zs[j] = nz;
    }
    if (nj == 4) {
      *reinterpret_cast<float4*>(A.e.px + b) = x4;
      *reinterpret_cast<float4*>(A.e.py + b) = y4;
      *reinterpret_cast<float4*>(A.e.pz + b) = z4;
    } else {
      for (int j = 0; j < nj; ++j) {
        A.e.px[b + j] = xs[j];
        A.e.py[b + j] = ys[j];
        A.e.pz[b + j] = zs[j];
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
// set by atomicOr (rare) and cleared by the event kernel after reading.

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
// Cells per chunk: a launch-shape choice (2, 4 or 8), picked per context.
constexpr int kChunkDefault = AXPIC_DEC_CHUNK;
static_assert(kChunkDefault == 2 || kChunkDefault == 4 || kChunkDefault == 8, "cells per decision chunk");
constexpr int kListCap = 32 + 4 * 32;  // < 32 pending + one pass of flags

// Per-warp lists: {cell, slot, decision word(s)}.
struct DecLists {
  uint4 a[kDecWarps][kListCap];
  uint4 g[kDecWarps][kListCap];
};

// Flat quad range of a chunk: lanes < nc hold their cell's slot count n; on
// return every lane holds its cell's first quad (qoff), the starts of cells
// 1..C-1 (qo, cells beyond nc start at the total) and the total.
template <int C>
struct QuadRange {
  int qoff, total;
  int qo[C];
};

template <int C>
__device__ __forceinline__ QuadRange<C> quad_range(int n, int lane, int nc) {
  QuadRange<C> R;
  const int nq = lane < nc ? (n + 3) >> 2 : 0;
  R.qoff = warp_excl_scan(nq, &R.total);
#pragma unroll
  for (int c = 0; c < C; ++c) R.qo[c] = __shfl_sync(kFull, R.qoff, c);
#pragma unroll
  for (int c = 0; c < C; ++c)
    if (c >= nc) R.qo[c] = R.total;
  return R;
}

// Cell (in the chunk) of flat quad g.
template <int C>
__device__ __forceinline__ int quad_cell(const QuadRange<C>& R, int g) {
  int lc = 0;
#pragma unroll
  for (int c = 1; c < C; ++c) lc += g >= R.qo[c] ? 1 : 0;
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

__device__ __forceinline__ void axion_full(const StepArgs& A, uint4 it) {
  const int cell = (int)it.x;
  const long idx = (long)cell * A.a.cap + it.y;
  const AxionDecision d =
      axion_decide_slow(A, cell, A.mask, A.a.w[idx], A.a.px[idx], A.a.py[idx], A.a.pz[idx], it.z, it.w);
  uint32_t f = (uint32_t)d.K;
  if (d.keep) f |= DF_KEEP;
  if (d.absorbed) f |= DF_ABSORBED;
  if (d.abs_c) f |= DF_ABS_C;
  if (d.capped) f |= DF_CAPPED;
  if (d.over) f |= DF_OVER;
  A.recA[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wnew), 0u);
}

__device__ __forceinline__ void photon_full(const StepArgs& A, uint4 it) {
  const int cell = (int)it.x;
  const long idx = (long)cell * A.g.cap + it.y;
  const PhotonDecision d = photon_decide_slow(A, cell, A.g.w[idx], A.g.px[idx], A.g.py[idx], A.g.pz[idx], it.z);
  uint32_t f = (uint32_t)d.K;
  if (d.wrem > 0.f) f |= DF_KEEP;
  if (d.capped) f |= DF_CAPPED;
  if (d.over) f |= DF_OVER;
  A.recG[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wrem), 0u);
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
      // u23(w) > F0 exactly when (w >> 9) > floor(F0 2^23 - 1/2): the
      // scaling and the subtraction are exact in binary32
      thr = (int)floorf(__fsub_rn(__fmul_rn(expf(-lsum), 8388608.0f), 0.5f));
    }
  }
  const QuadRange<C> R = quad_range<C>(n, lane, nc);
  if (__all_sync(kFull, lane >= nc || wu > 0.f)) {
    // every cell of the chunk has a common weight: the decision is the
    // integer compare alone. Two quads per lane and pass, so that two
    // independent Philox chains are in flight.
    for (int g0 = 0; g0 < R.total; g0 += 64) {
      int g[2], cell[2], q[2], nj[2], cthr[2];
      float cls[2];
      uint4 r[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        g[h] = g0 + 32 * h + lane;
        const int lc = quad_cell(R, g[h]);
        const int qb = __shfl_sync(kFull, R.qoff, lc);
        const int nn = __shfl_sync(kFull, n, lc);
        cthr[h] = __shfl_sync(kFull, thr, lc);
        cls[h] = __shfl_sync(kFull, lsum, lc);
        cell[h] = c0 + lc;
        q[h] = g[h] - qb;
        nj[h] = min(4, nn - 4 * q[h]);
        r[h] = philox4x32_10(make_uint4(step, A.cell_base + (uint32_t)cell[h], (uint32_t)q[h], S_EMIT_E << 24), A.rk);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (g[h] >= R.total) continue;
        const long b = (long)cell[h] * A.e.cap + 4 * q[h];
        uint32_t nib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t wj = word(r[h], j);
          if (j < nj[h] && (int)(wj >> 9) > cthr[h]) {
            A.recE[b + j] = (uint32_t)poisson_inv(u23(wj), cls[h]);
            nib |= 1u << j;
          }
        }
        flag_quad(A.bitsE, A.We, cell[h], q[h], nib);
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
      const float4 w4 = ld4(A.e.w + b);
      const float rsum = ((eC ? ccc : 0.f) + (eB ? ccb : 0.f)) * 1.0001f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float wj = f4(w4, j);
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
    ap = __ldg(rec + R_AP);
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
      const float4 w4 = ld4(A.g.w + b), x4 = ld4(A.g.px + b), y4 = ld4(A.g.py + b), z4 = ld4(A.g.pz + b);
      r = philox4x32_10(make_uint4(step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_PRIM_FWD << 24), A.rk);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float px = f4(x4, j), py = f4(y4, j), pz = f4(z4, j);
        const float p2 = px * px + py * py + pz * pz;
        if (j < nj && !no_conversion(f4(w4, j), p2, cs, ca, A.inv_w_a, u23(word(r, j)), A.lam_cap, A.guard_margin))
          nib |= 1u << j;
      }
      flag_quad(A.bitsG, A.Wg, cell, q, nib);
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
    apinv = __ldg(rec + R_APINV);
    invT = __ldg(rec + R_INVT);
    r_bc = __ldg(rec + R_BC);
    r_bb = __ldg(rec + R_BB);
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
      const float4 w4 = ld4(A.a.w + b), x4 = ld4(A.a.px + b), y4 = ld4(A.a.py + b), z4 = ld4(A.a.pz + b);
      if (prim) rP = philox4x32_10(make_uint4(step, gcell, (uint32_t)q, S_PRIM_INV << 24), A.rk);
      if (bath) rA = philox4x32_10(make_uint4(step, gcell, (uint32_t)q, S_ABSORB << 24), A.rk);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float px = f4(x4, j), py = f4(y4, j), pz = f4(z4, j);
        const float p2 = px * px + py * py + pz * pz;
        bool fast = !all;
        if (fast && prim)
          fast = no_conversion(f4(w4, j), p2, cs, cap_inv, A.inv_w_gref, u23(word(rP, j)), A.lam_cap, A.guard_margin);
        if (fast && bath) fast = no_absorption(cbc, cbb, A, mask, sqrtf(p2) * kMeC2f * cinvT, u23(word(rA, j)));
        if (j < nj && !fast) nib |= 1u << j;
      }
      flag_quad(A.bitsA, A.Wa, cell, q, nib);
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
  int pa = 0, pg = 0;
  for (int ch = blockIdx.x * kDecWarps + wid; ch < nchunks; ch += nwarps) {
    const int c0 = ch * C;
    const int nc = min(C, A.ncells - c0);
    if (kinds & DK_ELECTRON) electron_chunk<C>(A, step, c0, nc, lane);
    if (kinds & DK_PHOTON) pg = photon_chunk<C>(A, step, c0, nc, lane, L.g[wid], pg);
    if (kinds & DK_AXION) pa = axion_chunk<C>(A, step, c0, nc, lane, L.a[wid], pa);
  }
  if (lane < pg) photon_full(A, L.g[wid][lane]);
  if (lane < pa) axion_full(A, L.a[wid][lane]);
}

// ---------------------------------------------------------------- event kernel
// Per-warp shared scratch: ascending lists of flagged slots and of removed
// slots (u16), and removed-slot bit masks.
// Flagged items staged in shared memory by asynchronous copies (no register
// holds a load in flight): the first 32 flagged axions and photons of a cell,
// and the first 32 tail positions of each species' tail fill.
struct Fields7 {
  float w[32], px[32], py[32], pz[32], x[32], y[32], z[32];
};
struct EvStage {
  uint4 ar[32];
  Fields7 a;  // flagged axions; then the axion tail-fill movers
  uint4 gr[32];
  Fields7 g;   // flagged photons (w unused)
  Fields7 mg;  // photon tail-fill movers
};

// Per-warp scratch: flagged-slot lists (the removed lists reuse them: a
// chunk's entries are read before removed entries at or below their index
// are written), removed-slot bits and the stage.
struct EvScratch {
  uint16_t *flA, *flG, *flE, *rmA, *rmG;
  uint32_t *rbA, *rbG;
  EvStage* st;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t ev_scratch_bytes(int acap, int gcap, int ecap) {
  size_t b = align16(2 * ((size_t)acap + (size_t)gcap + (size_t)ecap));
  b = align16(b + 4 * (size_t)((acap + 31) / 32 + (gcap + 31) / 32));
  return b + sizeof(EvStage);
}

__device__ inline EvScratch ev_carve(unsigned char* base, int acap, int gcap, int ecap) {
  EvScratch s;
  uint16_t* h = reinterpret_cast<uint16_t*>(base);
  s.flA = h; h += acap;
  s.flG = h; h += gcap;
  s.flE = h; h += ecap;
  s.rmA = s.flA;
  s.rmG = s.flG;
  uint32_t* u = reinterpret_cast<uint32_t*>(base + align16(2 * ((size_t)acap + gcap + ecap)));
  s.rbA = u; u += (acap + 31) / 32;
  s.rbG = u;
  s.st = reinterpret_cast<EvStage*>(base + align16(align16(2 * ((size_t)acap + gcap + ecap)) +
                                                   4 * (size_t)((acap + 31) / 32 + (gcap + 31) / 32)));
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

// Reads and clears the cell's bit-mask words covering [0, n) and writes the
// flagged slots in ascending order to `list`. Returns their number.
__device__ __noinline__ int gather_flags(uint32_t* bits, int W, int cell, int n, uint16_t* list) {
  const int lane = lane_id();
  const int nw = (n + 31) >> 5;
  uint32_t* row = bits + (size_t)cell * W;
  int total = 0;
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int wi = w0 + lane;
    const uint32_t v = wi < nw ? row[wi] : 0u;
    if (v) row[wi] = 0u;
    total = list_flags(v, wi, nw, n, list, total);
  }
  return total;
}

// Tail fill with the ascending removed list: holes are the removed slots
// below n_surv, movers the kept slots at or beyond it, matched in order. The
// movers of the first 32 positions of the tail [n_surv, n) are staged by
// mover_stage (so that their copies are in flight with other work) and
// written by mover_commit; compact_rest moves the positions from n_surv + 32
// on.
// Stages the movers of the first 32 tail positions; *dst is the slot this
// lane's mover fills (or -1). Returns the number of movers staged.
__device__ __forceinline__ int mover_stage(const SpeciesPtrs& s, long base, const uint16_t* rm, const uint32_t* rb,
                                           int n_surv, int n, Fields7& F, int* dst) {
  const int lane = lane_id();
  const int i = n_surv + lane;
  const bool mv = i < n && !bit(rb, i);
  const unsigned msk = __ballot_sync(kFull, mv);
  *dst = -1;
  if (mv) {
    const long src = base + i;
    *dst = rm[__popc(msk & ((1u << lane) - 1u))];
    cp_async4(&F.w[lane], s.w + src);
    cp_async4(&F.px[lane], s.px + src);
    cp_async4(&F.py[lane], s.py + src);
    cp_async4(&F.pz[lane], s.pz + src);
    cp_async4(&F.x[lane], s.x + src);
    cp_async4(&F.y[lane], s.y + src);
    cp_async4(&F.z[lane], s.z + src);
  }
  return __popc(msk);
}

__device__ __forceinline__ void mover_commit(const SpeciesPtrs& s, long base, const Fields7& F, int dst) {
  const int lane = lane_id();
  if (dst >= 0) write_particle(s, base + dst, F.w[lane], F.px[lane], F.py[lane], F.pz[lane], F.x[lane], F.y[lane], F.z[lane]);
}

__device__ __noinline__ void compact_rest(const SpeciesPtrs& s, long base, const uint16_t* rm, int run,
                                          const uint32_t* rb, int n_surv, int n) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  for (int b0 = n_surv + 32; b0 < n; b0 += 32) {
    const int i = b0 + lane;
    const bool mv = i < n && !bit(rb, i);
    const unsigned m = __ballot_sync(kFull, mv);
    if (mv) {
      const long src = base + i;
      const long dst = base + rm[run + __popc(m & lt)];
      write_particle(s, dst, s.w[src], s.px[src], s.py[src], s.pz[src], s.x[src], s.y[src], s.z[src]);
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

__device__ __forceinline__ AxItem ax_load(const StepArgs& A, long base, const uint16_t* fl, int i, int n) {
  AxItem t;
  t.slot = -1;
  t.r = make_uint4(0, 0, 0, 0);
  t.w = t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (i < n) {
    t.slot = fl[i];
    const long src = base + t.slot;
    t.r = A.recA[src];
    t.w = A.a.w[src];
    t.px = A.a.px[src];
    t.py = A.a.py[src];
    t.pz = A.a.pz[src];
    t.x = A.a.x[src];
    t.y = A.a.y[src];
    t.z = A.a.z[src];
  }
  return t;
}

__device__ __forceinline__ PhItem ph_load(const StepArgs& A, long base, const uint16_t* fl, int i, int n) {
  PhItem t;
  t.slot = -1;
  t.r = make_uint4(0, 0, 0, 0);
  t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (i < n) {
    t.slot = fl[i];
    const long src = base + t.slot;
    t.r = A.recG[src];
    t.px = A.g.px[src];
    t.py = A.g.py[src];
    t.pz = A.g.pz[src];
    t.x = A.g.x[src];
    t.y = A.g.y[src];
    t.z = A.g.z[src];
  }
  return t;
}

__device__ __forceinline__ AxItem ax_staged(const EvStage& T, const uint16_t* fl, int lane, int n) {
  AxItem t;
  t.slot = -1;
  t.r = make_uint4(0, 0, 0, 0);
  t.w = t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (lane < n) {
    t.slot = fl[lane];
    t.r = T.ar[lane];
    t.w = T.a.w[lane];
    t.px = T.a.px[lane];
    t.py = T.a.py[lane];
    t.pz = T.a.pz[lane];
    t.x = T.a.x[lane];
    t.y = T.a.y[lane];
    t.z = T.a.z[lane];
  }
  return t;
}

__device__ __forceinline__ PhItem ph_staged(const EvStage& T, const uint16_t* fl, int lane, int n) {
  PhItem t;
  t.slot = -1;
  t.r = make_uint4(0, 0, 0, 0);
  t.px = t.py = t.pz = t.x = t.y = t.z = 0.f;
  if (lane < n) {
    t.slot = fl[lane];
    t.r = T.gr[lane];
    t.px = T.g.px[lane];
    t.py = T.g.py[lane];
    t.pz = T.g.pz[lane];
    t.x = T.g.x[lane];
    t.y = T.g.y[lane];
    t.z = T.g.z[lane];
  }
  return t;
}

__device__ __forceinline__ ElItem el_load(const StepArgs& A, long base, const uint16_t* fl, int i, int n, float wu) {
  ElItem t;
  t.slot = -1;
  t.f = 0u;
  t.w = wu;
  t.x = t.y = t.z = 0.f;
  if (i < n) {
    t.slot = fl[i];
    const long src = base + t.slot;
    t.f = A.recE[src];
    t.x = A.e.x[src];
    t.y = A.e.y[src];
    t.z = A.e.z[src];
    if (wu <= 0.f) t.w = A.e.w[src];
  }
  return t;
}

// One cell's events, by one warp. Round trips: (1) counts, decision masks,
// per-cell constants and the exchange buffer; (2) the records and fields of
// the flagged slots of every species; (3) the tail-fill movers of both
// species; then the stores. Output order is the method's: photon products of
// a->gamma after the photons present, axion products of gamma->a after the
// surviving axions, then the thermal-bath products in electron then event
// order; removed slots are refilled from the tail.
template <int PH>
__device__ __forceinline__ void event_cell(const StepArgs& A, uint32_t step, int cell, EvScratch& S, const Cnt& cnt) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t gcell = A.cell_base + (uint32_t)cell;
  const int mask = A.mask;
  const bool prim = mask & AXPIC_CH_PRIMAKOFF;
  const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
  const bool emitG = (PH & PH_EMIT) && prim;
  const bool emitE = (PH & PH_EMIT) && (eC || eB);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;

  // ------------------------------------------------------------ round trip 1
  const int ne = min(max(A.e.count[cell], 0), A.e.cap);
  const int ng_start = min(max(A.g.count[cell], 0), A.g.cap);
  const int na_start = min(max(A.a.count[cell], 0), A.a.cap);
  const int pstart = (!(PH & PH_ABSORB) && A.use_snapshot) ? A.photon_start[cell] : 0;
  float wu = 0.f, r_cc = 0.f, r_cb = 0.f, r_T = 0.f;
  if (emitE) {
    const float* rec = A.rec + (size_t)cell * kRecLen;
    wu = A.mom[(size_t)cell * kMomLen + M_WU];
    r_cc = rec[R_CC];
    r_cb = rec[R_CB];
    r_T = rec[R_T];
  }
  // lanes 0..3 hold one component each of the cell's exchange buffer
  double* xb = A.xbuf + (size_t)cell * 4;
  const double xb_old = lane < 4 ? xb[lane] : 0.0;
  int nflA = 0, nflG = 0, nflE = 0;
  const int ng0 = (PH & PH_ABSORB) ? ng_start : (A.use_snapshot ? min(pstart, ng_start) : ng_start);
  {
    // whole mask rows are loaded without waiting for the counts: bits beyond
    // a count are never set
    if (A.Wa <= 32 && A.Wg <= 32 && A.We <= 32) {
      uint32_t* rA = A.bitsA + (size_t)cell * A.Wa;
      uint32_t* rG = A.bitsG + (size_t)cell * A.Wg;
      uint32_t* rE = A.bitsE + (size_t)cell * A.We;
      const uint32_t vA = (PH & PH_ABSORB) && lane < A.Wa ? rA[lane] : 0u;
      const uint32_t vG = emitG && lane < A.Wg ? rG[lane] : 0u;
      const uint32_t vE = emitE && lane < A.We ? rE[lane] : 0u;
      if (vA) rA[lane] = 0u;
      if (vG) rG[lane] = 0u;
      if (vE) rE[lane] = 0u;
      if (__any_sync(kFull, vA != 0)) nflA = list_flags(vA, lane, (na_start + 31) >> 5, na_start, S.flA, 0);
      if (__any_sync(kFull, vG != 0)) nflG = list_flags(vG, lane, (ng0 + 31) >> 5, ng0, S.flG, 0);
      if (__any_sync(kFull, vE != 0)) nflE = list_flags(vE, lane, (ne + 31) >> 5, ne, S.flE, 0);
    } else {
      if (PH & PH_ABSORB) nflA = gather_flags(A.bitsA, A.Wa, cell, na_start, S.flA);
      if (emitG) nflG = gather_flags(A.bitsG, A.Wg, cell, ng0, S.flG);
      if (emitE) nflE = gather_flags(A.bitsE, A.We, cell, ne, S.flE);
    }
    __syncwarp();
  }
  // particles present at the start of the step: counted by the absorb phase,
  // or by the emit phase when no absorb ran this step
  if (lane == 0 && ((PH & PH_ABSORB) || ((PH & PH_EMIT) && !A.use_snapshot))) {
    cnt.add(C_NE, ne);
    cnt.add(C_NG, ng_start);
    cnt.add(C_NA, na_start);
    cnt.add(C_CELLS, 1);
  }
  if ((PH & PH_ABSORB) && lane == 0) A.photon_start[cell] = ng_start;

  // ------------------------------------------------------------ round trip 2
  // records and fields of the first 32 flagged axions and photons, staged by
  // asynchronous copies
  EvStage& T = *S.st;
  if ((PH & PH_ABSORB) && lane < nflA) {
    const long src = abase + S.flA[lane];
    cp_async16(&T.ar[lane], A.recA + src);
    cp_async4(&T.a.w[lane], A.a.w + src);
    cp_async4(&T.a.px[lane], A.a.px + src);
    cp_async4(&T.a.py[lane], A.a.py + src);
    cp_async4(&T.a.pz[lane], A.a.pz + src);
    cp_async4(&T.a.x[lane], A.a.x + src);
    cp_async4(&T.a.y[lane], A.a.y + src);
    cp_async4(&T.a.z[lane], A.a.z + src);
  }
  if (emitG && lane < nflG) {
    const long src = gbase + S.flG[lane];
    cp_async16(&T.gr[lane], A.recG + src);
    cp_async4(&T.g.px[lane], A.g.px + src);
    cp_async4(&T.g.py[lane], A.g.py + src);
    cp_async4(&T.g.pz[lane], A.g.pz + src);
    cp_async4(&T.g.x[lane], A.g.x + src);
    cp_async4(&T.g.y[lane], A.g.y + src);
    cp_async4(&T.g.z[lane], A.g.z + src);
  }
  cp_async_wait_all();
  __syncwarp();

  Lane64 x64;
  double xa[4] = {0.0, 0.0, 0.0, 0.0};
  bool xa_any = false;
  int ng = ng_start, na = na_start, nrmA = 0;

  // ------------------------------------------------------------ absorb
  if ((PH & PH_ABSORB) && nflA > 0) {
    for (int i = lane; i < (na_start + 31) / 32; i += 32) S.rbA[i] = 0u;
    __syncwarp();
    int run = 0, NPg = 0;
    for (int i0 = 0; i0 < nflA; i0 += 32) {
      const AxItem t = i0 == 0 ? ax_staged(T, S.flA, lane, nflA) : ax_load(A, abase, S.flA, i0 + lane, nflA);
      int K = 0;
      bool removed = false;
      float wprod = 0.f;
      if (t.slot >= 0) {
        K = t.r.x & 0xFF;
        wprod = __uint_as_float(t.r.y);
        const float wnew = __uint_as_float(t.r.z);
        const float om = sqrtf(t.px * t.px + t.py * t.py + t.pz * t.pz) * kMeC2f;
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
        removed = !(t.r.x & DF_KEEP);
        if (!removed && wnew != t.w) A.a.w[abase + t.slot] = wnew;
      }
      // photon products of a->gamma after the photons present
      int tot;
      int off = run + warp_excl_scan(K, &tot);
      for (int k = 0; k < K; ++k, ++off) {
        const int dst = ng + off;
        if (dst < A.g.cap) write_particle(A.g, gbase + dst, wprod, t.px, t.py, t.pz, t.x, t.y, t.z);
        else cnt.add(C_DROP, 1);
      }
      run += tot;
      NPg += K;
      const unsigned m = __ballot_sync(kFull, removed);
      if (removed) {
        S.rmA[nrmA + __popc(m & lt)] = (uint16_t)t.slot;
        atomicOr(&S.rbA[t.slot >> 5], 1u << (t.slot & 31));
      }
      nrmA += __popc(m);
    }
    NPg = warp_sum_i(NPg);
    ng = min(ng + NPg, A.g.cap);
    if (__any_sync(kFull, x64.any)) {
      xa[0] = warp_sum_d(x64.dE);
      xa[1] = warp_sum_d(x64.dPx);
      xa[2] = warp_sum_d(x64.dPy);
      xa[3] = warp_sum_d(x64.dPz);
      xa_any = true;
    }
    x64 = Lane64();
    na = na_start - nrmA;
  }

  // ------------------------------------------------------------ emit: photons
  const int ng_tot = ng;
  int nrmG = 0, NPa = 0;
  float pw_prod = 0.f;
  int pK = 0, p_off = 0;
  if (emitG && nflG > 0) {
    for (int i = lane; i < (ng_tot + 31) / 32; i += 32) S.rbG[i] = 0u;
    __syncwarp();
    // decisions of the first 32 (products are written after the axion tail
    // fill); longer lists are taken whole below
    if (nflG <= 32) {
      bool removed = false;
      int slot = -1;
      if (lane < nflG) {
        slot = S.flG[lane];
        const uint4 r = T.gr[lane];
        pK = r.x & 0xFF;
        pw_prod = __uint_as_float(r.y);
        cnt.add(C_CAP, (r.x & DF_CAPPED) ? 1u : 0u);
        cnt.add(C_CLAMP, (r.x & DF_OVER) ? 1u : 0u);
        cnt.add(C_EV_P, (unsigned)pK);
        removed = !(r.x & DF_KEEP);
        if (pK && !removed) A.g.w[gbase + slot] = __uint_as_float(r.z);
      }
      int tot;
      p_off = warp_excl_scan(pK, &tot);
      NPa = tot;
      const unsigned m = __ballot_sync(kFull, removed);
      if (removed) {
        S.rmG[__popc(m & lt)] = (uint16_t)slot;
        atomicOr(&S.rbG[slot >> 5], 1u << (slot & 31));
      }
      nrmG = __popc(m);
    }
  }
  __syncwarp();

  // ------------------------------------------------------------ round trip 3
  // tail-fill movers of both species (axion movers are read before any
  // product is written over them)
  int runA = 0, runG = 0, dA = -1, dG = -1;
  const bool fillA = (PH & PH_ABSORB) && nrmA > 0;
  const bool fillG = emitG && nflG <= 32 && nrmG > 0;
  if (fillA) runA = mover_stage(A.a, abase, S.rmA, S.rbA, na, na_start, T.a, &dA);
  if (fillG) runG = mover_stage(A.g, gbase, S.rmG, S.rbG, ng_tot - nrmG, ng_tot, T.mg, &dG);
  if (fillA || fillG) {
    cp_async_wait_all();
    __syncwarp();
  }
  if (fillA) {
    mover_commit(A.a, abase, T.a, dA);
    if (na_start - na > 32) compact_rest(A.a, abase, S.rmA, runA, S.rbA, na, na_start);
  }

  if (PH & PH_EMIT) {
    const int abase_new = na;
    // (c) gamma->a products after the surviving axions
    if (emitG && nflG > 0) {
      if (nflG <= 32) {
        if (pK) {
          const float px = T.g.px[lane], py = T.g.py[lane], pz = T.g.pz[lane];
          const float xx = T.g.x[lane], yy = T.g.y[lane], zz = T.g.z[lane];
          const float om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
          int off = p_off;
          for (int k = 0; k < pK; ++k, ++off) {
            const int dst = abase_new + off;
            if (dst < A.a.cap) {
              write_particle(A.a, abase + dst, pw_prod, px, py, pz, xx, yy, zz);
              if (A.tally_enable) tally_add(A, 0, pw_prod, om);
            } else {
              cnt.add(C_DROP, 1);
            }
          }
        }
      } else {
        int run = 0;
        for (int i0 = 0; i0 < nflG; i0 += 32) {
          const PhItem t = i0 == 0 ? ph_staged(T, S.flG, lane, nflG) : ph_load(A, gbase, S.flG, i0 + lane, nflG);
          int K = 0;
          bool removed = false;
          float wprod = 0.f, om = 0.f;
          if (t.slot >= 0) {
            K = t.r.x & 0xFF;
            wprod = __uint_as_float(t.r.y);
            cnt.add(C_CAP, (t.r.x & DF_CAPPED) ? 1u : 0u);
            cnt.add(C_CLAMP, (t.r.x & DF_OVER) ? 1u : 0u);
            cnt.add(C_EV_P, (unsigned)K);
            removed = !(t.r.x & DF_KEEP);
            if (K) {
              om = sqrtf(t.px * t.px + t.py * t.py + t.pz * t.pz) * kMeC2f;
              if (!removed) A.g.w[gbase + t.slot] = __uint_as_float(t.r.z);
            }
          }
          int tot;
          int off = run + warp_excl_scan(K, &tot);
          for (int k = 0; k < K; ++k, ++off) {
            const int dst = abase_new + off;
            if (dst < A.a.cap) {
              write_particle(A.a, abase + dst, wprod, t.px, t.py, t.pz, t.x, t.y, t.z);
              if (A.tally_enable) tally_add(A, 0, wprod, om);
            } else {
              cnt.add(C_DROP, 1);
            }
          }
          run += tot;
          NPa += K;
          const unsigned m = __ballot_sync(kFull, removed);
          if (removed) {
            S.rmG[nrmG + __popc(m & lt)] = (uint16_t)t.slot;
            atomicOr(&S.rbG[t.slot >> 5], 1u << (t.slot & 31));
          }
          nrmG += __popc(m);
        }
        NPa = warp_sum_i(NPa);
      }
    }
    // (d) electron events, in electron then event order; event k of
    // electron i: cos theta, phi, energy and channel from one Philox block
    int NE = 0;
    if (emitE) {
      if (wu > 0.f && lane == 0) {
        float fac;
        bool cc = false, cb = false;
        if (eC) cap_lambda(wu * r_cc, A.lam_cap, &fac, &cc);
        if (eB) cap_lambda(wu * r_cb, A.lam_cap, &fac, &cb);
        cnt.add(C_CAP, (unsigned)ne * ((unsigned)cc + (unsigned)cb));
      }
      if (nflE > 0) {
        const float* tabC = A.tables + TAB_COMPTON * kTableN;
        const float* tabB = A.tables + TAB_BREMS * kTableN;
        int run = 0;
        for (int i0 = 0; i0 < nflE; i0 += 32) {
          const ElItem t = el_load(A, ebase, S.flE, i0 + lane, nflE, wu);
          int K = 0;
          if (t.slot >= 0) {
            K = t.f & 0xFF;
            if (wu <= 0.f) cnt.add(C_CAP, ((t.f & DF_CAPPED) ? 1u : 0u) + ((t.f & DF_CAPPED_B) ? 1u : 0u));
          }
          int tot;
          int off = run + warp_excl_scan(K, &tot);
          if (K) {
            float facC = 1.f, facB = 1.f;
            bool cc = false, cb = false;
            const float lc = eC ? cap_lambda(t.w * r_cc, A.lam_cap, &facC, &cc) : 0.f;
            const float lb = eB ? cap_lambda(t.w * r_cb, A.lam_cap, &facB, &cb) : 0.f;
            const float fracC = lc / (lc + lb);
            const float wvC = cc ? A.w_a * facC : A.w_a;
            const float wvB = cb ? A.w_a * facB : A.w_a;
            for (int k = 0; k < K; ++k, ++off) {
              const uint4 r = philox4x32_10(make_uint4(step, gcell, (uint32_t)t.slot, (S_EV_E << 24) | (uint32_t)k),
                                            A.rk);
              const bool isC = u23(r.w) < fracC;
              const float3 dv = iso_dir(u23(r.x), u23(r.y));
              const float E = (A.rate_model ? sr_sample_x(A.sr + (size_t)cell * kSrLen, isC ? 1 : 2, u23(r.z))
                                            : icdf_lookup(isC ? tabC : tabB, u23(r.z))) *
                              r_T;
              const float wv = isC ? wvC : wvB;
              const float pm = E * kInvMeC2f;
              const float px = pm * dv.x, py = pm * dv.y, pz = pm * dv.z;
              const int dst = abase_new + NPa + off;
              if (dst < A.a.cap) {
                write_particle(A.a, abase + dst, wv, px, py, pz, t.x, t.y, t.z);
                if (A.tally_enable) tally_add(A, isC ? 1 : 2, wv, E);
              } else {
                cnt.add(C_DROP, 1);
              }
              x64.add(-(double)wv, E, px, py, pz);
              cnt.add(isC ? C_EV_C : C_EV_B, 1);
            }
          }
          run += tot;
          NE += K;
        }
        NE = warp_sum_i(NE);
      }
    }
    na = min(na + NPa + NE, A.a.cap);
    __syncwarp();
    // (e) tail fill of the photons (a->gamma products included)
    if (fillG) {
      mover_commit(A.g, gbase, T.mg, dG);
      if (nrmG > 32) compact_rest(A.g, gbase, S.rmG, runG, S.rbG, ng_tot - nrmG, ng_tot);
    } else if (emitG && nflG > 32 && nrmG > 0) {
      int d = -1;
      const int run0 = mover_stage(A.g, gbase, S.rmG, S.rbG, ng_tot - nrmG, ng_tot, T.mg, &d);
      cp_async_wait_all();
      __syncwarp();
      mover_commit(A.g, gbase, T.mg, d);
      if (nrmG > 32) compact_rest(A.g, gbase, S.rmG, run0, S.rbG, ng_tot - nrmG, ng_tot);
    }
    ng = ng_tot - nrmG;
  }
  if (lane == 0) {
    A.a.count[cell] = na;
    A.g.count[cell] = ng;
  }

  // ------------------------------------------------------------ exchange
  // the absorb and emit contributions are reduced separately and added to the
  // cell's buffer in that order, whichever way the step was called
  bool xe_any = false;
  double xe[4] = {0.0, 0.0, 0.0, 0.0};
  if (__any_sync(kFull, x64.any)) {
    xe[0] = warp_sum_d(x64.dE);
    xe[1] = warp_sum_d(x64.dPx);
    xe[2] = warp_sum_d(x64.dPy);
    xe[3] = warp_sum_d(x64.dPz);
    xe_any = true;
  }
  if (lane < 4 && (xa_any || xe_any)) {
    const double a = lane == 0 ? xa[0] : (lane == 1 ? xa[1] : (lane == 2 ? xa[2] : xa[3]));
    const double e = lane == 0 ? xe[0] : (lane == 1 ? xe[1] : (lane == 2 ? xe[2] : xe[3]));
    double v = xb_old;
    if (xa_any) v += a;
    if (xe_any) v += e;
    xb[lane] = v;
  }
}

#ifndef AXPIC_EVENT_MIN_CTAS
#define AXPIC_EVENT_MIN_CTAS 8
#endif

template <int PH>
__global__ void __launch_bounds__(128, AXPIC_EVENT_MIN_CTAS) event_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long warp_cnt[4][kNumCounters];
  const int wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * nw + wid;
  if (lane < kNumCounters) warp_cnt[wid][lane] = 0ull;
  __syncwarp();
  const Cnt cnt{warp_cnt[wid]};
  if (cell < A.ncells) {
    const size_t bytes = ev_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
    EvScratch S = ev_carve(smem + wid * bytes, A.a.cap, A.g.cap, A.e.cap);
    event_cell<PH>(A, step_of(A), cell, S, cnt);
  }
  __syncwarp();
  if (lane < kNumCounters) {
    const unsigned long long v = warp_cnt[wid][lane];
    if (v) atomicAdd(A.counters + (size_t)(blockIdx.x % A.ctr_rows) * kNumCounters + lane, v);
    if (lane == C_DROP && v) atomicOr(A.err, ERR_CAPACITY);
  }
}

// ---------------------------------------------------------------- feedback kernel
// One lane per cell: the exchange of this step plus the carried part; when it
// is representable in binary32 momenta the whole warp remaps that cell's
// electrons (Eqs. delta_def to b_def, affine_map), measuring what was applied;
// then the temperature update (Eqs. Te_est, Te_relax) and the record's
// temperature half.
struct RemapJob {
  int cell, ne;
  float s1, bx, by, bz;
};

// Thread per cell: every load it needs is issued first (exchange, carried
// exchange, moments, count, T and the record); cells whose exchange needs an
// affine remap go to a CTA list and the CTA's warps remap them side by side,
// a warp per cell; then each thread finishes its cell (carry, diagnostics,
// temperature update and the record's temperature half).
constexpr int kFeedbackThreads = 128;

__global__ void __launch_bounds__(kFeedbackThreads) feedback_kernel(StepArgs A) {
  // a replayed graph takes its step index from the device counter: the last
  // kernel of the step advances it (no kernel of this launch reads it)
  if (A.step_dev && blockIdx.x == 0 && threadIdx.x == 0) *A.step_dev += 1u;
  __shared__ RemapJob jobs[kFeedbackThreads];
  __shared__ RemapOut outs[kFeedbackThreads];
  __shared__ int njobs;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < A.ncells;
  if (threadIdx.x == 0) njobs = 0;
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0, rE = 0.0, rPx = 0.0, rPy = 0.0, rPz = 0.0, T = 0.0;
  float W = 0.f, Px = 0.f, Py = 0.f, Pz = 0.f, U2 = 0.f, var = 0.f;
  float4 rc0 = make_float4(0.f, 0.f, 0.f, 0.f), rc1 = rc0, rc2 = rc0, rc3 = rc0;
  bool has_x = false, has_res = false, need = false;
  int ne = 0;
  double qE = 0.0, qPx = 0.0, qPy = 0.0, qPz = 0.0, s1d = 0.0, bx = 0.0, by = 0.0, bz = 0.0, vnd = 0.0;
  if (valid) {
    double* xb = A.xbuf + (size_t)cell * 4;
    dE = xb[0];
    dPx = xb[1];
    dPy = xb[2];
    dPz = xb[3];
    const double* rs = A.res + (size_t)cell * 4;
    rE = rs[0];
    rPx = rs[1];
    rPy = rs[2];
    rPz = rs[3];
    const float* mom = A.mom + (size_t)cell * kMomLen;
    W = mom[M_W];
    Px = mom[M_PX];
    Py = mom[M_PY];
    Pz = mom[M_PZ];
    U2 = mom[M_U2];
    var = mom[M_VAR];
    ne = min(max(A.e.count[cell], 0), A.e.cap);
    if (A.T_mode == 2) {
      T = A.T[cell];
      const float4* r4 = reinterpret_cast<const float4*>(A.rec + (size_t)cell * kRecLen);
      rc0 = r4[0];
      rc1 = r4[1];
      rc2 = r4[2];
      rc3 = r4[3];
    }
    has_x = nz64(dE) || nz64(dPx) || nz64(dPy) || nz64(dPz);
    if (has_x) {
      xb[0] = 0.0;
      xb[1] = 0.0;
      xb[2] = 0.0;
      xb[3] = 0.0;
    }
    has_res = nz64(rE) || nz64(rPx) || nz64(rPy) || nz64(rPz);
    if (has_x || has_res) {
      qE = dE + rE;
      qPx = dPx + rPx;
      qPy = dPy + rPy;
      qPz = dPz + rPz;
      // Exchanges below 2^-22 of the cell's kinetic energy (or momentum
      // spread) cannot be represented by binary32 momenta; they stay pending.
      const float ekin = 0.5f * U2 * kMeC2f;
      const float prms = sqrtf(fmaxf(U2 * W, 0.f));
      need = W > 0.f && (fabsf((float)qE) >= 2.384185791015625e-07f * ekin ||
                         sqrtf((float)(qPx * qPx + qPy * qPy + qPz * qPz)) >= 2.384185791015625e-07f * prms);
      if (need) {
        // Eqs. delta_def, dE_bulk, dE_th, var_new, s_def, b_def (mu = 1)
        const double Wd = W;
        const double dx = qPx / Wd, dy = qPy / Wd, dz = qPz / Wd;
        const double dEb = (2.0 * (dx * Px + dy * Py + dz * Pz) + Wd * (dx * dx + dy * dy + dz * dz)) * 0.5;
        const double dEth = qE / kMeC2 - dEb;
        vnd = var;
        if (var > 0.f) {
          vnd = fmax(0.0, (double)var + 2.0 * dEth);
          const double S = sqrt(vnd / (double)var);
          s1d = ((vnd - (double)var) / (double)var) / (S + 1.0);
        }
        bx = -s1d * Px / Wd + dx;
        by = -s1d * Py / Wd + dy;
        bz = -s1d * Pz / Wd + dz;
      }
    }
  }
  __syncthreads();
  int job = -1;
  if (need) {
    job = atomicAdd(&njobs, 1);
    jobs[job] = RemapJob{cell, ne, (float)s1d, (float)bx, (float)by, (float)bz};
  }
  __syncthreads();
  const int nj = njobs;
  for (int k = wid; k < nj; k += kFeedbackThreads / 32) {
    const RemapJob J = jobs[k];
    const RemapOut r = remap_electrons(A, (long)J.cell * A.e.cap, J.ne, J.s1, J.bx, J.by, J.bz);
    if (lane == 0) outs[k] = r;
  }
  __syncthreads();
  if (!valid) return;
  double nrE = qE, nrPx = qPx, nrPy = qPy, nrPz = qPz, applied_E = 0.0;
  float var_new = var;
  if (job >= 0) {
    const RemapOut r = outs[job];
    applied_E = r.applied_E;
    nrE = qE - r.applied_E;
    nrPx = qPx - r.apx;
    nrPy = qPy - r.apy;
    nrPz = qPz - r.apz;
    var_new = (float)vnd;
    float* mom = A.mom + (size_t)cell * kMomLen;
    mom[M_W] = r.mW;
    mom[M_PX] = r.mPx;
    mom[M_PY] = r.mPy;
    mom[M_PZ] = r.mPz;
    mom[M_U2] = r.mU2;
    mom[M_VAR] = fmaxf(0.f, r.mU2 - (r.mPx * r.mPx + r.mPy * r.mPy + r.mPz * r.mPz) / r.mW);
  }
  if (has_x || has_res) {
    double* rs = A.res + (size_t)cell * 4;
    rs[0] = nrE;
    rs[1] = nrPx;
    rs[2] = nrPy;
    rs[3] = nrPz;
  }
  if (need) {
    atomicAdd(A.counters + C_REMAP, 1ull);
    atomicAdd(A.counters + C_REMAP_E, (unsigned long long)ne);
  }
  if (A.diag_enable) {
    double* dg = A.diag + (size_t)cell * AXPIC_CELL_DIAG_LEN;
    dg[AXPIC_CD_DE] = dE;
    dg[AXPIC_CD_DPX] = dPx;
    dg[AXPIC_CD_DPY] = dPy;
    dg[AXPIC_CD_DPZ] = dPz;
    dg[AXPIC_CD_S_MINUS_1] = s1d;
    dg[AXPIC_CD_BX] = bx;
    dg[AXPIC_CD_BY] = by;
    dg[AXPIC_CD_BZ] = bz;
    dg[AXPIC_CD_VAR] = var;
    dg[AXPIC_CD_VAR_NEW] = need ? vnd : (double)var;
    dg[AXPIC_CD_W] = W;
    dg[AXPIC_CD_APPLIED_E] = applied_E;
    dg[AXPIC_CD_RES_E] = has_x || has_res ? nrE : 0.0;
    dg[AXPIC_CD_RES_PX] = has_x || has_res ? nrPx : 0.0;
    dg[AXPIC_CD_RES_PY] = has_x || has_res ? nrPy : 0.0;
    dg[AXPIC_CD_RES_PZ] = has_x || has_res ? nrPz : 0.0;
  }
  // temperature (Eqs. Te_est, Te_relax), then the record's temperature half;
  // T stays FP64, the relaxation step is formed in binary32 and added once
  if (A.T_mode == 2 && W > 0.f) {
    const float Tf = (float)T;
    const float Test = (kMeC2f / 3.0f) * var_new / W;
    const float dT = A.relax_r * (Test - Tf);
    double Tn = T + (double)dT;
    const float Tnf = Tf + dT;
    if (Tnf <= A.T_floor_f || Tnf >= A.T_ceil_f) Tn = fmin(fmax(Tn, A.T_floor), A.T_ceil);
    float rec[kRecLen] = {rc0.x, rc0.y, rc0.z, rc0.w, rc1.x, rc1.y, rc1.z, rc1.w,
                          rc2.x, rc2.y, rc2.z, rc2.w, rc3.x, rc3.y, rc3.z, rc3.w};
    compute_temperature(A.cc, (float)Tn, rec);
    A.T[cell] = Tn;
    float4* r4 = reinterpret_cast<float4*>(A.rec + (size_t)cell * kRecLen);
    r4[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
    r4[1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
  }
}


// ---------------------------------------------------------------- launchers
size_t step_smem_per_warp(int acap, int gcap, int ecap) { return ev_scratch_bytes(acap, gcap, ecap); }

template <int PH>
static cudaError_t launch_events(const StepArgs& A, int warps, cudaStream_t st) {
  const size_t per = ev_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
  const int grid = (A.ncells + warps - 1) / warps;
  event_kernel<PH><<<grid, warps * 32, per * warps, st>>>(A);
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
    case 2:
      decide_kernel<2><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
    case 8:
      decide_kernel<8><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
    default:
      decide_kernel<4><<<dec_blocks(A), kDecThreads, 0, st>>>(A, kinds);
      break;
  }
  return cudaGetLastError();
}

static cudaError_t launch_feedback(const StepArgs& A, cudaStream_t st) {
  feedback_kernel<<<(A.ncells + kFeedbackThreads - 1) / kFeedbackThreads, kFeedbackThreads, 0, st>>>(A);
  return cudaGetLastError();
}

const char* step_kernel_names() { return "decide_kernel,event_kernel,feedback_kernel"; }

__global__ void set_step_kernel(uint32_t* p, uint32_t v) { *p = v; }

cudaError_t launch_set_step(uint32_t* p, uint32_t v, cudaStream_t st) {
  set_step_kernel<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t decide_resident_ctas(int chunk, int* out) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return e;
  if (chunk == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<2>, kDecThreads, 0);
  else if (chunk == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<8>, kDecThreads, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decide_kernel<4>, kDecThreads, 0);
  if (e) return e;
  *out = max(1, nb) * max(1, sms);
  return cudaSuccess;
}

// After the temperature update of an evolved-T step the spectral records are
// rebuilt for the new T (rate models 1 and 2).
static cudaError_t launch_records_update(const StepArgs& A, const SrArgs* sra, cudaStream_t st) {
  if (!sra || A.T_mode != 2) return cudaSuccess;
  cudaError_t e = launch_sr_table(*sra, st);
  if (!e && sra->trust) e = launch_sr_mlp(*sra, st);
  return e;
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
      if ((e = launch_feedback(A, st)) || (e = launch_records_update(A, sra, st)) || (e = mark(3))) return e;
      return cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t set_step_smem_limits(size_t bytes) {
  cudaError_t e;
  const int b = (int)bytes;
  if ((e = cudaFuncSetAttribute(event_kernel<PH_ABSORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) ||
      (e = cudaFuncSetAttribute(event_kernel<PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)) ||
      (e = cudaFuncSetAttribute(event_kernel<PH_ABSORB | PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)))
    return e;
  return cudaSuccess;
}

}  // namespace axpic
