// The per-cell step: absorb -> emit -> feedback (Sec. II.D-II.J).
//
// A step is four kernels:
//  * axion_decide_kernel and emit_decide_kernel: one thread per quad of
//    consecutive slots (float4 loads from the SoA slabs, one Philox4x32-10
//    block per quad and stream, word j for slot 4q+j). Each slot gets a cheap
//    exact test that proves "no event this step"; slots it cannot clear are
//    flagged in a per-cell bit mask. These kernels carry almost all the
//    per-particle work and have no per-cell serialisation.
//  * event_kernel: one warp per cell. It reads only the bit masks, takes the
//    full decision for the flagged slots (few), writes products and compacts
//    at offsets from warp prefix sums, so the output order is the
//    deterministic one of the method's definition, and accumulates the FP64
//    exchange (Delta E, Delta P).
//  * feedback_kernel: one lane per cell for the temperature update; the rare
//    cells whose exchange needs an affine remap are remapped by the whole warp.
// The separate API calls run the same kernels with one phase each; the
// exchange passes through an FP64 per-cell buffer in the same summation order,
// so results do not depend on how a step is called.
#include "common.cuh"
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

// Quads are consumed element by element from .x and then rotated, so that a
// runtime slot index never forces them into local memory.
__device__ __forceinline__ void rot(float4& v) { v = make_float4(v.y, v.z, v.w, v.x); }
__device__ __forceinline__ void rot(uint4& v) { v = make_uint4(v.y, v.z, v.w, v.x); }

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

// ---------------------------------------------------------------- decisions
// One axion at the start of the step: a->gamma conversion (Sec. II.F.1, last
// paragraph) then detailed-balance absorption of the thermal-bath channels
// (Sec. II.I).
struct AxionDecision {
  int K;
  float wprod, wnew, om;
  bool keep, absorbed, capped, over, abs_c;
};

__device__ __forceinline__ AxionDecision axion_decide(const float* rec, const StepArgs& A, int mask, float w, float px,
                                                      float py, float pz, uint32_t wP, uint32_t wA) {
  AxionDecision d;
  d.om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
  d.K = 0;
  d.wprod = 0.f;
  d.capped = false;
  d.over = false;
  d.absorbed = false;
  d.abs_c = false;
  float wrem = w;
  if (mask & AXPIC_CH_PRIMAKOFF) {
    const float P = prim_prob(rec, d.om, rec[R_APINV]);
    float fac;
    const float le = cap_lambda(w * P * A.inv_w_gref, A.lam_cap, &fac, &d.capped);
    d.K = poisson_inv(u23(wP), le);
    if (d.K > 0) d.wprod = deplete(w, d.K, d.capped ? A.w_gref * fac : A.w_gref, &wrem, &d.over);
  }
  d.keep = wrem > 0.f;
  d.wnew = wrem;
  if (d.keep && (mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS))) {
    const float x = d.om * rec[R_INVT];
    const float tc = (mask & AXPIC_CH_COMPTON) ? tau_compton(rec, x, A.eq_stats) : 0.f;
    const float tb = (mask & AXPIC_CH_BREMS) ? tau_brems(rec, x, A.brems_am3, A.eq_stats) : 0.f;
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
  return axion_decide(rec, A, mask, w, px, py, pz, wP, wA);
}

// One photon at the start of the step: gamma->a conversion (Sec. II.F,
// Eqs. prim_rate, prim_prob, lambda_P, depletion).
struct PhotonDecision {
  int K;
  float wprod, wrem, om;
  bool capped, over;
};

__device__ __forceinline__ PhotonDecision photon_decide(const float* rec, const StepArgs& A, float w, float px,
                                                        float py, float pz, uint32_t wd) {
  PhotonDecision d;
  d.om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
  const float P = prim_prob(rec, d.om, rec[R_AP]);
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
  return photon_decide(rec, A, w, px, py, pz, wd);
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
                                              float lam_cap) {
  const float s = p2 * c_s;
  const float Fb = s < 2.5f ? 0.5f * s : __logf(1.0f + s);
  const float lb = w * Acoef * Fb * inv_wref * 1.0001f;
  return lb < lam_cap && u <= 1.0f - lb - 1e-6f;
}

// Absorption: P_abs <= tau; x/(1-e^-x) <= 1 + x bounds the Compton-like
// factor, (1 - e^-x) <= 1 the Bose-Einstein one.
__device__ __forceinline__ bool no_absorption(const float* rec, const StepArgs& A, int mask, float x, float u) {
  float tb = 0.f;
  if (mask & AXPIC_CH_COMPTON) tb += rec[R_BC] * x * (1.0f + x);
  if (mask & AXPIC_CH_BREMS) tb += rec[R_BB] * __expf(A.brems_am3 * __logf(x));
  return u >= tb * 1.001f + 1e-6f;
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

// Decision CTAs take A.dec_cells consecutive cells and give their quads to
// threads in one flat range (thread per quad, cell-major), so uneven counts
// still fill the warps. Slots that the guards cannot clear go to a CTA-wide
// list in shared memory, and their full decisions are taken with the
// list spread over all threads: the out-of-line chain then runs with full
// warps instead of a few lanes of every warp. List order does not matter:
// records are indexed by slot.
constexpr int kDecThreads = 256;
static_assert(AXPIC_DEC_CELLS >= 1 && AXPIC_DEC_CELLS <= kDecMaxCells, "cells per decision CTA");
constexpr int kDecListCap = 5 * kDecThreads;  // one pass of flags (4 per thread) + a partial batch

struct DecideSmem {
  int qoff[kDecMaxCells + 1];  // prefix of the cells' quad counts
  int n[kDecMaxCells];         // slots to decide per cell
  float c0[kDecMaxCells], c1[kDecMaxCells], c2[kDecMaxCells], c3[kDecMaxCells], c4[kDecMaxCells];  // per cell
  int count;
  uint32_t item[kDecListCap];  // (cell in CTA << 16) | slot
  uint2 u[kDecListCap];        // the slot's decision words
};

// Quad counts of this CTA's cells, from the per-cell slot counts n (set by
// lanes < ncell of warp 0 before the call).
__device__ __forceinline__ void dec_prefix(DecideSmem& S, int ncell, int n) {
  if (threadIdx.x < 32) {
    const int nq = threadIdx.x < ncell ? (n + 3) >> 2 : 0;
    int tot;
    const int off = warp_excl_scan(nq, &tot);
    if (threadIdx.x < ncell) {
      S.qoff[threadIdx.x] = off;
      S.n[threadIdx.x] = n;
    }
    if (threadIdx.x == 0) {
      S.qoff[ncell] = tot;
      S.count = 0;
    }
  }
  __syncthreads();
}

// Cell in CTA of flat quad g (g < qoff[ncell]).
__device__ __forceinline__ int dec_cell_of(const DecideSmem& S, int ncell, int g) {
  int lc = 0;
  while (lc + 1 < ncell && S.qoff[lc + 1] <= g) ++lc;
  return lc;
}

// Appends the flagged slots of this thread's quad (bits of nib; words w0/w1
// rotate with the slot) to the CTA list with one shared atomic per warp.
__device__ __forceinline__ void dec_append(DecideSmem& S, int lc, int slot0, uint32_t nib, uint4 w0, uint4 w1) {
  const int cnt = __popc(nib);
  int tot;
  const int off = warp_excl_scan(cnt, &tot);
  int base = 0;
  if (lane_id() == 0 && tot) base = atomicAdd(&S.count, tot);
  base = __shfl_sync(kFull, base, 0) + off;
#pragma unroll
  for (int j = 0; j < 4; ++j, rot(w0), rot(w1)) {
    if ((nib >> j) & 1u) {
      S.item[base] = ((uint32_t)lc << 16) | (uint32_t)(slot0 + j);
      S.u[base] = make_uint2(w0.x, w1.x);
      ++base;
    }
  }
}

// Runs f(item, words) for every listed slot: full batches of kDecThreads
// after each pass over the quads (drain == true), the rest at the end.
template <class F>
__device__ __forceinline__ void dec_drain(DecideSmem& S, bool final_pass, F f) {
  __syncthreads();
  int cnt = S.count;
  if (final_pass) {
    if ((int)threadIdx.x < cnt) f(S.item[threadIdx.x], S.u[threadIdx.x]);
    return;
  }
  while (cnt >= kDecThreads) {
    cnt -= kDecThreads;
    f(S.item[cnt + threadIdx.x], S.u[cnt + threadIdx.x]);
  }
  __syncthreads();
  if (threadIdx.x == 0) S.count = cnt;
  __syncthreads();
}

// Axions present at the start of the step: a->gamma and absorption.
__global__ void __launch_bounds__(kDecThreads) axion_decide_kernel(StepArgs A) {
  __shared__ DecideSmem S;
  const int cfirst = blockIdx.x * A.dec_cells;
  const int ncell = min(A.dec_cells, A.ncells - cfirst);
  const int mask = A.mask;
  const bool prim = mask & AXPIC_CH_PRIMAKOFF;
  const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const bool all = A.absorb_mode == 1 && bath;  // weight reduction changes every axion
  if (threadIdx.x < ncell) {
    const int c = cfirst + threadIdx.x;
    const float* rec = A.rec + (size_t)c * kRecLen;
    S.c0[threadIdx.x] = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    S.c1[threadIdx.x] = __ldg(rec + R_APINV);
    S.c2[threadIdx.x] = __ldg(rec + R_INVT);
  }
  dec_prefix(S, ncell, threadIdx.x < ncell ? min(max(A.a.count[cfirst + threadIdx.x], 0), A.a.cap) : 0);
  const int nq = S.qoff[ncell];
  auto full = [&](uint32_t it, uint2 uu) {
    const int cell = cfirst + (int)(it >> 16);
    const long idx = (long)cell * A.a.cap + (it & 0xFFFFu);
    const AxionDecision d =
        axion_decide_slow(A, cell, mask, A.a.w[idx], A.a.px[idx], A.a.py[idx], A.a.pz[idx], uu.x, uu.y);
    uint32_t f = (uint32_t)d.K;
    if (d.keep) f |= DF_KEEP;
    if (d.absorbed) f |= DF_ABSORBED;
    if (d.abs_c) f |= DF_ABS_C;
    if (d.capped) f |= DF_CAPPED;
    if (d.over) f |= DF_OVER;
    A.recA[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wnew), 0u);
  };
  for (int g0 = 0; g0 < nq; g0 += kDecThreads) {
    const int g = g0 + threadIdx.x;
    uint32_t nib = 0;
    int lc = 0, q = 0;
    uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
    if (g < nq) {
      lc = dec_cell_of(S, ncell, g);
      q = g - S.qoff[lc];
      const int cell = cfirst + lc;
      const int nj = min(4, S.n[lc] - 4 * q);
      const float* rec = A.rec + (size_t)cell * kRecLen;
      const float c_s = S.c0[lc], apinv = S.c1[lc], invT = S.c2[lc];
      const uint32_t gcell = A.cell_base + (uint32_t)cell;
      const long b = (long)cell * A.a.cap + 4 * q;
      float4 w4 = ld4(A.a.w + b), x4 = ld4(A.a.px + b), y4 = ld4(A.a.py + b), z4 = ld4(A.a.pz + b);
      if (prim) rP = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_PRIM_INV << 24), A.key0, A.key1);
      if (bath) rA = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_ABSORB << 24), A.key0, A.key1);
      uint4 tP = rP, tA = rA;
#pragma unroll
      for (int j = 0; j < 4; ++j, rot(w4), rot(x4), rot(y4), rot(z4), rot(tP), rot(tA)) {
        if (j >= nj) break;
        const float p2 = x4.x * x4.x + y4.x * y4.x + z4.x * z4.x;
        bool fast = !all;
        if (fast && prim) fast = no_conversion(w4.x, p2, c_s, apinv, A.inv_w_gref, u23(tP.x), A.lam_cap);
        if (fast && bath) fast = no_absorption(rec, A, mask, sqrtf(p2) * kMeC2f * invT, u23(tA.x));
        if (!fast) nib |= 1u << j;
      }
      flag_quad(A.bitsA, A.Wa, cell, q, nib);
    }
    dec_append(S, lc, 4 * q, nib, rP, rA);
    dec_drain(S, false, full);
  }
  dec_drain(S, true, full);
}

// Photons present at the start of the step (gamma->a): y == 0 of the grid.
__device__ __forceinline__ void photon_decide_cta(const StepArgs& A, DecideSmem& S, int cfirst, int ncell) {
  if (threadIdx.x < ncell) {
    const int c = cfirst + threadIdx.x;
    const float* rec = A.rec + (size_t)c * kRecLen;
    S.c0[threadIdx.x] = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    S.c1[threadIdx.x] = __ldg(rec + R_AP);
  }
  int n = 0;
  if (threadIdx.x < ncell) {
    const int c = cfirst + threadIdx.x;
    const int cnt = min(max(A.g.count[c], 0), A.g.cap);
    n = A.use_snapshot ? min(A.photon_start[c], cnt) : cnt;
  }
  dec_prefix(S, ncell, n);
  const int nq = S.qoff[ncell];
  auto full = [&](uint32_t it, uint2 uu) {
    const int cell = cfirst + (int)(it >> 16);
    const long idx = (long)cell * A.g.cap + (it & 0xFFFFu);
    const PhotonDecision d = photon_decide_slow(A, cell, A.g.w[idx], A.g.px[idx], A.g.py[idx], A.g.pz[idx], uu.x);
    uint32_t f = (uint32_t)d.K;
    if (d.wrem > 0.f) f |= DF_KEEP;
    if (d.capped) f |= DF_CAPPED;
    if (d.over) f |= DF_OVER;
    A.recG[idx] = make_uint4(f, __float_as_uint(d.wprod), __float_as_uint(d.wrem), 0u);
  };
  for (int g0 = 0; g0 < nq; g0 += kDecThreads) {
    const int g = g0 + threadIdx.x;
    uint32_t nib = 0;
    int lc = 0, q = 0;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (g < nq) {
      lc = dec_cell_of(S, ncell, g);
      q = g - S.qoff[lc];
      const int cell = cfirst + lc;
      const int nj = min(4, S.n[lc] - 4 * q);
      const float c_s = S.c0[lc], ap = S.c1[lc];
      const long b = (long)cell * A.g.cap + 4 * q;
      float4 w4 = ld4(A.g.w + b), x4 = ld4(A.g.px + b), y4 = ld4(A.g.py + b), z4 = ld4(A.g.pz + b);
      r = philox4x32_10(make_uint4(A.step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_PRIM_FWD << 24), A.key0,
                        A.key1);
      uint4 t = r;
#pragma unroll
      for (int j = 0; j < 4; ++j, rot(w4), rot(x4), rot(y4), rot(z4), rot(t)) {
        if (j >= nj) break;
        const float p2 = x4.x * x4.x + y4.x * y4.x + z4.x * z4.x;
        if (!no_conversion(w4.x, p2, c_s, ap, A.inv_w_a, u23(t.x), A.lam_cap)) nib |= 1u << j;
      }
      flag_quad(A.bitsG, A.Wg, cell, q, nib);
    }
    dec_append(S, lc, 4 * q, nib, r, r);
    dec_drain(S, false, full);
  }
  dec_drain(S, true, full);
}

// Electrons (thermal-bath emission): y == 1 of the grid. Their full
// decision is a short Poisson inversion, taken in place.
__device__ __forceinline__ void electron_decide_cta(const StepArgs& A, DecideSmem& S, int cfirst, int ncell) {
  const int mask = A.mask;
  const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
  if (threadIdx.x < ncell) {
    const int c = cfirst + threadIdx.x;
    const float* rec = A.rec + (size_t)c * kRecLen;
    const float rcc = __ldg(rec + R_CC), rcb = __ldg(rec + R_CB);
    const float wu = __ldg(A.mom + (size_t)c * kMomLen + M_WU);
    S.c0[threadIdx.x] = rcc;
    S.c1[threadIdx.x] = rcb;
    S.c2[threadIdx.x] = wu;
    float lsum = 0.f, F0 = 0.f;
    if (wu > 0.f) {
      // common weight: K > 0 exactly when u > exp(-lambda), lambda shared
      float fac;
      bool cc = false, cb = false;
      const float lc = eC ? cap_lambda(wu * rcc, A.lam_cap, &fac, &cc) : 0.f;
      const float lb = eB ? cap_lambda(wu * rcb, A.lam_cap, &fac, &cb) : 0.f;
      lsum = lc + lb;
      F0 = expf(-lsum);
    }
    S.c3[threadIdx.x] = F0;
    S.c4[threadIdx.x] = lsum;
  }
  dec_prefix(S, ncell, threadIdx.x < ncell ? min(max(A.e.count[cfirst + threadIdx.x], 0), A.e.cap) : 0);
  const int nq = S.qoff[ncell];
  for (int g = threadIdx.x; g < nq; g += kDecThreads) {
    const int lc = dec_cell_of(S, ncell, g);
    const int q = g - S.qoff[lc];
    const int cell = cfirst + lc;
    const int nj = min(4, S.n[lc] - 4 * q);
    uint4 r = philox4x32_10(make_uint4(A.step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_EMIT_E << 24), A.key0,
                            A.key1);
    const long b = (long)cell * A.e.cap + 4 * q;
    uint32_t nib = 0;
    if (S.c2[lc] > 0.f) {
      const float F0 = S.c3[lc], lsum = S.c4[lc];
#pragma unroll
      for (int j = 0; j < 4; ++j, rot(r)) {
        if (j >= nj) break;
        const float u = u23(r.x);
        if (u > F0) {
          A.recE[b + j] = (uint32_t)poisson_inv(u, lsum);
          nib |= 1u << j;
        }
      }
    } else {
      const float rcc = S.c0[lc], rcb = S.c1[lc];
      float4 w4 = ld4(A.e.w + b);
      const float rsum = ((eC ? rcc : 0.f) + (eB ? rcb : 0.f)) * 1.0001f;
#pragma unroll
      for (int j = 0; j < 4; ++j, rot(w4), rot(r)) {
        if (j >= nj) break;
        const float lbnd = w4.x * rsum;
        if (!(lbnd < A.lam_cap && u23(r.x) <= 1.0f - lbnd - 1e-6f)) {
          float fac;
          bool cc = false, cb = false;
          const float lc2 = eC ? cap_lambda(w4.x * rcc, A.lam_cap, &fac, &cc) : 0.f;
          const float lb2 = eB ? cap_lambda(w4.x * rcb, A.lam_cap, &fac, &cb) : 0.f;
          uint32_t f = (uint32_t)poisson_inv(u23(r.x), lc2 + lb2);
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

__global__ void __launch_bounds__(kDecThreads) emit_decide_kernel(StepArgs A) {
  __shared__ DecideSmem S;
  const int cfirst = blockIdx.x * A.dec_cells;
  const int ncell = min(A.dec_cells, A.ncells - cfirst);
  if (blockIdx.y == 0) {
    if (A.mask & AXPIC_CH_PRIMAKOFF) photon_decide_cta(A, S, cfirst, ncell);
  } else if (A.mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS)) {
    electron_decide_cta(A, S, cfirst, ncell);
  }
}

// ---------------------------------------------------------------- event kernel
// Per-warp shared scratch: ascending lists of flagged slots and of removed
// slots (u16), and removed-slot bit masks.
struct EvScratch {
  uint16_t *flA, *flG, *flE, *rmA, *rmG;
  uint32_t *rbA, *rbG;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t ev_scratch_bytes(int acap, int gcap, int ecap) {
  size_t b = 2 * (2 * (size_t)acap + 2 * (size_t)gcap + (size_t)ecap);
  b = align16(b) + 4 * (size_t)((acap + 31) / 32 + (gcap + 31) / 32);
  return align16(b);
}

__device__ inline EvScratch ev_carve(unsigned char* base, int acap, int gcap, int ecap) {
  EvScratch s;
  uint16_t* h = reinterpret_cast<uint16_t*>(base);
  s.flA = h; h += acap;
  s.flG = h; h += gcap;
  s.flE = h; h += ecap;
  s.rmA = h; h += acap;
  s.rmG = h; h += gcap;
  uint32_t* u = reinterpret_cast<uint32_t*>(align16(reinterpret_cast<size_t>(h)));
  s.rbA = u; u += (acap + 31) / 32;
  s.rbG = u;
  return s;
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
// below n_surv, movers the kept slots at or beyond it, matched in order.
__device__ __noinline__ void compact_removed(const SpeciesPtrs& s, long base, const uint16_t* rm, int nrm,
                                             const uint32_t* rb, int n) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const int n_surv = n - nrm;
  int run = 0;
  for (int b0 = n_surv; b0 < n; b0 += 32) {
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

template <int PH>
__device__ __forceinline__ void event_cell(const StepArgs& A, int cell, EvScratch& S, const Cnt& cnt) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t gcell = A.cell_base + (uint32_t)cell;
  const int mask = A.mask;
  const int ne = min(max(A.e.count[cell], 0), A.e.cap);
  const int ng_start = min(max(A.g.count[cell], 0), A.g.cap);
  const int na_start = min(max(A.a.count[cell], 0), A.a.cap);
  int ng = ng_start;
  int na = na_start;
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  const bool prim = mask & AXPIC_CH_PRIMAKOFF;
  const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
  const int ng0 = (PH & PH_ABSORB) ? ng_start : (A.use_snapshot ? min(A.photon_start[cell], ng) : ng);
  // particles present at the start of the step: counted by the absorb phase,
  // or by the emit phase when no absorb ran this step
  if (lane == 0 && ((PH & PH_ABSORB) || ((PH & PH_EMIT) && !A.use_snapshot))) {
    cnt.add(C_NE, ne);
    cnt.add(C_NG, ng_start);
    cnt.add(C_NA, na);
    cnt.add(C_CELLS, 1);
  }
  // all decision masks of this call are read (and cleared) up front
  int nflA = 0, nflG = 0, nflE = 0;
  {
    const int nwA = (PH & PH_ABSORB) ? (na_start + 31) >> 5 : 0;
    const int nwG = ((PH & PH_EMIT) && prim) ? (ng0 + 31) >> 5 : 0;
    const int nwE = ((PH & PH_EMIT) && (eC || eB)) ? (ne + 31) >> 5 : 0;
    if (nwA <= 32 && nwG <= 32 && nwE <= 32) {
      uint32_t* rA = A.bitsA + (size_t)cell * A.Wa;
      uint32_t* rG = A.bitsG + (size_t)cell * A.Wg;
      uint32_t* rE = A.bitsE + (size_t)cell * A.We;
      const uint32_t vA = lane < nwA ? rA[lane] : 0u;
      const uint32_t vG = lane < nwG ? rG[lane] : 0u;
      const uint32_t vE = lane < nwE ? rE[lane] : 0u;
      if (vA) rA[lane] = 0u;
      if (vG) rG[lane] = 0u;
      if (vE) rE[lane] = 0u;
      if (__any_sync(kFull, vA != 0)) nflA = list_flags(vA, lane, nwA, na_start, S.flA, 0);
      if (__any_sync(kFull, vG != 0)) nflG = list_flags(vG, lane, nwG, ng0, S.flG, 0);
      if (__any_sync(kFull, vE != 0)) nflE = list_flags(vE, lane, nwE, ne, S.flE, 0);
    } else {
      if (nwA) nflA = gather_flags(A.bitsA, A.Wa, cell, na_start, S.flA);
      if (nwG) nflG = gather_flags(A.bitsG, A.Wg, cell, ng0, S.flG);
      if (nwE) nflE = gather_flags(A.bitsE, A.We, cell, ne, S.flE);
    }
    __syncwarp();
  }
  Lane64 x64;
  double xa[4] = {0.0, 0.0, 0.0, 0.0};
  bool xa_any = false;

  // ------------------------------------------------------------ absorb
  if (PH & PH_ABSORB) {
    if (lane == 0) A.photon_start[cell] = ng;
    if (nflA > 0) {
      for (int i = lane; i < (na_start + 31) / 32; i += 32) S.rbA[i] = 0u;
      __syncwarp();
      int run = 0, nrm = 0, NPg = 0;
      for (int i0 = 0; i0 < nflA; i0 += 32) {
        const int i = i0 + lane;
        int K = 0, slot = 0;
        bool removed = false;
        float wprod = 0.f, px = 0.f, py = 0.f, pz = 0.f, xx = 0.f, yy = 0.f, zz = 0.f;
        if (i < nflA) {
          slot = S.flA[i];
          const long src = abase + slot;
          const uint4 r = A.recA[src];
          const float w = A.a.w[src];
          px = A.a.px[src];
          py = A.a.py[src];
          pz = A.a.pz[src];
          K = r.x & 0xFF;
          wprod = __uint_as_float(r.y);
          const float wnew = __uint_as_float(r.z);
          const float om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
          cnt.add(C_CAP, (r.x & DF_CAPPED) ? 1u : 0u);
          cnt.add(C_CLAMP, (r.x & DF_OVER) ? 1u : 0u);
          cnt.add(C_EV_PINV, (unsigned)K);
          if (r.x & DF_ABSORBED) {
            x64.add((double)wnew, om, px, py, pz);
            cnt.add((r.x & DF_ABS_C) ? C_ABS_C : C_ABS_B, 1);
          } else if (A.absorb_mode == 1 && bath) {
            // weight reduction: the lost weight's energy goes to the plasma
            float wrem = w;
            if (K > 0) wrem = (r.x & DF_OVER) ? 0.f : __fsub_rn(w, __fmul_rn((float)K, wprod));
            x64.add((double)wrem - (double)wnew, om, px, py, pz);
          }
          removed = !(r.x & DF_KEEP);
          if (K) {
            xx = A.a.x[src];
            yy = A.a.y[src];
            zz = A.a.z[src];
          }
          if (!removed && wnew != w) A.a.w[src] = wnew;
        }
        // photon products of a->gamma after the photons present
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        for (int k = 0; k < K; ++k, ++off) {
          const int dst = ng + off;
          if (dst < A.g.cap) write_particle(A.g, gbase + dst, wprod, px, py, pz, xx, yy, zz);
          else cnt.add(C_DROP, 1);
        }
        run += tot;
        NPg += K;
        const unsigned m = __ballot_sync(kFull, removed);
        if (removed) {
          S.rmA[nrm + __popc(m & lt)] = (uint16_t)slot;
          atomicOr(&S.rbA[slot >> 5], 1u << (slot & 31));
        }
        nrm += __popc(m);
      }
      NPg = warp_sum_i(NPg);
      ng = min(ng + NPg, A.g.cap);
      __syncwarp();
      if (nrm > 0) compact_removed(A.a, abase, S.rmA, nrm, S.rbA, na_start);
      __syncwarp();
      na = na_start - nrm;
    }
    if (__any_sync(kFull, x64.any)) {
      xa[0] = warp_sum_d(x64.dE);
      xa[1] = warp_sum_d(x64.dPx);
      xa[2] = warp_sum_d(x64.dPy);
      xa[3] = warp_sum_d(x64.dPz);
      xa_any = true;
    }
    x64 = Lane64();
  }

  // ------------------------------------------------------------ emit
  if (PH & PH_EMIT) {
    const int ng_tot = ng;
    const int abase_new = na;
    int NPa = 0, nrm = 0;
    // (c) flagged photons; axion products after the surviving axions
    if (nflG > 0) {
      for (int i = lane; i < (ng_tot + 31) / 32; i += 32) S.rbG[i] = 0u;
      __syncwarp();
      int run = 0;
      for (int i0 = 0; i0 < nflG; i0 += 32) {
        const int i = i0 + lane;
        int K = 0, slot = 0;
        bool removed = false;
        float wprod = 0.f, om = 0.f, px = 0.f, py = 0.f, pz = 0.f, xx = 0.f, yy = 0.f, zz = 0.f;
        if (i < nflG) {
          slot = S.flG[i];
          const long src = gbase + slot;
          const uint4 r = A.recG[src];
          K = r.x & 0xFF;
          wprod = __uint_as_float(r.y);
          const float wrem = __uint_as_float(r.z);
          cnt.add(C_CAP, (r.x & DF_CAPPED) ? 1u : 0u);
          cnt.add(C_CLAMP, (r.x & DF_OVER) ? 1u : 0u);
          cnt.add(C_EV_P, (unsigned)K);
          removed = !(r.x & DF_KEEP);
          if (K) {
            px = A.g.px[src];
            py = A.g.py[src];
            pz = A.g.pz[src];
            xx = A.g.x[src];
            yy = A.g.y[src];
            zz = A.g.z[src];
            om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
            if (!removed) A.g.w[src] = wrem;
          }
        }
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        for (int k = 0; k < K; ++k, ++off) {
          const int dst = abase_new + off;
          if (dst < A.a.cap) {
            write_particle(A.a, abase + dst, wprod, px, py, pz, xx, yy, zz);
            if (A.tally_enable) tally_add(A, 0, wprod, om);
          } else {
            cnt.add(C_DROP, 1);
          }
        }
        run += tot;
        NPa += K;
        const unsigned m = __ballot_sync(kFull, removed);
        if (removed) {
          S.rmG[nrm + __popc(m & lt)] = (uint16_t)slot;
          atomicOr(&S.rbG[slot >> 5], 1u << (slot & 31));
        }
        nrm += __popc(m);
      }
      NPa = warp_sum_i(NPa);
    }
    // (d) electron events, in electron then event order; event k of
    // electron i: cos theta, phi, energy and channel from one Philox block
    int NE = 0;
    if (eC || eB) {
      const float* rec = A.rec + (size_t)cell * kRecLen;
      const float wu = A.mom[(size_t)cell * kMomLen + M_WU];
      if (wu > 0.f && lane == 0) {
        float fac;
        bool cc = false, cb = false;
        if (eC) cap_lambda(wu * rec[R_CC], A.lam_cap, &fac, &cc);
        if (eB) cap_lambda(wu * rec[R_CB], A.lam_cap, &fac, &cb);
        cnt.add(C_CAP, (unsigned)ne * ((unsigned)cc + (unsigned)cb));
      }
      if (nflE > 0) {
        const float* tabC = A.tables + TAB_COMPTON * kTableN;
        const float* tabB = A.tables + TAB_BREMS * kTableN;
        int run = 0;
        for (int i0 = 0; i0 < nflE; i0 += 32) {
          const int i = i0 + lane;
          int K = 0, slot = 0;
          if (i < nflE) {
            slot = S.flE[i];
            const uint32_t f = A.recE[ebase + slot];
            K = f & 0xFF;
            if (wu <= 0.f) cnt.add(C_CAP, ((f & DF_CAPPED) ? 1u : 0u) + ((f & DF_CAPPED_B) ? 1u : 0u));
          }
          int tot;
          int off = run + warp_excl_scan(K, &tot);
          if (K) {
            const long src = ebase + slot;
            const float w = wu > 0.f ? wu : A.e.w[src];
            const float xx = A.e.x[src], yy = A.e.y[src], zz = A.e.z[src];
            float facC = 1.f, facB = 1.f;
            bool cc = false, cb = false;
            const float lc = eC ? cap_lambda(w * rec[R_CC], A.lam_cap, &facC, &cc) : 0.f;
            const float lb = eB ? cap_lambda(w * rec[R_CB], A.lam_cap, &facB, &cb) : 0.f;
            const float fracC = lc / (lc + lb);
            const float wvC = cc ? A.w_a * facC : A.w_a;
            const float wvB = cb ? A.w_a * facB : A.w_a;
            for (int k = 0; k < K; ++k, ++off) {
              const uint4 r = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)slot, (S_EV_E << 24) | (uint32_t)k),
                                            A.key0, A.key1);
              const bool isC = u23(r.w) < fracC;
              const float3 dv = iso_dir(u23(r.x), u23(r.y));
              const float E = icdf_lookup(isC ? tabC : tabB, u23(r.z)) * rec[R_T];
              const float wv = isC ? wvC : wvB;
              const float pm = E * kInvMeC2f;
              const float px = pm * dv.x, py = pm * dv.y, pz = pm * dv.z;
              const int dst = abase_new + NPa + off;
              if (dst < A.a.cap) {
                write_particle(A.a, abase + dst, wv, px, py, pz, xx, yy, zz);
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
    // (e) tail-fill compaction of the photons (a->gamma products included)
    if (nrm > 0) compact_removed(A.g, gbase, S.rmG, nrm, S.rbG, ng_tot);
    ng = ng_tot - nrm;
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
  if (lane == 0 && (xa_any || xe_any)) {
    double* xb = A.xbuf + (size_t)cell * 4;
    if (xa_any) {
      xb[0] += xa[0];
      xb[1] += xa[1];
      xb[2] += xa[2];
      xb[3] += xa[3];
    }
    if (xe_any) {
      xb[0] += xe[0];
      xb[1] += xe[1];
      xb[2] += xe[2];
      xb[3] += xe[3];
    }
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
    event_cell<PH>(A, cell, S, cnt);
  }
  __syncwarp();
  if (lane < kNumCounters) {
    const unsigned long long v = warp_cnt[wid][lane];
    if (v) atomicAdd(A.counters + (size_t)blockIdx.x * kNumCounters + lane, v);
    if (lane == C_DROP && v) atomicOr(A.err, ERR_CAPACITY);
  }
}

// ---------------------------------------------------------------- feedback kernel
// One lane per cell: the exchange of this step plus the carried part; when it
// is representable in binary32 momenta the whole warp remaps that cell's
// electrons (Eqs. delta_def to b_def, affine_map), measuring what was applied;
// then the temperature update (Eqs. Te_est, Te_relax) and the record's
// temperature half.
__global__ void __launch_bounds__(128) feedback_kernel(StepArgs A) {
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < A.ncells;
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0, rE = 0.0, rPx = 0.0, rPy = 0.0, rPz = 0.0;
  float W = 0.f, Px = 0.f, Py = 0.f, Pz = 0.f, U2 = 0.f, var = 0.f;
  bool has_x = false, has_res = false, need = false;
  int ne = 0;
  double qE = 0.0, qPx = 0.0, qPy = 0.0, qPz = 0.0, s1d = 0.0, bx = 0.0, by = 0.0, bz = 0.0, vnd = 0.0;
  if (valid) {
    double* xb = A.xbuf + (size_t)cell * 4;
    dE = xb[0];
    dPx = xb[1];
    dPy = xb[2];
    dPz = xb[3];
    has_x = nz64(dE) || nz64(dPx) || nz64(dPy) || nz64(dPz);
    if (has_x) {
      xb[0] = 0.0;
      xb[1] = 0.0;
      xb[2] = 0.0;
      xb[3] = 0.0;
    }
    const double* rs = A.res + (size_t)cell * 4;
    rE = rs[0];
    rPx = rs[1];
    rPy = rs[2];
    rPz = rs[3];
    has_res = nz64(rE) || nz64(rPx) || nz64(rPy) || nz64(rPz);
    const float* mom = A.mom + (size_t)cell * kMomLen;
    W = mom[M_W];
    Px = mom[M_PX];
    Py = mom[M_PY];
    Pz = mom[M_PZ];
    U2 = mom[M_U2];
    var = mom[M_VAR];
    ne = min(max(A.e.count[cell], 0), A.e.cap);
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
  // the warp remaps each cell that needs it, one after the other
  double nrE = qE, nrPx = qPx, nrPy = qPy, nrPz = qPz, applied_E = 0.0;
  float var_new = var;
  unsigned m = __ballot_sync(kFull, need);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1u;
    const int c_src = __shfl_sync(kFull, cell, src);
    const int ne_src = __shfl_sync(kFull, ne, src);
    const float s1 = __shfl_sync(kFull, (float)s1d, src);
    const float fbx = __shfl_sync(kFull, (float)bx, src);
    const float fby = __shfl_sync(kFull, (float)by, src);
    const float fbz = __shfl_sync(kFull, (float)bz, src);
    const RemapOut r = remap_electrons(A, (long)c_src * A.e.cap, ne_src, s1, fbx, fby, fbz);
    if (lane == src) {
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
  }
  if (!valid) return;
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
    const double T = A.T[cell];
    const float Tf = (float)T;
    const float Test = (kMeC2f / 3.0f) * var_new / W;
    const float dT = A.relax_r * (Test - Tf);
    double Tn = T + (double)dT;
    const float Tnf = Tf + dT;
    if (Tnf <= A.T_floor_f || Tnf >= A.T_ceil_f) Tn = fmin(fmax(Tn, A.T_floor), A.T_ceil);
    float rec[kRecLen];
    load_rec(A, cell, rec);
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

static int dec_blocks(const StepArgs& A) { return (A.ncells + A.dec_cells - 1) / A.dec_cells; }

static cudaError_t launch_axion_decide(const StepArgs& A, cudaStream_t st) {
  if (A.a.cap == 0 || A.ncells == 0) return cudaSuccess;
  axion_decide_kernel<<<dec_blocks(A), kDecThreads, 0, st>>>(A);
  return cudaGetLastError();
}

static cudaError_t launch_emit_decide(const StepArgs& A, cudaStream_t st) {
  if ((A.g.cap == 0 && A.e.cap == 0) || A.ncells == 0) return cudaSuccess;
  emit_decide_kernel<<<dim3(dec_blocks(A), 2), kDecThreads, 0, st>>>(A);
  return cudaGetLastError();
}

static cudaError_t launch_feedback(const StepArgs& A, cudaStream_t st) {
  feedback_kernel<<<(A.ncells + 127) / 128, 128, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st, cudaEvent_t* ev) {
  if (A.ncells == 0) return cudaSuccess;
  cudaError_t e;
  // optional measurement: events between the kernels of a full step
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], st) : cudaSuccess; };
  switch (phases) {
    case PH_ABSORB:
      if ((e = launch_axion_decide(A, st))) return e;
      return launch_events<PH_ABSORB>(A, warps, st);
    case PH_EMIT:
      if ((e = launch_emit_decide(A, st))) return e;
      return launch_events<PH_EMIT>(A, warps, st);
    case PH_FEEDBACK:
      return launch_feedback(A, st);
    case PH_ALL: {
      // the photon decisions of the emit phase read the photons present at
      // the start of the step, before the absorb phase appends a->gamma
      // products, so both decision kernels run first
      if ((e = mark(0)) || (e = launch_axion_decide(A, st)) || (e = mark(1))) return e;
      if ((e = launch_emit_decide(A, st)) || (e = mark(2))) return e;
      if ((e = launch_events<PH_ABSORB | PH_EMIT>(A, warps, st)) || (e = mark(3))) return e;
      if ((e = launch_feedback(A, st)) || (e = mark(4))) return e;
      return cudaSuccess;
    }
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t set_step_smem_limits(size_t bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(event_kernel<PH_ABSORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)))
    return e;
  if ((e = cudaFuncSetAttribute(event_kernel<PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)))
    return e;
  return cudaFuncSetAttribute(event_kernel<PH_ABSORB | PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

}  // namespace axpic
