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

// ---------------------------------------------------------------- decision kernels
// Bit masks: word (cell * W + s / 32), bit s % 32 flags slot s. Words are
// set by atomicOr (rare) and cleared by the event kernel after reading.

__device__ __forceinline__ void flag_quad(uint32_t* bits, int W, int cell, int q, uint32_t nib) {
  if (nib) atomicOr(bits + (size_t)cell * W + ((4 * q) >> 5), nib << ((4 * q) & 31));
}

// Axions present at the start of the step: a->gamma and absorption.
__global__ void __launch_bounds__(256) axion_decide_kernel(StepArgs A) {
  const int Q = A.a.cap >> 2;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cell = (int)(t / Q);
  const int q = (int)(t - (long)cell * Q);
  if (cell >= A.ncells) return;
  const int n = min(max(A.a.count[cell], 0), A.a.cap);
  if (4 * q >= n) return;
  const int nj = min(4, n - 4 * q);
  const int mask = A.mask;
  const bool prim = mask & AXPIC_CH_PRIMAKOFF;
  const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
  uint32_t nib;
  if (A.absorb_mode == 1 && bath) {
    nib = (1u << nj) - 1u;  // weight reduction changes every axion
  } else {
    const float* rec = A.rec + (size_t)cell * kRecLen;
    const float c_s = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    const float apinv = __ldg(rec + R_APINV);
    const float invT = __ldg(rec + R_INVT);
    const uint32_t gcell = A.cell_base + (uint32_t)cell;
    const long b = (long)cell * A.a.cap + 4 * q;
    float4 w4 = ld4(A.a.w + b), x4 = ld4(A.a.px + b), y4 = ld4(A.a.py + b), z4 = ld4(A.a.pz + b);
    uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
    if (prim) rP = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_PRIM_INV << 24), A.key0, A.key1);
    if (bath) rA = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_ABSORB << 24), A.key0, A.key1);
    nib = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j, rot(w4), rot(x4), rot(y4), rot(z4), rot(rP), rot(rA)) {
      if (j >= nj) break;
      const float p2 = x4.x * x4.x + y4.x * y4.x + z4.x * z4.x;
      bool fast = true;
      if (prim) fast = no_conversion(w4.x, p2, c_s, apinv, A.inv_w_gref, u23(rP.x), A.lam_cap);
      if (fast && bath) fast = no_absorption(rec, A, mask, sqrtf(p2) * kMeC2f * invT, u23(rA.x));
      if (!fast) nib |= 1u << j;
    }
  }
  flag_quad(A.bitsA, A.Wa, cell, q, nib);
}

// Photons present at the start of the step (gamma->a) and electrons
// (thermal-bath emission): photon quads first, then electron quads.
__global__ void __launch_bounds__(256) emit_decide_kernel(StepArgs A) {
  const int Qg = A.g.cap >> 2, Qe = A.e.cap >> 2;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long ng_quads = (long)A.ncells * Qg;
  const int mask = A.mask;
  if (t < ng_quads) {
    if (!(mask & AXPIC_CH_PRIMAKOFF)) return;
    const int cell = (int)(t / Qg);
    const int q = (int)(t - (long)cell * Qg);
    const int cnt = min(max(A.g.count[cell], 0), A.g.cap);
    const int n = A.use_snapshot ? min(A.photon_start[cell], cnt) : cnt;
    if (4 * q >= n) return;
    const int nj = min(4, n - 4 * q);
    const float* rec = A.rec + (size_t)cell * kRecLen;
    const float c_s = kMeC2f * kMeC2f * __ldg(rec + R_FOURK2);
    const float ap = __ldg(rec + R_AP);
    const long b = (long)cell * A.g.cap + 4 * q;
    float4 w4 = ld4(A.g.w + b), x4 = ld4(A.g.px + b), y4 = ld4(A.g.py + b), z4 = ld4(A.g.pz + b);
    uint4 r = philox4x32_10(make_uint4(A.step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_PRIM_FWD << 24), A.key0,
                            A.key1);
    uint32_t nib = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j, rot(w4), rot(x4), rot(y4), rot(z4), rot(r)) {
      if (j >= nj) break;
      const float p2 = x4.x * x4.x + y4.x * y4.x + z4.x * z4.x;
      if (!no_conversion(w4.x, p2, c_s, ap, A.inv_w_a, u23(r.x), A.lam_cap)) nib |= 1u << j;
    }
    flag_quad(A.bitsG, A.Wg, cell, q, nib);
    return;
  }
  const long te = t - ng_quads;
  const int cell = (int)(te / Qe);
  const int q = (int)(te - (long)cell * Qe);
  if (cell >= A.ncells) return;
  const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
  if (!(eC || eB)) return;
  const int n = min(max(A.e.count[cell], 0), A.e.cap);
  if (4 * q >= n) return;
  const int nj = min(4, n - 4 * q);
  const float* rec = A.rec + (size_t)cell * kRecLen;
  const float rcc = __ldg(rec + R_CC), rcb = __ldg(rec + R_CB);
  uint4 r = philox4x32_10(make_uint4(A.step, A.cell_base + (uint32_t)cell, (uint32_t)q, S_EMIT_E << 24), A.key0,
                          A.key1);
  const float wu = __ldg(A.mom + (size_t)cell * kMomLen + M_WU);
  uint32_t nib = 0;
  if (wu > 0.f) {
    // common weight: K > 0 exactly when u > exp(-lambda), lambda shared
    float fac;
    bool cc = false, cb = false;
    const float lc = eC ? cap_lambda(wu * rcc, A.lam_cap, &fac, &cc) : 0.f;
    const float lb = eB ? cap_lambda(wu * rcb, A.lam_cap, &fac, &cb) : 0.f;
    const float F0 = expf(-(lc + lb));
#pragma unroll
    for (int j = 0; j < 4; ++j, rot(r)) {
      if (j >= nj) break;
      if (u23(r.x) > F0) nib |= 1u << j;
    }
  } else {
    float4 w4 = ld4(A.e.w + (long)cell * A.e.cap + 4 * q);
    const float rsum = ((eC ? rcc : 0.f) + (eB ? rcb : 0.f)) * 1.0001f;
#pragma unroll
    for (int j = 0; j < 4; ++j, rot(w4), rot(r)) {
      if (j >= nj) break;
      const float lb = w4.x * rsum;
      if (!(lb < A.lam_cap && u23(r.x) <= 1.0f - lb - 1e-6f)) nib |= 1u << j;
    }
  }
  flag_quad(A.bitsE, A.We, cell, q, nib);
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

// Reads the cell's bit-mask words covering [0, n), clears them, and writes
// the flagged slots in ascending order to `list`. Returns their number.
__device__ __forceinline__ int gather_flags(uint32_t* bits, int W, int cell, int n, uint16_t* list) {
  const int lane = lane_id();
  const int nw = (n + 31) >> 5;
  uint32_t* row = bits + (size_t)cell * W;
  int total = 0;
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int wi = w0 + lane;
    uint32_t v = wi < nw ? row[wi] : 0u;
    if (v) row[wi] = 0u;
    if (wi == nw - 1 && (n & 31)) v &= (1u << (n & 31)) - 1u;  // bits beyond n never count
    int tot;
    int at = total + warp_excl_scan(__popc(v), &tot);
    while (v) {
      const int bpos = __ffs(v) - 1;
      v &= v - 1u;
      list[at++] = (uint16_t)(32 * wi + bpos);
    }
    total += tot;
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
  int ng = ng_start;
  int na = min(max(A.a.count[cell], 0), A.a.cap);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  // particles present at the start of the step: counted by the absorb phase,
  // or by the emit phase when no absorb ran this step
  if (lane == 0 && ((PH & PH_ABSORB) || ((PH & PH_EMIT) && !A.use_snapshot))) {
    cnt.add(C_NE, ne);
    cnt.add(C_NG, ng_start);
    cnt.add(C_NA, na);
    cnt.add(C_CELLS, 1);
  }
  Lane64 x64;
  double xa[4] = {0.0, 0.0, 0.0, 0.0};
  bool xa_any = false;

  // ------------------------------------------------------------ absorb
  if (PH & PH_ABSORB) {
    if (lane == 0) A.photon_start[cell] = ng;
    const int na0 = na;
    const int nfl = gather_flags(A.bitsA, A.Wa, cell, na0, S.flA);
    if (nfl > 0) {
      const bool prim = mask & AXPIC_CH_PRIMAKOFF;
      const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
      for (int i = lane; i < (na0 + 31) / 32; i += 32) S.rbA[i] = 0u;
      __syncwarp();
      int run = 0, nrm = 0, NPg = 0;
      for (int i0 = 0; i0 < nfl; i0 += 32) {
        const int i = i0 + lane;
        int K = 0;
        bool removed = false;
        AxionDecision d;
        d.K = 0;
        d.keep = true;
        int slot = 0;
        float px = 0.f, py = 0.f, pz = 0.f, xx = 0.f, yy = 0.f, zz = 0.f;
        if (i < nfl) {
          slot = S.flA[i];
          const uint32_t q = slot >> 2;
          uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
          if (prim) rP = philox4x32_10(make_uint4(A.step, gcell, q, S_PRIM_INV << 24), A.key0, A.key1);
          if (bath) rA = philox4x32_10(make_uint4(A.step, gcell, q, S_ABSORB << 24), A.key0, A.key1);
          const long src = abase + slot;
          const float w = A.a.w[src];
          px = A.a.px[src];
          py = A.a.py[src];
          pz = A.a.pz[src];
          d = axion_decide_slow(A, cell, mask, w, px, py, pz, word(rP, slot & 3), word(rA, slot & 3));
          cnt.add(C_CAP, d.capped);
          cnt.add(C_CLAMP, d.over);
          cnt.add(C_EV_PINV, d.K);
          if (d.absorbed) {
            x64.add((double)d.wnew, d.om, px, py, pz);
            if (d.abs_c) cnt.add(C_ABS_C, 1);
            else cnt.add(C_ABS_B, 1);
          } else if (A.absorb_mode == 1 && bath) {
            // weight reduction: the lost weight's energy goes to the plasma
            float wrem = w;
            if (d.K > 0) wrem = d.over ? 0.f : __fsub_rn(w, __fmul_rn((float)d.K, d.wprod));
            x64.add((double)wrem - (double)d.wnew, d.om, px, py, pz);
          }
          K = d.K;
          removed = !d.keep;
          if (K) {
            xx = A.a.x[src];
            yy = A.a.y[src];
            zz = A.a.z[src];
          }
          if (d.keep && d.wnew != w) A.a.w[src] = d.wnew;
        }
        // photon products of a->gamma after the photons present
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        for (int k = 0; k < K; ++k, ++off) {
          const int dst = ng + off;
          if (dst < A.g.cap) write_particle(A.g, gbase + dst, d.wprod, px, py, pz, xx, yy, zz);
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
      if (nrm > 0) compact_removed(A.a, abase, S.rmA, nrm, S.rbA, na0);
      __syncwarp();
      na = na0 - nrm;
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
    const int ng0 = (PH & PH_ABSORB) ? ng_start : (A.use_snapshot ? min(A.photon_start[cell], ng) : ng);
    const int ng_tot = ng;
    const bool prim = mask & AXPIC_CH_PRIMAKOFF;
    const int abase_new = na;
    int NPa = 0, nrm = 0;
    // (c) photon decisions for the flagged photons; axion products after the
    // surviving axions
    if (prim) {
      const int nfl = gather_flags(A.bitsG, A.Wg, cell, ng0, S.flG);
      if (nfl > 0) {
        for (int i = lane; i < (ng_tot + 31) / 32; i += 32) S.rbG[i] = 0u;
        __syncwarp();
        int run = 0;
        for (int i0 = 0; i0 < nfl; i0 += 32) {
          const int i = i0 + lane;
          int K = 0;
          bool removed = false;
          int slot = 0;
          PhotonDecision d;
          d.K = 0;
          float px = 0.f, py = 0.f, pz = 0.f, xx = 0.f, yy = 0.f, zz = 0.f;
          if (i < nfl) {
            slot = S.flG[i];
            const uint4 r =
                philox4x32_10(make_uint4(A.step, gcell, (uint32_t)(slot >> 2), S_PRIM_FWD << 24), A.key0, A.key1);
            const long src = gbase + slot;
            const float w = A.g.w[src];
            px = A.g.px[src];
            py = A.g.py[src];
            pz = A.g.pz[src];
            d = photon_decide_slow(A, cell, w, px, py, pz, word(r, slot & 3));
            cnt.add(C_CAP, d.capped);
            cnt.add(C_CLAMP, d.over);
            cnt.add(C_EV_P, d.K);
            K = d.K;
            removed = !(d.wrem > 0.f);
            if (K) {
              xx = A.g.x[src];
              yy = A.g.y[src];
              zz = A.g.z[src];
              if (!removed) A.g.w[src] = d.wrem;
            }
          }
          int tot;
          int off = run + warp_excl_scan(K, &tot);
          for (int k = 0; k < K; ++k, ++off) {
            const int dst = abase_new + off;
            if (dst < A.a.cap) {
              write_particle(A.a, abase + dst, d.wprod, px, py, pz, xx, yy, zz);
              if (A.tally_enable) tally_add(A, 0, d.wprod, d.om);
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
    }
    // (d) electron events, in electron then event order; event k of
    // electron i: cos theta, phi, energy and channel from one Philox block
    const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
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
      const int nfl = gather_flags(A.bitsE, A.We, cell, ne, S.flE);
      if (nfl > 0) {
        const float* tabC = A.tables + TAB_COMPTON * kTableN;
        const float* tabB = A.tables + TAB_BREMS * kTableN;
        int run = 0;
        for (int i0 = 0; i0 < nfl; i0 += 32) {
          const int i = i0 + lane;
          int K = 0, slot = 0;
          float w = 0.f, lc = 0.f, lb = 0.f, facC = 1.f, facB = 1.f;
          bool cc = false, cb = false;
          if (i < nfl) {
            slot = S.flE[i];
            const uint4 r =
                philox4x32_10(make_uint4(A.step, gcell, (uint32_t)(slot >> 2), S_EMIT_E << 24), A.key0, A.key1);
            w = wu > 0.f ? wu : A.e.w[ebase + slot];
            lc = eC ? cap_lambda(w * rec[R_CC], A.lam_cap, &facC, &cc) : 0.f;
            lb = eB ? cap_lambda(w * rec[R_CB], A.lam_cap, &facB, &cb) : 0.f;
            if (wu <= 0.f) cnt.add(C_CAP, (unsigned)cc + (unsigned)cb);
            K = poisson_inv(u23(word(r, slot & 3)), lc + lb);
          }
          int tot;
          int off = run + warp_excl_scan(K, &tot);
          if (K) {
            const long src = ebase + slot;
            const float xx = A.e.x[src], yy = A.e.y[src], zz = A.e.z[src];
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
              if (isC) cnt.add(C_EV_C, 1);
              else cnt.add(C_EV_B, 1);
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

static cudaError_t launch_axion_decide(const StepArgs& A, cudaStream_t st) {
  const long threads = (long)A.ncells * (A.a.cap >> 2);
  if (threads == 0) return cudaSuccess;
  axion_decide_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A);
  return cudaGetLastError();
}

static cudaError_t launch_emit_decide(const StepArgs& A, cudaStream_t st) {
  const long threads = (long)A.ncells * ((A.g.cap >> 2) + (A.e.cap >> 2));
  if (threads == 0) return cudaSuccess;
  emit_decide_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A);
  return cudaGetLastError();
}

static cudaError_t launch_feedback(const StepArgs& A, cudaStream_t st) {
  feedback_kernel<<<(A.ncells + 127) / 128, 128, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st) {
  if (A.ncells == 0) return cudaSuccess;
  cudaError_t e;
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
      if ((e = launch_axion_decide(A, st))) return e;
      if ((e = launch_emit_decide(A, st))) return e;
      if ((e = launch_events<PH_ABSORB | PH_EMIT>(A, warps, st))) return e;
      return launch_feedback(A, st);
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
