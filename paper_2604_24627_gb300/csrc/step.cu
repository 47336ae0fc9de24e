// The per-cell step kernel: absorb -> emit -> feedback (Sec. II.D-II.J).
//
// One warp owns one cell. Particles are read as float4 quads of consecutive
// slots (coalesced 128-bit loads from the SoA slabs); one Philox4x32-10 block
// supplies the decision uniforms of a quad, word j for slot 4q+j. Decisions
// are made in a first pass that touches only (w, p) of photons and axions and
// w of electrons; products, compaction and the remap are a second pass whose
// addresses come from warp prefix sums, so the output order is the
// deterministic one of the method's definition (never atomic append order).
//
// Phases (template bit mask): ABSORB (inverse operators on the axions present
// at the start), EMIT (forward operators), FEEDBACK (affine remap and
// temperature update). The fused step uses all three and keeps the exchange
// (Delta E, Delta P) in registers; separate calls pass it through an FP64
// per-cell buffer.
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

// Per-warp shared scratch (dynamic shared memory): keep bit masks written by
// warp ballots, ascending lists of the slots that have events (slot | K << 16)
// and the hole list of the tail-fill compaction.
struct WarpScratch {
  uint32_t *kA, *kG;
  uint32_t *evA, *evG, *evE;
  uint16_t* holes;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t warp_scratch_bytes(int acap, int gcap, int ecap) {
  const size_t wa = (acap + 31) / 32, wg = (gcap + 31) / 32;
  size_t b = 4 * (wa + wg) + 4 * ((size_t)acap + gcap + ecap);
  b = align16(b) + align16(2 * (size_t)(acap > gcap ? acap : gcap));
  return align16(b);
}

__device__ inline WarpScratch carve(unsigned char* base, int acap, int gcap, int ecap) {
  WarpScratch s;
  const size_t wa = (acap + 31) / 32, wg = (gcap + 31) / 32;
  uint32_t* u = reinterpret_cast<uint32_t*>(base);
  s.kA = u; u += wa;
  s.kG = u; u += wg;
  s.evA = u; u += acap;
  s.evG = u; u += gcap;
  s.evE = u; u += ecap;
  s.holes = reinterpret_cast<uint16_t*>(align16(reinterpret_cast<size_t>(u)));
  return s;
}

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

// Tail fill: survivors beyond n_surv move, in ascending order, into the holes
// below n_surv, also in ascending order. keep bits cover [0, n).
__device__ __noinline__ void tail_fill_move(const SpeciesPtrs& s, long base, const uint32_t* keep, int n, int n_surv,
                                            uint16_t* holes) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  int run = 0;
  for (int b0 = 0; b0 < n_surv; b0 += 32) {
    const int i = b0 + lane;
    const bool h = i < n_surv && !bit(keep, i);
    const unsigned m = __ballot_sync(kFull, h);
    if (h) holes[run + __popc(m & lt)] = (uint16_t)i;
    run += __popc(m);
  }
  __syncwarp();
  run = 0;
  for (int b0 = n_surv; b0 < n; b0 += 32) {
    const int i = b0 + lane;
    const bool mv = i < n && bit(keep, i);
    const unsigned m = __ballot_sync(kFull, mv);
    if (mv) {
      const long src = base + i;
      const long dst = base + holes[run + __popc(m & lt)];
      write_particle(s, dst, s.w[src], s.px[src], s.py[src], s.pz[src], s.x[src], s.y[src], s.z[src]);
    }
    run += __popc(m);
  }
}

// Word (slot & 3) of the Philox block of quad (slot >> 2), where lane l of the
// warp holds the block of quad (chunk_first_quad + l): four shuffles and a
// select, instead of four lanes recomputing the same block.
__device__ __forceinline__ uint32_t shfl_word(const uint4& r, int sub, int lane) {
  const int src = 8 * sub + (lane >> 2);
  const uint32_t wx = __shfl_sync(kFull, r.x, src), wy = __shfl_sync(kFull, r.y, src);
  const uint32_t wz = __shfl_sync(kFull, r.z, src), ww = __shfl_sync(kFull, r.w, src);
  const int j = lane & 3;
  return j == 0 ? wx : (j == 1 ? wy : (j == 2 ? wz : ww));
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
__device__ __forceinline__ bool no_conversion(float w, float p2, float c_s, float Acoef, float inv_wref, float u) {
  const float s = p2 * c_s;
  const float Fb = s < 2.5f ? 0.5f * s : __logf(1.0f + s);
  const float lb = w * Acoef * Fb * inv_wref * 1.0001f;
  return u <= 1.0f - lb - 1e-6f;
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

// Affine remap and temperature update of one cell (Sec. II.J). dE/dP: this
// step's exchange (keV, m_e c). Returns 1 when the cell was remapped.
__device__ __noinline__ int feedback_cell(const StepArgs& A, int cell, long ebase, int ne, double dE, double dPx,
                                          double dPy, double dPz, bool has_x) {
  int remapped = 0;
  const int lane = lane_id();
  double* rs = A.res + (size_t)cell * 4;
  const double rE = rs[0], rPx = rs[1], rPy = rs[2], rPz = rs[3];
  const bool has_res = nz64(rE) || nz64(rPx) || nz64(rPy) || nz64(rPz);
  float* mom = A.mom + (size_t)cell * kMomLen;
  const float W = mom[M_W], Px = mom[M_PX], Py = mom[M_PY], Pz = mom[M_PZ], U2 = mom[M_U2], var = mom[M_VAR];
  float var_new = var;
  double s1d = 0.0, bx = 0.0, by = 0.0, bz = 0.0, applied_E = 0.0, vnd = 0.0;
  double nrE = 0.0, nrPx = 0.0, nrPy = 0.0, nrPz = 0.0;
  if (has_x || has_res) {
    const double qE = dE + rE, qPx = dPx + rPx, qPy = dPy + rPy, qPz = dPz + rPz;
    nrE = qE;
    nrPx = qPx;
    nrPy = qPy;
    nrPz = qPz;
    // Exchanges below 2^-22 of the cell's kinetic energy (or momentum
    // spread) cannot be represented by binary32 momenta; they stay pending.
    const float ekin = 0.5f * U2 * kMeC2f;
    const float prms = sqrtf(fmaxf(U2 * W, 0.f));
    const bool big = fabsf((float)qE) >= 2.384185791015625e-07f * ekin ||
                     sqrtf((float)(qPx * qPx + qPy * qPy + qPz * qPz)) >= 2.384185791015625e-07f * prms;
    if (W > 0.f && big) {
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
      const RemapOut r = remap_electrons(A, ebase, ne, (float)s1d, (float)bx, (float)by, (float)bz);
      applied_E = r.applied_E;
      nrE = qE - r.applied_E;
      nrPx = qPx - r.apx;
      nrPy = qPy - r.apy;
      nrPz = qPz - r.apz;
      var_new = (float)vnd;
      if (lane == 0) {
        mom[M_W] = r.mW;
        mom[M_PX] = r.mPx;
        mom[M_PY] = r.mPy;
        mom[M_PZ] = r.mPz;
        mom[M_U2] = r.mU2;
        mom[M_VAR] = fmaxf(0.f, r.mU2 - (r.mPx * r.mPx + r.mPy * r.mPy + r.mPz * r.mPz) / r.mW);
      }
      remapped = 1;
    }
    if (lane == 0) {
      rs[0] = nrE;
      rs[1] = nrPx;
      rs[2] = nrPy;
      rs[3] = nrPz;
    }
  }
  if (A.diag_enable && lane == 0) {
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
    dg[AXPIC_CD_VAR_NEW] = remapped ? vnd : (double)var;
    dg[AXPIC_CD_W] = W;
    dg[AXPIC_CD_APPLIED_E] = applied_E;
    dg[AXPIC_CD_RES_E] = nrE;
    dg[AXPIC_CD_RES_PX] = nrPx;
    dg[AXPIC_CD_RES_PY] = nrPy;
    dg[AXPIC_CD_RES_PZ] = nrPz;
  }
  // temperature (Eqs. Te_est, Te_relax), then the record's temperature half
  if (A.T_mode == 2 && W > 0.f) {
    // T stays FP64; the relaxation step is formed in binary32 and added once
    const double T = A.T[cell];
    const float Tf = (float)T;
    const float Test = (kMeC2f / 3.0f) * var_new / W;
    const float dT = A.relax_r * (Test - Tf);
    double Tn = T + (double)dT;
    const float Tnf = Tf + dT;
    if (Tnf <= A.T_floor_f || Tnf >= A.T_ceil_f) Tn = fmin(fmax(Tn, A.T_floor), A.T_ceil);
    float rec[kRecLen];
    const float4* ri = reinterpret_cast<const float4*>(A.rec + (size_t)cell * kRecLen);
#pragma unroll
    for (int i = 0; i < kRecLen / 4; ++i) {
      const float4 v = ri[i];
      rec[4 * i] = v.x;
      rec[4 * i + 1] = v.y;
      rec[4 * i + 2] = v.z;
      rec[4 * i + 3] = v.w;
    }
    compute_temperature(A.cc, (float)Tn, rec);
    __syncwarp();
    if (lane == 0) {
      A.T[cell] = Tn;
      float4* r4 = reinterpret_cast<float4*>(A.rec + (size_t)cell * kRecLen);
      r4[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
      r4[1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
    }
  }
  return remapped;
}

// Appends (slot | K << 16) for the lanes with K > 0 to an ascending list.
__device__ __forceinline__ void append_events(uint32_t* list, int& n, int slot, int K, unsigned lt) {
  const unsigned m = __ballot_sync(kFull, K > 0);
  if (m) {
    if (K > 0) list[n + __popc(m & lt)] = (uint32_t)slot | ((uint32_t)K << 16);
    n += __popc(m);
  }
}

// ---------------------------------------------------------------- the cell
template <int PH>
__device__ __forceinline__ void process_cell(const StepArgs& A, int cell, WarpScratch& S, const Cnt& cnt) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t gcell = A.cell_base + (uint32_t)cell;
  const int mask = A.mask;
  // the cell's record is read where needed (L1-resident, 64 B)
  const float* rec = A.rec + (size_t)cell * kRecLen;
  // s = |p|^2 * c_s for the conversion guards
  const float c_s = kMeC2f * kMeC2f * rec[R_FOURK2];
  // counts come from the caller's arrays: clamp them to the slab capacity
  const int ne = min(max(A.e.count[cell], 0), A.e.cap);
  const int nqe = (ne + 3) >> 2;
  const int ng_start = min(max(A.g.count[cell], 0), A.g.cap);
  int ng = ng_start;
  int na = min(max(A.a.count[cell], 0), A.a.cap);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  Lane64 x64;
  double xa[4] = {0.0, 0.0, 0.0, 0.0};  // reduced absorb exchange (same order as separate calls)
  bool xa_any = false;
  // particles present at the start of the step: counted by the absorb phase,
  // or by the emit phase when no absorb ran this step
  if (lane == 0 && ((PH & PH_ABSORB) || ((PH & PH_EMIT) && !A.use_snapshot))) {
    cnt.add(C_NE, ne);
    cnt.add(C_NG, ng_start);
    cnt.add(C_NA, na);
    cnt.add(C_CELLS, 1);
  }

  // ------------------------------------------------------------ absorb
  int NPg = 0;
  if (PH & PH_ABSORB) {
    if (PH == PH_ABSORB && lane == 0) A.photon_start[cell] = ng;
    const int na0 = na;
    const bool prim = mask & AXPIC_CH_PRIMAKOFF;
    const bool bath = mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS);
    int n_surv_a = 0, nev = 0;
    for (int c0 = 0; c0 < na0; c0 += 128) {
      const uint32_t q = (uint32_t)(c0 >> 2) + lane;
      uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
      if ((int)(4 * q) < na0) {
        if (prim) rP = philox4x32_10(make_uint4(A.step, gcell, q, S_PRIM_INV << 24), A.key0, A.key1);
        if (bath) rA = philox4x32_10(make_uint4(A.step, gcell, q, S_ABSORB << 24), A.key0, A.key1);
      }
      for (int sb = 0; sb < 4 && c0 + 32 * sb < na0; ++sb) {
        const int slot = c0 + 32 * sb + lane;
        const uint32_t wP = shfl_word(rP, sb, lane);
        const uint32_t wA = shfl_word(rA, sb, lane);
        int K = 0;
        bool keep = false;
        if (slot < na0) {
          const long g = abase + slot;
          const float w = A.a.w[g], px = A.a.px[g], py = A.a.py[g], pz = A.a.pz[g];
          const float p2 = px * px + py * py + pz * pz;
          bool fast = A.absorb_mode == 0;
          if (fast && prim) fast = no_conversion(w, p2, c_s, rec[R_APINV], A.inv_w_gref, u23(wP));
          if (fast && bath) fast = no_absorption(rec, A, mask, sqrtf(p2) * kMeC2f * rec[R_INVT], u23(wA));
          if (fast) {
            keep = w > 0.f;
          } else {
            const AxionDecision d = axion_decide_slow(A, cell, mask, w, px, py, pz, wP, wA);
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
              if (d.K == 0 && d.wnew != w) A.a.w[g] = d.wnew;  // K > 0 slots are written in pass 2
            }
            K = d.K;
            keep = d.keep;
            NPg += d.K;
          }
        }
        const unsigned kb = __ballot_sync(kFull, keep);
        if (lane == 0) S.kA[(c0 + 32 * sb) >> 5] = kb;
        n_surv_a += __popc(kb);
        append_events(S.evA, nev, slot, K, lt);
      }
    }
    __syncwarp();
    // (a) photon products of a->gamma after the photons present; kept
    // parents get their depleted weight in place
    if (nev > 0) {
      NPg = warp_sum_i(NPg);
      int run = 0;
      for (int i0 = 0; i0 < nev; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t e = i < nev ? S.evA[i] : 0u;
        const int K = e >> 16;
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        if (K) {
          const int slot = e & 0xFFFF;
          const uint32_t q = slot >> 2;
          uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
          if (prim) rP = philox4x32_10(make_uint4(A.step, gcell, q, S_PRIM_INV << 24), A.key0, A.key1);
          if (bath) rA = philox4x32_10(make_uint4(A.step, gcell, q, S_ABSORB << 24), A.key0, A.key1);
          const long src = abase + slot;
          const float w = A.a.w[src], px = A.a.px[src], py = A.a.py[src], pz = A.a.pz[src];
          const float xx = A.a.x[src], yy = A.a.y[src], zz = A.a.z[src];
          const AxionDecision d = axion_decide_slow(A, cell, mask, w, px, py, pz, word(rP, slot & 3), word(rA, slot & 3));
          for (int k = 0; k < K; ++k, ++off) {
            const int dst = ng + off;
            if (dst < A.g.cap) write_particle(A.g, gbase + dst, d.wprod, px, py, pz, xx, yy, zz);
            else cnt.add(C_DROP, 1);
          }
          if (d.keep) A.a.w[src] = d.wnew;
        }
        run += tot;
      }
      ng = min(ng + NPg, A.g.cap);
    } else {
      NPg = 0;
    }
    __syncwarp();
    // (b) tail-fill compaction of the axions
    if (n_surv_a < na0) tail_fill_move(A.a, abase, S.kA, na0, n_surv_a, S.holes);
    __syncwarp();
    na = n_surv_a;
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
    int NPa = 0;
    int n_surv_g = ng_tot;
    const bool prim = mask & AXPIC_CH_PRIMAKOFF;
    int nevg = 0;
    if (prim) {
      for (int i = lane; i < (ng_tot + 31) / 32; i += 32) S.kG[i] = 0u;
      __syncwarp();
      int keep_cnt = 0;
      for (int c0 = 0; c0 < ng0; c0 += 128) {
        const uint32_t q = (uint32_t)(c0 >> 2) + lane;
        uint4 r = make_uint4(0, 0, 0, 0);
        if ((int)(4 * q) < ng0) r = philox4x32_10(make_uint4(A.step, gcell, q, S_PRIM_FWD << 24), A.key0, A.key1);
        for (int sb = 0; sb < 4 && c0 + 32 * sb < ng0; ++sb) {
          const int slot = c0 + 32 * sb + lane;
          const uint32_t wd = shfl_word(r, sb, lane);
          int K = 0;
          bool keep = false;
          if (slot < ng0) {
            const long g = gbase + slot;
            const float w = A.g.w[g], px = A.g.px[g], py = A.g.py[g], pz = A.g.pz[g];
            if (no_conversion(w, px * px + py * py + pz * pz, c_s, rec[R_AP], A.inv_w_a, u23(wd))) {
              keep = w > 0.f;
            } else {
              const PhotonDecision d = photon_decide_slow(A, cell, w, px, py, pz, wd);
              cnt.add(C_CAP, d.capped);
              cnt.add(C_CLAMP, d.over);
              cnt.add(C_EV_P, d.K);
              K = d.K;
              keep = d.wrem > 0.f;
              NPa += d.K;
            }
          }
          const unsigned kb = __ballot_sync(kFull, keep);
          if (lane == 0) S.kG[(c0 + 32 * sb) >> 5] = kb;
          keep_cnt += __popc(kb);
          append_events(S.evG, nevg, slot, K, lt);
        }
      }
      __syncwarp();
      // photons appended after ng0 (a->gamma products) are kept as they are
      for (int i = ng0 + lane; i < ng_tot; i += 32) atomicOr(&S.kG[i >> 5], 1u << (i & 31));
      n_surv_g = keep_cnt + (ng_tot - ng0);
      if (nevg > 0) NPa = warp_sum_i(NPa);
      else NPa = 0;
    }
    // electron decisions: one Philox block per quad; the Compton-like and
    // bremsstrahlung processes of an electron are drawn as their sum, and
    // with the cell's cached common weight lambda and e^-lambda are shared
    const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
    int NE = 0, neve = 0;
    if (eC || eB) {
      const float wu = A.mom[(size_t)cell * kMomLen + M_WU];
      float lsum_u = 0.f, F0 = 1.f;
      bool capC = false, capB = false;
      if (wu > 0.f) {
        float fac;
        const float lc = eC ? cap_lambda(wu * rec[R_CC], A.lam_cap, &fac, &capC) : 0.f;
        const float lb = eB ? cap_lambda(wu * rec[R_CB], A.lam_cap, &fac, &capB) : 0.f;
        lsum_u = lc + lb;
        F0 = expf(-lsum_u);
      }
      for (int q0 = 0; q0 < nqe; q0 += 32) {
        const int q = q0 + lane;
        uint32_t kw = 0;
        if (q < nqe) {
          uint4 r = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_EMIT_E << 24), A.key0, A.key1);
          const int nj = min(4, ne - 4 * q);
          if (wu > 0.f) {
            cnt.add(C_CAP, nj * ((eC && capC) + (eB && capB)));
#pragma unroll
            for (int j = 0; j < 4; ++j, rot(r)) {
              if (j >= nj) break;
              const float u = u23(r.x);
              if (u > F0) kw |= (uint32_t)poisson_inv(u, lsum_u) << (8 * j);
            }
          } else {
            float4 w4 = ld4(A.e.w + ebase + 4 * q);
#pragma unroll 1
            for (int j = 0; j < nj; ++j, rot(w4), rot(r)) {
              float fac;
              bool cc = false, cb = false;
              const float lc = eC ? cap_lambda(w4.x * rec[R_CC], A.lam_cap, &fac, &cc) : 0.f;
              const float lb = eB ? cap_lambda(w4.x * rec[R_CB], A.lam_cap, &fac, &cb) : 0.f;
              cnt.add(C_CAP, cc + cb);
              kw |= (uint32_t)poisson_inv(u23(r.x), lc + lb) << (8 * j);
            }
          }
        }
        // ascending event list: lanes hold 4 consecutive slots each
        if (__any_sync(kFull, kw != 0)) {
          const int ne_l = (kw & 0xFF ? 1 : 0) + (kw & 0xFF00 ? 1 : 0) + (kw & 0xFF0000 ? 1 : 0) + (kw >> 24 ? 1 : 0);
          int tot;
          int at = neve + warp_excl_scan(ne_l, &tot);
          for (int j = 0; j < 4; ++j) {
            const int K = (kw >> (8 * j)) & 0xFF;
            if (K) {
              S.evE[at++] = (uint32_t)(4 * q + j) | ((uint32_t)K << 16);
              NE += K;
            }
          }
          neve += tot;
        }
      }
      if (neve > 0) NE = warp_sum_i(NE);
    }
    __syncwarp();
    // (c) axion products of photons after the surviving axions; kept parents
    // get their depleted weight in place
    const int abase_new = na;
    if (nevg > 0) {
      int run = 0;
      for (int i0 = 0; i0 < nevg; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t e = i < nevg ? S.evG[i] : 0u;
        const int K = e >> 16;
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        if (K) {
          const int slot = e & 0xFFFF;
          const uint4 r =
              philox4x32_10(make_uint4(A.step, gcell, (uint32_t)(slot >> 2), S_PRIM_FWD << 24), A.key0, A.key1);
          const long src = gbase + slot;
          const float w = A.g.w[src], px = A.g.px[src], py = A.g.py[src], pz = A.g.pz[src];
          const float xx = A.g.x[src], yy = A.g.y[src], zz = A.g.z[src];
          const PhotonDecision d = photon_decide_slow(A, cell, w, px, py, pz, word(r, slot & 3));
          for (int k = 0; k < K; ++k, ++off) {
            const int dst = abase_new + off;
            if (dst < A.a.cap) {
              write_particle(A.a, abase + dst, d.wprod, px, py, pz, xx, yy, zz);
              if (A.tally_enable) tally_add(A, 0, d.wprod, d.om);
            } else {
              cnt.add(C_DROP, 1);
            }
          }
          if (d.wrem > 0.f) A.g.w[src] = d.wrem;
        }
        run += tot;
      }
    }
    // (d) electron events, in electron then event order; event k of
    // electron i: cos theta, phi, energy and channel from one Philox block
    if (neve > 0) {
      int run = 0;
      const float* tabC = A.tables + TAB_COMPTON * kTableN;
      const float* tabB = A.tables + TAB_BREMS * kTableN;
      for (int i0 = 0; i0 < neve; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t e = i < neve ? S.evE[i] : 0u;
        const int K = e >> 16;
        int tot;
        int off = run + warp_excl_scan(K, &tot);
        if (K) {
          const int slot = e & 0xFFFF;
          const long src = ebase + slot;
          const float w = A.e.w[src];
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
            if (isC) cnt.add(C_EV_C, 1);
            else cnt.add(C_EV_B, 1);
          }
        }
        run += tot;
      }
    }
    na = min(na + NPa + NE, A.a.cap);
    __syncwarp();
    // (e) tail-fill compaction of the photons
    if (prim) {
      if (n_surv_g < ng_tot) tail_fill_move(A.g, gbase, S.kG, ng_tot, n_surv_g, S.holes);
      ng = n_surv_g;
    }
  }
  if (lane == 0 && (PH & (PH_ABSORB | PH_EMIT))) {
    A.a.count[cell] = na;
    A.g.count[cell] = ng;
  }

  // ------------------------------------------------------------ exchange
  // absorb and emit contributions are reduced separately and added in that
  // order, exactly as the separate calls accumulate them in the buffer
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0;
  bool has_x = false;
  if (PH & (PH_ABSORB | PH_EMIT)) {
    double xe[4] = {0.0, 0.0, 0.0, 0.0};
    bool xe_any = false;
    if (__any_sync(kFull, x64.any)) {
      xe[0] = warp_sum_d(x64.dE);
      xe[1] = warp_sum_d(x64.dPx);
      xe[2] = warp_sum_d(x64.dPy);
      xe[3] = warp_sum_d(x64.dPz);
      xe_any = true;
    }
    if (!(PH & PH_FEEDBACK)) {
      if (lane == 0 && (xa_any || xe_any)) {
        double* xb = A.xbuf + (size_t)cell * 4;
        if (PH & PH_ABSORB) {
          xb[0] += xa[0];
          xb[1] += xa[1];
          xb[2] += xa[2];
          xb[3] += xa[3];
        } else {
          xb[0] += xe[0];
          xb[1] += xe[1];
          xb[2] += xe[2];
          xb[3] += xe[3];
        }
      }
      return;
    }
    has_x = xa_any || xe_any;
    if (has_x) {
      dE = (0.0 + xa[0]) + xe[0];
      dPx = (0.0 + xa[1]) + xe[1];
      dPy = (0.0 + xa[2]) + xe[2];
      dPz = (0.0 + xa[3]) + xe[3];
    }
  } else {
    double* xb = A.xbuf + (size_t)cell * 4;
    dE = xb[0];
    dPx = xb[1];
    dPy = xb[2];
    dPz = xb[3];
    has_x = nz64(dE) || nz64(dPx) || nz64(dPy) || nz64(dPz);
    __syncwarp();
    if (lane == 0 && has_x) {
      xb[0] = 0.0;
      xb[1] = 0.0;
      xb[2] = 0.0;
      xb[3] = 0.0;
    }
  }
  if (PH & PH_FEEDBACK) {
    if (feedback_cell(A, cell, ebase, ne, dE, dPx, dPy, dPz, has_x) && lane == 0) {
      cnt.add(C_REMAP, 1);
      cnt.add(C_REMAP_E, ne);
    }
  }
}

// Minimum resident CTAs of 128 threads per SM the register allocation aims for.
#ifndef AXPIC_STEP_MIN_CTAS
#define AXPIC_STEP_MIN_CTAS 8
#endif

template <int PH>
__global__ void __launch_bounds__(128, AXPIC_STEP_MIN_CTAS) step_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  // per-warp counters: each warp flushes its own, so no warp waits for the
  // slowest cell of its CTA
  __shared__ unsigned long long warp_cnt[4][kNumCounters];
  const int wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * nw + wid;
  if (lane < kNumCounters) warp_cnt[wid][lane] = 0ull;
  __syncwarp();
  const Cnt cnt{warp_cnt[wid]};
  if (cell < A.ncells) {
    const size_t bytes = warp_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
    WarpScratch S = carve(smem + wid * bytes, A.a.cap, A.g.cap, A.e.cap);
    process_cell<PH>(A, cell, S, cnt);
  }
  __syncwarp();
  if (lane < kNumCounters) {
    const unsigned long long v = warp_cnt[wid][lane];
    if (v) atomicAdd(A.counters + (size_t)blockIdx.x * kNumCounters + lane, v);
    if (lane == C_DROP && v) atomicOr(A.err, ERR_CAPACITY);
  }
}

size_t step_smem_per_warp(int acap, int gcap, int ecap) { return warp_scratch_bytes(acap, gcap, ecap); }

template <int PH>
static cudaError_t launch(const StepArgs& A, int warps, cudaStream_t st) {
  const size_t per = warp_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
  const int grid = (A.ncells + warps - 1) / warps;
  if (grid == 0) return cudaSuccess;
  step_kernel<PH><<<grid, warps * 32, per * warps, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st) {
  switch (phases) {
    case PH_ABSORB: return launch<PH_ABSORB>(A, warps, st);
    case PH_EMIT: return launch<PH_EMIT>(A, warps, st);
    case PH_FEEDBACK: return launch<PH_FEEDBACK>(A, warps, st);
    case PH_ALL: {
      // one step as three kernels: each phase's code and registers stay small
      // (a single fused kernel measured twice as slow); the exchange passes
      // through the per-cell FP64 buffer in the same summation order
      cudaError_t e = launch<PH_ABSORB>(A, warps, st);
      if (e) return e;
      StepArgs B = A;
      B.use_snapshot = 1;
      if ((e = launch<PH_EMIT>(B, warps, st))) return e;
      return launch<PH_FEEDBACK>(A, warps, st);
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t set_step_smem_limits(size_t bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(step_kernel<PH_ABSORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  if ((e = cudaFuncSetAttribute(step_kernel<PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  return cudaFuncSetAttribute(step_kernel<PH_FEEDBACK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace axpic
