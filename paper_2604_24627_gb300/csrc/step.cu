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

// Per-warp shared scratch, carved from dynamic shared memory.
struct WarpScratch {
  float *WNa, *WPa, *WNg, *WPg;
  uint32_t *kA, *cA, *kG, *cG;
  uint16_t* holes;
  uint8_t *Ka, *Kg, *KC, *KB;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t warp_scratch_bytes(int acap, int gcap, int ecap) {
  const size_t wa = (acap + 31) / 32, wg = (gcap + 31) / 32;
  size_t b = 4 * (2 * (size_t)acap + 2 * (size_t)gcap);
  b += 4 * (2 * wa + 2 * wg);
  b += align16(2 * (size_t)(acap > gcap ? acap : gcap));
  b += align16((size_t)acap + gcap + 2 * (size_t)ecap);
  return align16(b);
}

__device__ inline WarpScratch carve(unsigned char* base, int acap, int gcap, int ecap) {
  WarpScratch s;
  const size_t wa = (acap + 31) / 32, wg = (gcap + 31) / 32;
  float* f = reinterpret_cast<float*>(base);
  s.WNa = f; f += acap;
  s.WPa = f; f += acap;
  s.WNg = f; f += gcap;
  s.WPg = f; f += gcap;
  uint32_t* u = reinterpret_cast<uint32_t*>(f);
  s.kA = u; u += wa;
  s.cA = u; u += wa;
  s.kG = u; u += wg;
  s.cG = u; u += wg;
  unsigned char* c = reinterpret_cast<unsigned char*>(u);
  s.holes = reinterpret_cast<uint16_t*>(c);
  c += align16(2 * (size_t)(acap > gcap ? acap : gcap));
  s.Ka = c; c += acap;
  s.Kg = c; c += gcap;
  s.KC = c; c += ecap;
  s.KB = c;
  return s;
}

struct Lane64 {
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0;
};

struct LaneCnt {
  unsigned c[kNumCounters];
  __device__ LaneCnt() {
#pragma unroll
    for (int i = 0; i < kNumCounters; ++i) c[i] = 0;
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

__device__ __forceinline__ void tally_add(const StepArgs& A, int ch, float w, float E) {
  const int k = (int)floorf(E * A.inv_dE_bin);
  const double wE = (double)w * (double)E;
  if (k >= 0 && k < A.nbins) atomicAdd(A.tally + ch * A.nbins + k, wE);
  atomicAdd(A.tally + 3 * A.nbins + ch, (double)w);
  atomicAdd(A.tally + 3 * A.nbins + 3 + ch, wE);
}

// Tail fill: survivors beyond n_surv move, in ascending order, into the holes
// below n_surv, also in ascending order. keep bits cover [0, n).
__device__ void tail_fill_move(const SpeciesPtrs& s, long base, const uint32_t* keep, int n, int n_surv,
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

template <int PH>
__device__ void process_cell(const StepArgs& A, int cell, WarpScratch& S, LaneCnt& cnt) {
  const int lane = lane_id();
  const uint32_t gcell = A.cell_base + (uint32_t)cell;
  const int mask = A.mask;
  float rec[kRecLen];
  {
    const float4* r4 = reinterpret_cast<const float4*>(A.rec + (size_t)cell * kRecLen);
#pragma unroll
    for (int i = 0; i < kRecLen / 4; ++i) {
      const float4 v = __ldg(r4 + i);
      rec[4 * i] = v.x;
      rec[4 * i + 1] = v.y;
      rec[4 * i + 2] = v.z;
      rec[4 * i + 3] = v.w;
    }
  }
  // counts come from the caller's arrays: clamp them to the slab capacity
  const int ne = min(max(A.e.count[cell], 0), A.e.cap);
  const int nqe = (ne + 3) >> 2;
  const int ng_start = min(max(A.g.count[cell], 0), A.g.cap);
  int ng = ng_start;
  int na = min(max(A.a.count[cell], 0), A.a.cap);
  const long abase = (long)cell * A.a.cap;
  const long gbase = (long)cell * A.g.cap;
  const long ebase = (long)cell * A.e.cap;
  Lane64 x64;       // absorb-phase exchange, then emit-phase exchange
  double xa[4] = {0.0, 0.0, 0.0, 0.0};  // reduced absorb exchange (same order as separate calls)
  if (lane == 0 && (PH & (PH_ABSORB | PH_EMIT))) {
    cnt.c[C_NE] += ne;
    cnt.c[C_NG] += ng_start;
    cnt.c[C_NA] += na;
    cnt.c[C_CELLS] += 1;
  }

  // ------------------------------------------------------------ absorb
  int n_surv_a = na;
  int NPg = 0;
  if (PH & PH_ABSORB) {
    if (PH == PH_ABSORB && lane == 0) A.photon_start[cell] = ng;
    const int na0 = na;
    const int nqa = (na0 + 3) >> 2;
    for (int i = lane; i < (na0 + 31) / 32; i += 32) {
      S.kA[i] = 0u;
      S.cA[i] = 0u;
    }
    __syncwarp();
    int keep_cnt = 0;
    for (int q = lane; q < nqa; q += 32) {
      const long b = abase + 4 * q;
      const float4 w4 = ld4(A.a.w + b), x4 = ld4(A.a.px + b), y4 = ld4(A.a.py + b), z4 = ld4(A.a.pz + b);
      uint4 rP = make_uint4(0, 0, 0, 0), rA = make_uint4(0, 0, 0, 0);
      if (mask & AXPIC_CH_PRIMAKOFF)
        rP = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_PRIM_INV << 24), A.key0, A.key1);
      if (mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS))
        rA = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_ABSORB << 24), A.key0, A.key1);
      uint32_t kb = 0, cb = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int slot = 4 * q + j;
        if (slot >= na0) break;
        const float w = f4(w4, j), px = f4(x4, j), py = f4(y4, j), pz = f4(z4, j);
        const float om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
        float wrem = w, wprod = 0.f;
        int K = 0;
        if (mask & AXPIC_CH_PRIMAKOFF) {
          const float P = prim_prob(rec, om, rec[R_APINV]);
          const float lam = w * P * A.inv_w_gref;
          float fac;
          bool capped;
          const float le = cap_lambda(lam, A.lam_cap, &fac, &capped);
          cnt.c[C_CAP] += capped;
          K = poisson_inv(u23(word(rP, j)), le);
          if (K > 0) {
            bool over;
            wprod = deplete(w, K, capped ? A.w_gref * fac : A.w_gref, &wrem, &over);
            cnt.c[C_CLAMP] += over;
            cnt.c[C_EV_PINV] += K;
          }
        }
        bool keep = wrem > 0.f;
        if (keep && (mask & (AXPIC_CH_COMPTON | AXPIC_CH_BREMS))) {
          const float x = om * rec[R_INVT];
          const float tc = (mask & AXPIC_CH_COMPTON) ? tau_compton(rec, x, A.eq_stats) : 0.f;
          const float tb = (mask & AXPIC_CH_BREMS) ? tau_brems(rec, x, A.brems_am3, A.eq_stats) : 0.f;
          const float tau = tc + tb;
          if (A.absorb_mode == 0) {
            const float P = -expm1f(-tau);
            const float u = u23(word(rA, j));
            if (u < P) {
              x64.dE += (double)wrem * (double)om;
              x64.dPx += (double)wrem * (double)px;
              x64.dPy += (double)wrem * (double)py;
              x64.dPz += (double)wrem * (double)pz;
              keep = false;
              if (u / P < tc / tau) cnt.c[C_ABS_C]++;
              else cnt.c[C_ABS_B]++;
            }
          } else {
            const float wn = wrem * expf(-tau);
            const double lost = (double)wrem - (double)wn;
            x64.dE += lost * (double)om;
            x64.dPx += lost * (double)px;
            x64.dPy += lost * (double)py;
            x64.dPz += lost * (double)pz;
            wrem = wn;
            keep = wrem > 0.f;
          }
        }
        S.Ka[slot] = (uint8_t)K;
        S.WNa[slot] = keep ? wrem : 0.f;
        S.WPa[slot] = wprod;
        NPg += K;
        if (keep) {
          kb |= 1u << j;
          ++keep_cnt;
          if (wrem != w) cb |= 1u << j;
        }
      }
      const int sh = (4 * q) & 31;
      if (kb) atomicOr(&S.kA[(4 * q) >> 5], kb << sh);
      if (cb) atomicOr(&S.cA[(4 * q) >> 5], cb << sh);
    }
    n_surv_a = warp_sum_i(keep_cnt);
    NPg = warp_sum_i(NPg);
    __syncwarp();

    // (a) photon products of a->gamma, appended after the photons present
    if (NPg > 0) {
      int run = 0;
      for (int q0 = 0; q0 < nqa; q0 += 32) {
        const int q = q0 + lane;
        int s = 0;
        if (q < nqa)
          for (int j = 0; j < 4 && 4 * q + j < na0; ++j) s += S.Ka[4 * q + j];
        int tot;
        int off = run + warp_excl_scan(s, &tot);
        if (s > 0) {
          for (int j = 0; j < 4 && 4 * q + j < na0; ++j) {
            const int slot = 4 * q + j;
            const int K = S.Ka[slot];
            if (!K) continue;
            const long src = abase + slot;
            const float px = A.a.px[src], py = A.a.py[src], pz = A.a.pz[src];
            const float xx = A.a.x[src], yy = A.a.y[src], zz = A.a.z[src];
            const float wp = S.WPa[slot];
            for (int k = 0; k < K; ++k, ++off) {
              const int dst = ng + off;
              if (dst < A.g.cap) write_particle(A.g, gbase + dst, wp, px, py, pz, xx, yy, zz);
              else cnt.c[C_DROP]++;
            }
          }
        }
        run += tot;
      }
      ng = min(ng + NPg, A.g.cap);
    }
    __syncwarp();
    // (b) axion weights updated in place, then tail-fill compaction
    for (int q0 = 0; q0 < na0; q0 += 32) {
      const int i = q0 + lane;
      if (i < na0 && bit(S.cA, i)) A.a.w[abase + i] = S.WNa[i];
    }
    __syncwarp();
    if (n_surv_a < na0) tail_fill_move(A.a, abase, S.kA, na0, n_surv_a, S.holes);
    __syncwarp();
    na = n_surv_a;
    if (__any_sync(kFull, x64.dE != 0.0 || x64.dPx != 0.0 || x64.dPy != 0.0 || x64.dPz != 0.0)) {
      xa[0] = warp_sum_d(x64.dE);
      xa[1] = warp_sum_d(x64.dPx);
      xa[2] = warp_sum_d(x64.dPy);
      xa[3] = warp_sum_d(x64.dPz);
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
    const int nqg = (ng0 + 3) >> 2;
    if (prim) {
      for (int i = lane; i < (ng_tot + 31) / 32; i += 32) {
        S.kG[i] = 0u;
        S.cG[i] = 0u;
      }
      __syncwarp();
      int keep_cnt = 0;
      for (int q = lane; q < nqg; q += 32) {
        const long b = gbase + 4 * q;
        const float4 w4 = ld4(A.g.w + b), x4 = ld4(A.g.px + b), y4 = ld4(A.g.py + b), z4 = ld4(A.g.pz + b);
        const uint4 r = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_PRIM_FWD << 24), A.key0, A.key1);
        uint32_t kb = 0, cb = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int slot = 4 * q + j;
          if (slot >= ng0) break;
          const float w = f4(w4, j), px = f4(x4, j), py = f4(y4, j), pz = f4(z4, j);
          const float om = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
          const float P = prim_prob(rec, om, rec[R_AP]);
          const float lam = w * P * A.inv_w_a;
          float fac;
          bool capped;
          const float le = cap_lambda(lam, A.lam_cap, &fac, &capped);
          cnt.c[C_CAP] += capped;
          const int K = poisson_inv(u23(word(r, j)), le);
          float wrem = w, wprod = 0.f;
          if (K > 0) {
            bool over;
            wprod = deplete(w, K, capped ? A.w_a * fac : A.w_a, &wrem, &over);
            cnt.c[C_CLAMP] += over;
            cnt.c[C_EV_P] += K;
          }
          S.Kg[slot] = (uint8_t)K;
          S.WNg[slot] = wrem;
          S.WPg[slot] = wprod;
          NPa += K;
          if (wrem > 0.f) {
            kb |= 1u << j;
            ++keep_cnt;
            if (K > 0) cb |= 1u << j;
          }
        }
        const int sh = (4 * q) & 31;
        if (kb) atomicOr(&S.kG[(4 * q) >> 5], kb << sh);
        if (cb) atomicOr(&S.cG[(4 * q) >> 5], cb << sh);
      }
      // photons appended after ng0 (a->gamma products) are kept as they are
      for (int i = ng0 + lane; i < ng_tot; i += 32) atomicOr(&S.kG[i >> 5], 1u << (i & 31));
      n_surv_g = warp_sum_i(keep_cnt) + (ng_tot - ng0);
      NPa = warp_sum_i(NPa);
    }
    // electron decisions: one Philox block per quad and channel
    const bool eC = mask & AXPIC_CH_COMPTON, eB = mask & AXPIC_CH_BREMS;
    int NE = 0;
    if (eC || eB) {
      for (int q = lane; q < nqe; q += 32) {
        const float4 w4 = ld4(A.e.w + ebase + 4 * q);
        uint4 rC = make_uint4(0, 0, 0, 0), rB = make_uint4(0, 0, 0, 0);
        if (eC) rC = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_COMPTON << 24), A.key0, A.key1);
        if (eB) rB = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)q, S_BREMS << 24), A.key0, A.key1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int slot = 4 * q + j;
          if (slot >= ne) break;
          const float w = f4(w4, j);
          int kc = 0, kbb = 0;
          if (eC) {
            float fac;
            bool capped;
            const float le = cap_lambda(w * rec[R_CC], A.lam_cap, &fac, &capped);
            cnt.c[C_CAP] += capped;
            kc = poisson_inv(u23(word(rC, j)), le);
          }
          if (eB) {
            float fac;
            bool capped;
            const float le = cap_lambda(w * rec[R_CB], A.lam_cap, &fac, &capped);
            cnt.c[C_CAP] += capped;
            kbb = poisson_inv(u23(word(rB, j)), le);
          }
          S.KC[slot] = (uint8_t)kc;
          S.KB[slot] = (uint8_t)kbb;
          NE += kc + kbb;
        }
      }
      NE = warp_sum_i(NE);
    }
    __syncwarp();
    // (c) axion products of photons: appended after the surviving axions
    const int abase_new = na;
    if (NPa > 0) {
      int run = 0;
      for (int q0 = 0; q0 < nqg; q0 += 32) {
        const int q = q0 + lane;
        int s = 0;
        if (q < nqg)
          for (int j = 0; j < 4 && 4 * q + j < ng0; ++j) s += S.Kg[4 * q + j];
        int tot;
        int off = run + warp_excl_scan(s, &tot);
        if (s > 0) {
          for (int j = 0; j < 4 && 4 * q + j < ng0; ++j) {
            const int slot = 4 * q + j;
            const int K = S.Kg[slot];
            if (!K) continue;
            const long src = gbase + slot;
            const float px = A.g.px[src], py = A.g.py[src], pz = A.g.pz[src];
            const float xx = A.g.x[src], yy = A.g.y[src], zz = A.g.z[src];
            const float wp = S.WPg[slot];
            const float E = sqrtf(px * px + py * py + pz * pz) * kMeC2f;
            for (int k = 0; k < K; ++k, ++off) {
              const int dst = abase_new + off;
              if (dst < A.a.cap) {
                write_particle(A.a, abase + dst, wp, px, py, pz, xx, yy, zz);
                if (A.tally_enable) tally_add(A, 0, wp, E);
              } else {
                cnt.c[C_DROP]++;
              }
            }
          }
        }
        run += tot;
      }
    }
    // (d) electron events: Compton-like then bremsstrahlung per electron
    if (NE > 0) {
      int run = 0;
      const float* tabC = A.tables + TAB_COMPTON * kTableN;
      const float* tabB = A.tables + TAB_BREMS * kTableN;
      for (int q0 = 0; q0 < nqe; q0 += 32) {
        const int q = q0 + lane;
        int s = 0;
        if (q < nqe)
          for (int j = 0; j < 4 && 4 * q + j < ne; ++j) s += S.KC[4 * q + j] + S.KB[4 * q + j];
        int tot;
        int off = run + warp_excl_scan(s, &tot);
        if (s > 0) {
          for (int j = 0; j < 4 && 4 * q + j < ne; ++j) {
            const int slot = 4 * q + j;
            const int kc = S.KC[slot], kbb = S.KB[slot];
            if (!(kc + kbb)) continue;
            const long src = ebase + slot;
            const float w = A.e.w[src];
            const float xx = A.e.x[src], yy = A.e.y[src], zz = A.e.z[src];
            for (int ch = 0; ch < 2; ++ch) {
              const int K = ch == 0 ? kc : kbb;
              if (!K) continue;
              float fac;
              bool capped;
              cap_lambda(w * rec[ch == 0 ? R_CC : R_CB], A.lam_cap, &fac, &capped);
              const float wv = capped ? A.w_a * fac : A.w_a;
              const uint32_t stream = ch == 0 ? S_EV_COMPTON : S_EV_BREMS;
              const float* tab = ch == 0 ? tabC : tabB;
              for (int k = 0; k < K; ++k, ++off) {
                const uint4 r = philox4x32_10(make_uint4(A.step, gcell, (uint32_t)slot, (stream << 24) | (uint32_t)k),
                                              A.key0, A.key1);
                const float3 d = iso_dir(u23(r.x), u23(r.y));
                const float E = icdf_lookup(tab, u23(r.z)) * rec[R_T];
                const float pm = E * kInvMeC2f;
                const float px = pm * d.x, py = pm * d.y, pz = pm * d.z;
                const int dst = abase_new + NPa + off;
                if (dst < A.a.cap) {
                  write_particle(A.a, abase + dst, wv, px, py, pz, xx, yy, zz);
                  if (A.tally_enable) tally_add(A, 1 + ch, wv, E);
                } else {
                  cnt.c[C_DROP]++;
                }
                x64.dE -= (double)wv * (double)E;
                x64.dPx -= (double)wv * (double)px;
                x64.dPy -= (double)wv * (double)py;
                x64.dPz -= (double)wv * (double)pz;
                cnt.c[ch == 0 ? C_EV_C : C_EV_B]++;
              }
            }
          }
        }
        run += tot;
      }
    }
    na = min(na + NPa + NE, A.a.cap);
    __syncwarp();
    // (e) photon weights in place, then tail-fill compaction
    if (prim) {
      for (int q0 = 0; q0 < ng0; q0 += 32) {
        const int i = q0 + lane;
        if (i < ng0 && bit(S.cG, i)) A.g.w[gbase + i] = S.WNg[i];
      }
      __syncwarp();
      if (n_surv_g < ng_tot) tail_fill_move(A.g, gbase, S.kG, ng_tot, n_surv_g, S.holes);
      ng = n_surv_g;
    }
  }
  if (lane == 0) {
    if (PH & (PH_ABSORB | PH_EMIT)) {
      A.a.count[cell] = na;
      A.g.count[cell] = ng;
    }
  }

  // ------------------------------------------------------------ exchange
  // absorb and emit contributions are reduced separately and added in that
  // order, exactly as the separate calls accumulate them in the buffer
  double dE = 0.0, dPx = 0.0, dPy = 0.0, dPz = 0.0;
  if (PH & (PH_ABSORB | PH_EMIT)) {
    double xe[4] = {0.0, 0.0, 0.0, 0.0};
    if (__any_sync(kFull, x64.dE != 0.0 || x64.dPx != 0.0 || x64.dPy != 0.0 || x64.dPz != 0.0)) {
      xe[0] = warp_sum_d(x64.dE);
      xe[1] = warp_sum_d(x64.dPx);
      xe[2] = warp_sum_d(x64.dPy);
      xe[3] = warp_sum_d(x64.dPz);
    }
    const bool has_a = xa[0] != 0.0 || xa[1] != 0.0 || xa[2] != 0.0 || xa[3] != 0.0;
    const bool has_e = xe[0] != 0.0 || xe[1] != 0.0 || xe[2] != 0.0 || xe[3] != 0.0;
    if (!(PH & PH_FEEDBACK)) {
      if (lane == 0 && (has_a || has_e)) {
        double* xb = A.xbuf + (size_t)cell * 4;
        const double* src = (PH & PH_ABSORB) ? xa : xe;
        xb[0] += src[0];
        xb[1] += src[1];
        xb[2] += src[2];
        xb[3] += src[3];
      }
      return;
    }
    dE = (0.0 + xa[0]) + xe[0];
    dPx = (0.0 + xa[1]) + xe[1];
    dPy = (0.0 + xa[2]) + xe[2];
    dPz = (0.0 + xa[3]) + xe[3];
  } else {
    double* xb = A.xbuf + (size_t)cell * 4;
    dE = xb[0];
    dPx = xb[1];
    dPy = xb[2];
    dPz = xb[3];
    __syncwarp();
    if (lane == 0 && (dE != 0.0 || dPx != 0.0 || dPy != 0.0 || dPz != 0.0)) {
      xb[0] = 0.0;
      xb[1] = 0.0;
      xb[2] = 0.0;
      xb[3] = 0.0;
    }
  }

  // ------------------------------------------------------------ feedback
  if (PH & PH_FEEDBACK) {
    double* rs = A.res + (size_t)cell * 4;
    const double rE = rs[0], rPx = rs[1], rPy = rs[2], rPz = rs[3];
    const bool has_res = rE != 0.0 || rPx != 0.0 || rPy != 0.0 || rPz != 0.0;
    const bool has_x = dE != 0.0 || dPx != 0.0 || dPy != 0.0 || dPz != 0.0;
    float* mom = A.mom + (size_t)cell * kMomLen;
    float W = mom[M_W], Px = mom[M_PX], Py = mom[M_PY], Pz = mom[M_PZ], U2 = mom[M_U2], var = mom[M_VAR];
    float var_new = var;
    double qE = dE, qPx = dPx, qPy = dPy, qPz = dPz;  // requested this step
    double s1d = 0.0, bx = 0.0, by = 0.0, bz = 0.0, applied_E = 0.0, vnd = var;
    if (has_x || has_res) {
      qE += rE;
      qPx += rPx;
      qPy += rPy;
      qPz += rPz;
      // Exchanges below 2^-22 of the cell's kinetic energy (or momentum
      // spread) cannot be represented by binary32 momenta; they stay pending.
      const float ekin = 0.5f * U2 * kMeC2f;
      const float prms = sqrtf(fmaxf(U2 * W, 0.f));
      const bool big = fabsf((float)qE) >= 2.384185791015625e-07f * ekin ||
                       sqrtf((float)(qPx * qPx + qPy * qPy + qPz * qPz)) >= 2.384185791015625e-07f * prms;
      double nrE = qE, nrPx = qPx, nrPy = qPy, nrPz = qPz;
      if (W > 0.f && big) {
        // Eqs. delta_def, dE_bulk, dE_th, var_new, s_def, b_def (mu = 1)
        const double Wd = W;
        const double dx = qPx / Wd, dy = qPy / Wd, dz = qPz / Wd;
        const double dEb = (2.0 * (dx * Px + dy * Py + dz * Pz) + Wd * (dx * dx + dy * dy + dz * dz)) * 0.5;
        const double dEth = qE / kMeC2 - dEb;
        double S = 1.0;
        if (var > 0.f) {
          vnd = fmax(0.0, (double)var + 2.0 * dEth);
          S = sqrt(vnd / (double)var);
          s1d = ((vnd - (double)var) / (double)var) / (S + 1.0);
        } else {
          vnd = var;
        }
        bx = -s1d * Px / Wd + dx;
        by = -s1d * Py / Wd + dy;
        bz = -s1d * Pz / Wd + dz;
        const float s1 = (float)s1d, fbx = (float)bx, fby = (float)by, fbz = (float)bz;
        // remap p' = p + (s1 p + b), measure what binary32 actually applied
        float aE = 0.f, aPx = 0.f, aPy = 0.f, aPz = 0.f;
        float mW = 0.f, mPx = 0.f, mPy = 0.f, mPz = 0.f, mU2 = 0.f;
        for (int q = lane; q < nqe; q += 32) {
          const long b = ebase + 4 * q;
          const float4 w4 = ld4(A.e.w + b);
          float4 x4 = ld4(A.e.px + b), y4 = ld4(A.e.py + b), z4 = ld4(A.e.pz + b);
          float* xs = reinterpret_cast<float*>(&x4);
          float* ys = reinterpret_cast<float*>(&y4);
          float* zs = reinterpret_cast<float*>(&z4);
          const float* ws = reinterpret_cast<const float*>(&w4);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (4 * q + j >= ne) break;
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
          if (4 * q + 3 < ne) {
            *reinterpret_cast<float4*>(A.e.px + b) = x4;
            *reinterpret_cast<float4*>(A.e.py + b) = y4;
            *reinterpret_cast<float4*>(A.e.pz + b) = z4;
          } else {
            for (int j = 0; j < 4 && 4 * q + j < ne; ++j) {
              A.e.px[b + j] = xs[j];
              A.e.py[b + j] = ys[j];
              A.e.pz[b + j] = zs[j];
            }
          }
        }
        applied_E = warp_sum_d((double)aE) * 0.5 * kMeC2;
        const double apx = warp_sum_d((double)aPx), apy = warp_sum_d((double)aPy), apz = warp_sum_d((double)aPz);
        mW = warp_sum_f(mW);
        mPx = warp_sum_f(mPx);
        mPy = warp_sum_f(mPy);
        mPz = warp_sum_f(mPz);
        mU2 = warp_sum_f(mU2);
        nrE = qE - applied_E;
        nrPx = qPx - apx;
        nrPy = qPy - apy;
        nrPz = qPz - apz;
        var_new = (float)vnd;
        if (lane == 0) {
          mom[M_W] = mW;
          mom[M_PX] = mPx;
          mom[M_PY] = mPy;
          mom[M_PZ] = mPz;
          mom[M_U2] = mU2;
          mom[M_VAR] = fmaxf(0.f, mU2 - (mPx * mPx + mPy * mPy + mPz * mPz) / mW);
        }
        cnt.c[C_REMAP] += (lane == 0);
        cnt.c[C_REMAP_E] += (lane == 0) ? ne : 0;
      }
      if (lane == 0) {
        rs[0] = nrE;
        rs[1] = nrPx;
        rs[2] = nrPy;
        rs[3] = nrPz;
      }
      if (A.diag_enable && lane == 0) {
        double* dg = A.diag + (size_t)cell * AXPIC_CELL_DIAG_LEN;
        dg[AXPIC_CD_RES_E] = nrE;
        dg[AXPIC_CD_RES_PX] = nrPx;
        dg[AXPIC_CD_RES_PY] = nrPy;
        dg[AXPIC_CD_RES_PZ] = nrPz;
      }
    } else if (A.diag_enable && lane == 0) {
      double* dg = A.diag + (size_t)cell * AXPIC_CELL_DIAG_LEN;
      dg[AXPIC_CD_RES_E] = 0.0;
      dg[AXPIC_CD_RES_PX] = 0.0;
      dg[AXPIC_CD_RES_PY] = 0.0;
      dg[AXPIC_CD_RES_PZ] = 0.0;
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
      dg[AXPIC_CD_VAR_NEW] = vnd;
      dg[AXPIC_CD_W] = W;
      dg[AXPIC_CD_APPLIED_E] = applied_E;
    }
    // temperature (Eqs. Te_est, Te_relax), then the record's T part
    if (A.T_mode == 2 && W > 0.f) {
      const double T = A.T[cell];
      const float Test = (kMeC2f / 3.0f) * var_new / W;
      double Tn = T + (double)(A.relax_r * (Test - (float)T));
      Tn = fmin(fmax(Tn, A.T_floor), A.T_ceil);
      if (lane == 0) A.T[cell] = Tn;
      compute_temperature(A.cc, (float)Tn, rec);
      if (lane == 0) {
        float4* r4 = reinterpret_cast<float4*>(A.rec + (size_t)cell * kRecLen);
        r4[0] = make_float4(rec[0], rec[1], rec[2], rec[3]);
        r4[1] = make_float4(rec[4], rec[5], rec[6], rec[7]);
      }
    }
  }
}

template <int PH>
__global__ void __launch_bounds__(256) step_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long cta_cnt[kNumCounters];
  const int wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int cell = blockIdx.x * nw + wid;
  if (threadIdx.x < kNumCounters) cta_cnt[threadIdx.x] = 0ull;
  __syncthreads();
  LaneCnt cnt;
  if (cell < A.ncells) {
    const size_t bytes = warp_scratch_bytes(A.a.cap, A.g.cap, A.e.cap);
    WarpScratch S = carve(smem + wid * bytes, A.a.cap, A.g.cap, A.e.cap);
    process_cell<PH>(A, cell, S, cnt);
  }
#pragma unroll
  for (int i = 0; i < kNumCounters; ++i) {
    const int v = warp_sum_i((int)cnt.c[i]);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cta_cnt[i], (unsigned long long)v);
  }
  __syncthreads();
  if (threadIdx.x < kNumCounters && cta_cnt[threadIdx.x])
    A.counters[(size_t)blockIdx.x * kNumCounters + threadIdx.x] += cta_cnt[threadIdx.x];
  if (threadIdx.x == 0 && cta_cnt[C_DROP]) atomicOr(A.err, ERR_CAPACITY);
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
    case PH_ALL: return launch<PH_ALL>(A, warps, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t set_step_smem_limits(size_t bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(step_kernel<PH_ABSORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  if ((e = cudaFuncSetAttribute(step_kernel<PH_EMIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  if ((e = cudaFuncSetAttribute(step_kernel<PH_FEEDBACK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes))) return e;
  return cudaFuncSetAttribute(step_kernel<PH_ALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace axpic
