// Internal definitions shared by the CUDA translation units of libaxpic.
//
// Device helpers: Philox4x32-10, uniforms, the screened Primakoff factor
// F(s), Poisson inversion, inverse-CDF table lookup, isotropic directions and
// the per-cell rate record. Everything per particle is binary32; the record
// is computed in binary32 from constants folded in binary64 on the host, so
// that no per-particle or common-path per-cell work touches the FP64 pipe
// (about 1/60 of the FP32 rate on GB300).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/axpic.h"
#include "tables.h"

namespace axpic {

// ---------------------------------------------------------------- constants
constexpr double kMeC2 = 510.99895000;     // keV
constexpr float kMeC2f = 510.99895000f;
constexpr float kInvMeC2f = (float)(1.0 / 510.99895000);
constexpr int kMaxSpecies = 8;
constexpr int kPoissonKmax = 255;
constexpr float kLambdaHardCap = 64.0f;

// Philox streams (counter word 3 = stream << 24 | sub).
enum : uint32_t {
  S_PRIM_FWD = 0,  // gamma->a decision of a photon
  S_EMIT_E = 1,    // thermal-bath emission decision of an electron (both channels)
  S_PRIM_INV = 3,  // a->gamma decision of an axion
  S_ABSORB = 4,    // absorption decision of an axion
  S_EV_E = 5,      // thermal-bath event: cos theta, phi, energy, channel
  S_INIT_E = 8, S_INIT_G = 9, S_INIT_A = 10
};
constexpr uint32_t kInitStep = 0xFFFFFFFFu;

// Inverse-CDF tables: ln x tabulated on a uniform grid of y = logit(u)
// (layout and construction in tables.h / tables.cpp).

// Per-cell binary32 rate record (16 floats = 64 B). The composition part
// depends only on the ion densities; the temperature part is recomputed
// whenever T_e changes.
constexpr int kRecLen = 16;
enum {
  R_T = 0,     // T_e, keV
  R_INVT,      // 1/T_e
  R_FOURK2,    // 4/kappa^2 (s = omega^2 * R_FOURK2)
  R_CC,        // Gamma_C dt / w_a (lambda_C = w_e * R_CC)
  R_CB,        // Gamma_B dt / w_a
  R_BC,        // Compton absorption prefactor (tau_C = R_BC x^2 [/(1-e^-x)])
  R_BB,        // bremsstrahlung absorption prefactor (tau_B = R_BB x^(a-3) [(1-e^-x)])
  R_AP,        // Gamma_0 dt of gamma->a (Gamma dt = R_AP * F(s))   [composition; the
               // surrogate network's, per temperature, where rate model 2 trusts it]
  R_APINV,     // m * R_AP (a->gamma; the step forms m * R_AP itself) [composition]
  R_NE,        // n_e / 1e24 cm^-3                                  [composition]
  R_NEFF,      // n_eff / 1e24 cm^-3                                [composition]
  R_RHO,       // rho, g cm^-3                                      [composition]
  R_XH,        // hydrogen mass fraction                            [composition]
  R_SZ         // Primakoff target sum / 1e24 cm^-3                 [composition]
};

// Cached electron moments per cell (binary32): W, Px, Py, Pz, U2, var, and
// the common electron weight when every electron of the cell has the same
// weight (0 otherwise). Electrons change only through the remap.
constexpr int kMomLen = 8;

// Cells per chunk of a decision warp; the default is a compile-time choice
// that launch-shape sweeps override (c2 replayed in 8 branches: 8 cells
// 0.178 ms per step, 4 cells 0.185, 2 cells 0.210).
#ifndef AXPIC_DEC_CHUNK
#define AXPIC_DEC_CHUNK 32
#endif
enum { M_W = 0, M_PX, M_PY, M_PZ, M_U2, M_VAR, M_WU };

// Per-CTA counters (u64), reduced by axpic_tally_spectrum.
enum {
  C_EV_P = 0, C_EV_C, C_EV_B, C_EV_PINV, C_ABS_C, C_ABS_B, C_CAP, C_CLAMP, C_DROP, C_REMAP,
  C_NE, C_NG, C_NA, C_REMAP_E, C_CELLS,
  kNumCounters
};

// Device error flag bits.
enum { ERR_CAPACITY = 1, ERR_NUMERIC = 2, ERR_TIMEOUT = 4 };

// Rows of per-CTA event counters (CTAs share rows beyond this).
constexpr int kCounterRows = 4096;

// Constants folded on the host (binary64) for the binary32 record.
struct CellConst {
  int nspecies;
  float Z[kMaxSpecies];
  float A[kMaxSpecies];
  int is_h[kMaxSpecies];
  int kappa_mode;
  float kappa_fixed;
  int prim_targets;
  float prim_mult;
  int brems_ee;
  float k_kappa2;   // 4 pi alpha (hbar c)^3 * 1e24  [keV^3 per (1e24 cm^-3)]
  float k_rho;      // m_u * 1e24  [g per (1e24 cm^-3)]
  float k_T7;       // 1 / (k_B 1e7 K)  [1/keV]
  float afac;       // g_ae^2 / (4 pi 1.6e-23)
  float k_AP;       // alpha (g hbar c)^2 c / 8 * 1e24 * dt
  float k_CC;       // dt / (w_a <x>_C keV_erg 1e24)
  float k_CB;       // dt / (w_a a keV_erg 1e24)
  float k_BC;       // 2 pi^2 (hbar c)^3 dt / (Gamma(5) zeta(5) <x>_C keV_erg)
  float k_BB;       // 2 pi^2 (hbar c)^3 dt / (Gamma(a) a keV_erg)
};

// Per-cell spectral records (rate models 1 and 2) and the surrogate network
// that replaces them where it is trusted (rate model 2).
//  * rate model 1: every cell's Primakoff and absorption rates (x = omega/T in
//    [0.05, 20]) and emission energies come from its 192-float spectral
//    record, interpolated from the exact FP32 table;
//  * rate model 2: where the network is trusted (src[cell] = 0) it wrote the
//    cell's rate prefactors into the cell record's slots R_CC..R_AP (the
//    closed functional forms times the network's per-cell emissivity
//    constants) and the emission energies come from the network's
//    cell-independent quantiles (uni); elsewhere (src[cell] = 1) the cell has
//    the table's spectral record, as in rate model 1.
struct RecordArgs {
  float* sr;                  // [ncells * 192] spectral records
  const float* tab;           // exact table [2][nne][nkt][189]
  int nkt, nne;
  float Z;                    // the single ion species' charge
  float ln_gP, ln_gA;         // ln(g_agg^2 dt pi^2 (hbar c)^3 / keV), ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / keV)
  float lnK_CC, lnK_CB;       // network emission rates: R_CC = exp(c_C + lnK_CC) / (n_e' T), likewise R_CB
  float bee_c;                // (1 + X_H) / (2 sqrt 2) of the e-e bremsstrahlung term (0 without it)
  float k_T7;                 // 1 / (k_B 1e7 K) [1/keV]
  const uint8_t* trust;       // [2][tnne][tnT] trust map, NULL: the network is used nowhere
  int tnT, tnne;
  const unsigned char* img;   // the network in its shared-memory image (kNetImgBytes)
  uint8_t* src;               // [ncells] rate model 2: 1 = table record, 0 = network prefactors
  const float* uni;           // [192]: the network's cell-independent quantiles at a record's offsets
};

// A species' slabs: wp[i] = {w, px, py, pz} and xyz[i] = {x, y, z, 0} of
// slot i.
struct SpeciesPtrs {
  float4* wp;
  float4* xyz;
  int32_t* count;
  int32_t cap;
};

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ((word >> 9) + 0.5) * 2^-23: exact in binary32, in (0, 1). Formed from the
// bits: 1 + m 2^-23 (exponent 0, mantissa m = word >> 9) minus (1 - 2^-24)
// is exact by Sterbenz's lemma, with no integer-to-float conversion.
__device__ __forceinline__ float u23(uint32_t w) {
  return __fsub_rn(__uint_as_float((w >> 9) | 0x3F800000u), __uint_as_float(0x3F7FFFFFu));
}

// Round keys of Philox4x32-10 for one key (k + r W mod 2^32, r = 0..9),
// formed on the host so that the rounds take them as constant operands.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r],
                   (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint32_t word(const uint4& b, int j) {
  return j == 0 ? b.x : (j == 1 ? b.y : (j == 2 ? b.z : b.w));
}

// ---------------------------------------------------------------- physics
// F(s) = (1 + 1/s) ln(1 + s) - 1; below s = 0.25 its power series
// sum_{n>=1} (-1)^(n+1) s^n / (n (n+1)) (12 terms) avoids the cancellation.
__device__ __forceinline__ float prim_F(float s) {
  if (s < 0.25f) {
    float acc = 0.0f;
#pragma unroll
    for (int n = 12; n >= 1; --n) {
      const float c = ((n & 1) ? 1.0f : -1.0f) / (float)(n * (n + 1));
      acc = fmaf(acc, s, c);
    }
    return acc * s;
  }
  return (1.0f + 1.0f / s) * log1pf(s) - 1.0f;
}

// K = min{k : u <= F_k}, p_k = p_{k-1} * (lambda / k), F_k = F_{k-1} + p_k,
// binary32 with no contraction, bounded by 255 iterations.
__device__ __forceinline__ int poisson_inv(float u, float lam) {
  float p = expf(-lam);
  float F = p;
  int k = 0;
  while (u > F && k < kPoissonKmax) {
    ++k;
    p = __fmul_rn(p, __fdiv_rn(lam, (float)k));
    F = __fadd_rn(F, p);
    if (p == 0.0f) break;
  }
  return k;
}

// Cap-and-rescale (Eqs. lambda_eff, wa_rescaled): returns lambda_eff and sets
// *fac = lambda_macro / lambda_eff (1 exactly when no cap applies).
__device__ __forceinline__ float cap_lambda(float lam, float cap, float* fac, bool* capped) {
  if (lam > cap) {
    *fac = lam / cap;
    *capped = true;
    return cap;
  }
  *fac = 1.0f;
  *capped = false;
  return lam;
}

// Weight depletion in binary32: returns the product weight and sets *wrem.
__device__ __forceinline__ float deplete(float w, int K, float wprod, float* wrem, bool* over) {
  const float conv = __fmul_rn((float)K, wprod);
  *over = (K > 0) && (conv > w);
  if (*over) {
    *wrem = 0.0f;
    return __fdiv_rn(w, (float)K);
  }
  *wrem = __fsub_rn(w, conv);
  return wprod;
}

// x = exp(g(logit u)), g linearly interpolated on kTableN nodes.
__device__ __forceinline__ float icdf_lookup(const float* __restrict__ tab, float u) {
  const float y = logf(u) - logf(1.0f - u);
  const float inv_h = (float)(kTableN - 1) / (kTableY1 - kTableY0);
  float t = (y - kTableY0) * inv_h;
  t = fminf(fmaxf(t, 0.0f), (float)(kTableN - 1) - 1e-3f);
  const int i = (int)t;
  const float f = t - (float)i;
  const float g0 = __ldg(tab + i);
  const float g1 = __ldg(tab + i + 1);
  return expf(fmaf(f, g1 - g0, g0));
}

// Isotropic unit vector: cos(theta) = 2u0 - 1, phi = 2 pi u1.
__device__ __forceinline__ float3 iso_dir(float u0, float u1) {
  const float ct = fmaf(2.0f, u0, -1.0f);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
  float sp, cp;
  sincospif(2.0f * u1, &sp, &cp);
  return make_float3(st * cp, st * sp, ct);
}

// Composition part of the record from the ion densities (Eqs. rho_def,
// qn_def, kappa_debye's n_eff, prim_rate's sum Z^2 n).
__device__ __forceinline__ void compute_composition(const CellConst& cc,
                                                    const double* __restrict__ n_ion, float* rec) {
  float rho_u = 0.f, ne = 0.f, zsq = 0.f, mh = 0.f;
  for (int s = 0; s < cc.nspecies; ++s) {
    const float n = (float)(n_ion[s] * 1e-24);
    rho_u += n * cc.A[s];
    ne += n * cc.Z[s];
    zsq += n * cc.Z[s] * cc.Z[s];
    if (cc.is_h[s]) mh += n * cc.A[s];
  }
  const float neff = ne + zsq;
  rec[R_NE] = ne;
  rec[R_NEFF] = neff;
  rec[R_RHO] = rho_u * cc.k_rho;
  rec[R_XH] = rho_u > 0.f ? mh / rho_u : 0.f;
  rec[R_SZ] = cc.prim_targets == 0 ? zsq : neff;
  rec[R_AP] = cc.k_AP * rec[R_SZ];
  rec[R_APINV] = cc.prim_mult * rec[R_AP];
}

struct CellExtras {
  float kappa, QC, QB, eta;
};

// Temperature part of the record (Eqs. kappa_debye, epsC, QC, GammaC,
// eps_eZ, eps_ee, gamma_abs), binary32 from the composition slots.
__device__ __forceinline__ CellExtras compute_temperature(const CellConst& cc, float T, float* rec) {
  const float invT = 1.0f / T;
  const float ne = rec[R_NE];
  const float rho = rec[R_RHO];
  const float XH = rec[R_XH];
  float kappa2;
  if (cc.kappa_mode == 0) kappa2 = cc.k_kappa2 * rec[R_NEFF] * invT;
  else kappa2 = cc.kappa_fixed * cc.kappa_fixed;
  const float T7 = T * cc.k_T7;
  const float rho2 = rho * 0.01f;
  const float T7sq = T7 * T7;
  const float eta = (3.0f + XH) * rho2 / T7sq;
  const float onepx = 1.0f + XH;
  const float eps_C = 2.67e-2f * onepx * (T7sq * T7sq * T7sq) * cc.afac;
  const float t25 = T7sq * sqrtf(T7);
  const float eps_eZ = 0.150f * t25 * rho2 * onepx * cc.afac * fmaxf(0.f, 1.0f - 6.98e-2f * eta);
  float eps_ee = 0.f;
  if (cc.brems_ee)
    eps_ee = 0.150f * t25 * rho2 * onepx * (onepx * 0.35355339059327373f) * cc.afac *
             fmaxf(0.f, 1.0f - 0.140f * eta);
  const float QC = rho * eps_C;
  const float QB = rho * (eps_eZ + eps_ee);
  rec[R_T] = T;
  rec[R_INVT] = invT;
  rec[R_FOURK2] = 4.0f / kappa2;
  rec[R_CC] = ne > 0.f ? QC * cc.k_CC / (ne * T) : 0.f;
  rec[R_CB] = ne > 0.f ? QB * cc.k_CB / (ne * T) : 0.f;
  const float invT2 = invT * invT;
  rec[R_BC] = QC * cc.k_BC * (invT2 * invT2);
  rec[R_BB] = QB * cc.k_BB * (invT2 * invT2);
  CellExtras ex;
  ex.kappa = sqrtf(kappa2);
  ex.QC = QC;
  ex.QB = QB;
  ex.eta = eta;
  return ex;
}

// Massive axions (Sec. II.B: E = sqrt(p^2 + m_a^2)): the axion phase-space
// factor p/E at energy e (m_e c^2 units) for mass mu (mu2 = mu mu, both
// binary32), p = sqrt(max(e^2 - mu^2, 0)): 0 at and below the threshold.
// It thins emission (the massive process is the massless one kept with
// probability beta) and carries gamma->a's product momentum.
__device__ __forceinline__ float axion_beta(float e, float mu2) {
  const float pm = sqrtf(fmaxf(__fsub_rn(__fmul_rn(e, e), mu2), 0.0f));
  return e > 0.0f ? __fdiv_rn(pm, e) : 0.0f;
}

// Primakoff conversion probability over one step (Eqs. prim_xs to
// prim_prob): P = 1 - exp(-A F(4 omega^2 / kappa^2)), A = R_AP or R_APINV.
__device__ __forceinline__ float prim_prob(const float* rec, float omega, float A) {
  const float s = omega * omega * rec[R_FOURK2];
  return -expm1f(-A * prim_F(s));
}

// Detailed-balance absorption optical depths over one step (Eq. gamma_abs):
// Compton-like tau_C = R_BC x^2 e^x/(e^x-1) (MB) or R_BC x^2 (BE);
// bremsstrahlung tau_B = R_BB x^(a-3) (MB) or R_BB x^(a-3) (1-e^-x) (BE).
__device__ __forceinline__ float tau_compton(const float* rec, float x, int eq_stats) {
  const float base = rec[R_BC] * x * x;
  return eq_stats ? base : base / (-expm1f(-x));
}

__device__ __forceinline__ float tau_brems(const float* rec, float x, float am3, int eq_stats) {
  const float base = rec[R_BB] * exp2f(am3 * log2f(x));
  return eq_stats ? base * (-expm1f(-x)) : base;
}

// Kernel parameters shared by the step kernels (passed by value).
struct StepArgs {
  SpeciesPtrs e, g, a;
  int ncells;             // cells of this launch: [cell0, cell0 + ncells)
  int cell0;              // first cell of this launch (a branch of a replayed step)
  uint32_t cell_base;     // global index of cell 0 (low 32 bits)
  uint32_t step;
  uint32_t key0, key1;
  PhiloxKeys rk;  // round keys of (key0, key1)
  int mask;
  float w_a, w_gref, inv_w_a, inv_w_gref;
  float lam_cap;          // effective cap, <= 64
  float brems_am3;        // a - 3
  int eq_stats, absorb_mode, T_mode, tally_enable, diag_enable, use_snapshot;
  float relax_r;
  double T_floor, T_ceil;
  float T_floor_f, T_ceil_f;  // binary32 copies for the common-path test
  float* rec;             // [ncells * kRecLen]
  float* mom;             // [ncells * kMomLen]
  double* T;              // [ncells]
  const double* n_ion;    // [ncells * nspecies]
  double* xbuf;           // [ncells * 4] exchange buffer (separate calls)
  double* res;            // [ncells * 4] carried energy / momentum
  double* diag;           // [ncells * AXPIC_CELL_DIAG_LEN]
  int32_t* photon_start;  // [ncells] photon count before absorb
  const float* tables;    // [kNumTables * kTableN]
  double* tally;          // [3 * nbins + 6]
  int nbins;
  float inv_dE_bin;
  unsigned long long* counters;  // [ctr_rows * kNumCounters]
  int ctr_rows;                  // CTA b adds to row b % ctr_rows
  uint32_t *bitsA, *bitsG, *bitsE;  // per-cell "needs a full decision" bit masks
  int Wa, Wg, We;                   // words per cell of each mask
  uint4 *recA, *recG;               // full decisions of flagged slots (slot-indexed)
  uint32_t* recE;
  int* err;
  int dec_grid;   // CTAs of the persistent decision kernel
  int dec_chunk;  // cells per chunk of a decision warp: 4, 8, 16 or 32
  uint32_t* step_dev;  // NULL, or the device step counter of a replayed graph
  // cells a full step's event kernel leaves to the warp-path kernel, stored
  // from index cell0 on, and their count (one counter per branch of a
  // replayed step)
  int32_t* heavy;
  int32_t* heavy_n;
  // rate model: 0 the closed forms; 1 the exact table's spectral records for
  // the full decisions' rates and the emission energies; 2 the surrogate
  // network where it is trusted, the table's records elsewhere
  int rate_model;
  RecordArgs ra;
  // axion mass m_a / m_e c^2 and its square (binary32); 0: massless, and every
  // mass factor is skipped
  float mu, mu2;
  float guard_margin;  // factor on the no-event bounds (covers the records' error)
  CellConst cc;
};

}  // namespace axpic
