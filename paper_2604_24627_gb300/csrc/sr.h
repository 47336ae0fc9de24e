// Per-cell spectral records of the table rate model and the surrogate
// network of rate model 2 (internal to libaxpic).
//
// Spectral record of one cell (kSrLen floats):
//   [0, 96)    ln(dQ_c/dx) + x_k (the Boltzmann factor taken out) at
//              x_k = 0.05 e^((k - 1) h), h = ln(400) / 29,
//              k = 0..31 (x_1 = 0.05, x_30 = 20: one point beyond each end),
//              unit coupling, c = 0 Primakoff, 1 Compton-like, 2 brems (c * 32 + k)
//   [96, 189)  number-spectrum quantiles x(j/32), j = 1..31 (96 + c * 31 + j - 1)
//   [189]      ln(g_agg^2 dt pi^2 (hbar c)^3 / (T^4 keV)): Gamma_P dt = exp(L_P + this) (e^x - 1) / x^3
//   [190]      ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / (T^4 keV)): tau_c = exp(L_c + this) e^x / x^3 (MB)
//   [191]      T [keV] the record was built for
//
// The exact table holds these values at nodes uniform in ln(kappa/T) and
// log10 n_e (Z = 1, 2), with the bremsstrahlung row's fit brackets
// [1 - c eta] (floored at 1e-3) divided out: a cell's record adds them back
// for its own eta, so the interpolation never crosses the brackets' floor
// (where ln Q_B has a kink).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace axpic {

constexpr int kSrLen = 192;
constexpr int kSrGrid = 32;
constexpr int kSrKnots = 31;
constexpr int SR_LNKP = 189, SR_LNKA = 190, SR_T = 191;
constexpr float kSrLnXLo = -2.99573227355399099f;  // ln 0.05
constexpr float kSrH = 0.20660222576234421f;        // ln(400) / 29: grid step in ln x
constexpr float kSrLnX0 = kSrLnXLo - kSrH;          // ln x_0
constexpr float kSrLnKt0 = -4.42284862919413700f;   // ln 0.012 (kappa/T)
constexpr float kSrLnKtSpan = 8.13642069589844400f;  // ln(41 / 0.012)
constexpr int kSrTabOut = 189;                      // table outputs per node
constexpr float kSrTLo = 0.5f, kSrTHi = 10.0f;      // the validated temperature range
constexpr float kSrLnTSpan = 2.99573227355399099f;  // ln(10 / 0.5)
constexpr int kNetImgBytes = 11584;                 // the network's image (srnet.cuh)

// Record-kernel inputs.
struct SrArgs {
  int ncells;        // cells of this launch: [cell0, cell0 + ncells)
  int cell0;         // first cell of the launch
  float* rec;        // [ncells * kRecLen] cell records
  RecordArgs ra;
  int* err;
};

// ---------------------------------------------------------------- per-cell pieces
// Cell quantities the records and the network need.
struct SrCellIn {
  float T, kT;
  float lkT, lne;  // ln(kappa/T), log10 n_e
  float eta;       // the bremsstrahlung fit's degeneracy parameter (3 + X_H) rho_2 / T_7^2
};
__device__ __forceinline__ SrCellIn sr_cell_from(const float* rec, float k_T7) {
  SrCellIn c;
  c.T = rec[R_T];
  c.kT = 2.0f * rsqrtf(rec[R_FOURK2]) / c.T;
  c.lkT = __logf(c.kT);
  c.lne = log10f(rec[R_NE] * 1e24f);
  const float T7 = c.T * k_T7;
  c.eta = (3.0f + rec[R_XH]) * (rec[R_RHO] * 0.01f) / (T7 * T7);
  return c;
}

// ln of the bremsstrahlung fit's brackets, (b_eZ + c_ee b_ee) / (1 + c_ee)
// with b = max(1e-3, 1 - k eta) (Eqs. eps_eZ, eps_ee; c_ee = (1 + X_H) /
// (2 sqrt 2), the e-e term's weight): the factor the table divides out.
__device__ __forceinline__ float sr_ln_brackets(float eta, float cee) {
  const float bz = fmaxf(1e-3f, 1.0f - 6.98e-2f * eta);
  const float be = fmaxf(1e-3f, 1.0f - 0.140f * eta);
  return __logf(__fdividef(fmaf(cee, be, bz), 1.0f + cee));
}

// A cell's table interpolation constants: the corner node (i, j) at the
// cell's Z, the weights in (ln kappa/T, log10 n_e), and the record's
// per-cell constants.
struct SrInterp {
  const float* t00;
  float fu, fv, lnKP, lnKA, T, lnbr;
};

// The record's per-cell constants (entries 189, 190).
__device__ __forceinline__ void sr_consts(const RecordArgs& a, float T, float* lnKP, float* lnKA) {
  *lnKP = fmaf(-4.0f, __logf(T), a.ln_gP);
  *lnKA = fmaf(-4.0f, __logf(T), a.ln_gA);
}

__device__ __forceinline__ void sr_interp(const RecordArgs& a, const SrCellIn& c, SrInterp* q) {
  float u = (c.lkT - kSrLnKt0) / kSrLnKtSpan * (a.nkt - 1);
  float v = (c.lne - 23.0f) / 3.0f * (a.nne - 1);
  u = fminf(fmaxf(u, 0.f), (float)(a.nkt - 1));
  v = fminf(fmaxf(v, 0.f), (float)(a.nne - 1));
  const int i = min((int)u, a.nkt - 2), j = min((int)v, a.nne - 2);
  const int z = a.Z > 1.5f ? 1 : 0;
  q->t00 = a.tab + ((size_t)(z * a.nne + j) * a.nkt + i) * kSrTabOut;
  q->fu = u - i;
  q->fv = v - j;
  sr_consts(a, c.T, &q->lnKP, &q->lnKA);
  q->T = c.T;
  q->lnbr = sr_ln_brackets(c.eta, a.bee_c);
}

// Entry o of the table record (bilinear, each rounding step explicit so that
// every kernel that writes records gives the same bits); the bremsstrahlung
// rate row gets the cell's brackets back.
__device__ __forceinline__ float sr_table_entry(const RecordArgs& a, const SrInterp& q, int o) {
  if (o >= kSrTabOut) return o == SR_LNKP ? q.lnKP : (o == SR_LNKA ? q.lnKA : q.T);
  const float* t01 = q.t00 + (size_t)a.nkt * kSrTabOut;  // j + 1
  const float v00 = q.t00[o], v10 = q.t00[kSrTabOut + o], v01 = t01[o], v11 = t01[kSrTabOut + o];
  const float u0 = fmaf(q.fu, v10, __fmul_rn(1.f - q.fu, v00));
  const float u1 = fmaf(q.fu, v11, __fmul_rn(1.f - q.fu, v01));
  const float v = fmaf(q.fv, u1, __fmul_rn(1.f - q.fv, u0));
  return (o >= 64 && o < 96) ? __fadd_rn(v, q.lnbr) : v;
}

// Whether the network is trusted at (T, n_e, Z): the four validation nodes
// around it (log-spaced in T and n_e) all passed (inside the validated grid
// only).
__device__ __forceinline__ bool sr_trusted(const RecordArgs& a, float T, float lne) {
  float fu = __logf(T * (1.0f / kSrTLo)) * (1.0f / kSrLnTSpan) * (a.tnT - 1);
  float fv = (lne - 23.0f) / 3.0f * (a.tnne - 1);
  // inside the validated grid (binary32 rounding at its edges tolerated)
  const float tol = 1e-4f;
  if (!(fu >= -tol && fu <= (float)(a.tnT - 1) + tol && fv >= -tol && fv <= (float)(a.tnne - 1) + tol)) return false;
  fu = fminf(fmaxf(fu, 0.f), (float)(a.tnT - 1));
  fv = fminf(fmaxf(fv, 0.f), (float)(a.tnne - 1));
  const int i = min((int)fu, a.tnT - 2), j = min((int)fv, a.tnne - 2);
  const int z = a.Z > 1.5f ? 1 : 0;
  const uint8_t* t = a.trust + (size_t)(z * a.tnne + j) * a.tnT + i;
  return t[0] && t[1] && t[a.tnT] && t[a.tnT + 1];
}

// A warp writes one cell's whole table record (lane l: entries l + 32 k).
__device__ __forceinline__ void sr_table_record_warp(const RecordArgs& a, const SrCellIn& c, float* out, int lane) {
  SrInterp q;
  sr_interp(a, c, &q);
#pragma unroll
  for (int k = 0; k < kSrLen / 32; ++k) out[lane + 32 * k] = sr_table_entry(a, q, lane + 32 * k);
}

// ---------------------------------------------------------------- host side
// The exact table, nkt x nne x 2 nodes (ln(kappa/T) uniform on
// [ln 0.012, ln 41], log10 n_e uniform on [23, 26], Z = 1, 2), binary64
// targets stored as binary32 (the bremsstrahlung rate row without its
// brackets).
void build_sr_table(int nkt, int nne, double brems_shape, float* out);

// Rate model 1: every cell's table record.
cudaError_t launch_sr_table(const SrArgs& a, cudaStream_t st);
// Rate model 2: per cell of [cell0, cell0 + ncells), from its current cell
// record: the network's prefactors into the record's rate slots where it is
// trusted, the table's spectral record elsewhere (src set accordingly). The
// record's closed-form slots must be current (launch_records) before it runs.
cudaError_t launch_sr_cells(const SrArgs& a, cudaStream_t st);
// The records of rate model `model` (1 or 2) for cells [cell0, cell0 + ncells).
cudaError_t launch_sr_records(int model, const SrArgs& a, cudaStream_t st);
cudaError_t sr_init_kernels();
// Lays out the network (FP32 parameters P and the output model's mu, sigma
// and S, all device) as the image of srnet.cuh in img (device, kNetImgBytes).
cudaError_t launch_net_image(const float* P, const float* mu, const float* sigma, const float* skip, void* img,
                             cudaStream_t st);

}  // namespace axpic
