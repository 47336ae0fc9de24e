// Per-cell spectral records of the table and surrogate rate models (internal
// to libaxpic).
//
// Record of one cell (kSrLen floats):
//   [0, 96)    ln(dQ_c/dx) + x_k (the Boltzmann factor taken out) at
//              x_k = 0.05 e^((k - 1) h), h = ln(400) / 29,
//              k = 0..31 (x_1 = 0.05, x_30 = 20: one point beyond each end),
//              unit coupling, c = 0 Primakoff, 1 Compton-like, 2 brems (c * 32 + k)
//   [96, 189)  number-spectrum quantiles x(j/32), j = 1..31 (96 + c * 31 + j - 1)
//   [189]      ln(g_agg^2 dt pi^2 (hbar c)^3 / (T^4 keV)): Gamma_P dt = exp(L_P + this) (e^x - 1) / x^3
//   [190]      ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / (T^4 keV)): tau_c = exp(L_c + this) e^x / x^3 (MB)
//   [191]      T [keV] the record was built for
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

// Rate-model inputs of the record kernels.
struct SrArgs {
  int ncells;            // cells of this launch: [cell0, cell0 + ncells)
  int cell0;             // first cell (a branch of a replayed step: a multiple of 128)
  const float* rec;      // [ncells * kRecLen]
  float* sr;             // [ncells * kSrLen]
  const float* tab;      // [2][nne][nkt][kSrTabOut]
  int nkt, nne;
  float Z;               // the single ion species' charge
  float ln_gP, ln_gA;    // ln(g_agg^2 dt pi^2 (hbar c)^3 / keV), ln(g_ae^2 dt 2 pi^2 (hbar c)^3 / keV)
  // surrogate network (FP32 master parameters, output affine, trust map)
  const float* P;
  const float* mu;
  const float* sigma;
  const float* skip;     // S[96][4]: y = shape(x, kappa/T) + mu + S f + sigma z
  float brems_a;         // the bremsstrahlung shape's exponent a
  const uint8_t* trust;  // [2][tnne][tnT], 1 = trusted node
  const void* W16;       // W2^T, W3^T in bfloat16, core-matrix layout (launch_sr_weights)
  int tnT, tnne;
  uint8_t* net;          // [ncells]: 1 = the network kernel wrote this cell's record (surrogate model)
  int* err;
};

// Host: the exact table, nkt x nne x 2 nodes (ln(kappa/T) uniform on
// [ln 0.012, ln 41], log10 n_e uniform on [23, 26], Z = 1, 2), binary64
// targets stored as binary32.
void build_sr_table(int nkt, int nne, double brems_shape, float* out);

cudaError_t launch_sr_table(const SrArgs& a, cudaStream_t st);
cudaError_t launch_sr_mlp(const SrArgs& a, cudaStream_t st);
// The records of cells [cell0, cell0 + ncells) for their current T: the
// network kernel over the cells where it is trusted (when a trust map is
// set), then the table kernel over the others.
cudaError_t launch_sr_records(const SrArgs& a, cudaStream_t st);
// Lays out layers 2 and 3 of the parameters P (FP32, device) for sr_mlp:
// out holds (64 * 64 + 96 * 64) bfloat16 values (20 KB, 16-byte aligned).
cudaError_t launch_sr_weights(const float* P, void* out, cudaStream_t st);
constexpr size_t kSrW16Bytes = (64 * 64 + 96 * 64) * 2;
cudaError_t sr_init_kernels();

}  // namespace axpic
