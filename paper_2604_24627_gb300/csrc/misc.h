// Launch interface of the auxiliary kernels (internal to libaxpic).
#pragma once
#include "common.cuh"

namespace axpic {

struct SampleArgs {
  SpeciesPtrs e, g, a;
  int ncells, n_el, n_ph, n_ax;
  uint32_t cell_base, key0, key1;
  float k_we;   // V * 1e24 / n_el: w_e = n_e[1e24 cm^-3] * k_we
  float k_wg;   // 2 zeta(3) / (pi^2 (hbar c)^3) * V / n_ph: w_gamma = T^3 * k_wg
  float w_a;
  const float* rec;
  const float* tables;
};

// n_i = (sum of the cell's electron weights) * coef[i], coef[i] including 1/V
struct DepositCoef {
  double coef[kMaxSpecies];
};

cudaError_t launch_deposit(int ncells, int nspecies, const SpeciesPtrs& e, const DepositCoef& k, double* n_ion,
                           cudaStream_t st);
cudaError_t launch_records(int ncells, int nspecies, const CellConst& cc, const double* T, const double* n_ion,
                           float* rec, int* err, cudaStream_t st);
cudaError_t launch_info(int first, int count, const CellConst& cc, double k_gamma, const float* rec, double* out,
                        cudaStream_t st);
cudaError_t launch_moments(int ncells, const SpeciesPtrs& e, float* mom, cudaStream_t st);
cudaError_t launch_sample(const SampleArgs& S, cudaStream_t st);
cudaError_t launch_rates(const float* rec, int cell, const float* E, int n, int eq_stats, float am3, float prim_mult,
                         float mu2, float* out,
                         cudaStream_t st);
cudaError_t launch_totals(int ncells, const SpeciesPtrs& e, const SpeciesPtrs& g, const SpeciesPtrs& a,
                          const double* res, const unsigned long long* ctr, int ctr_rows, double* out8,
                          double* out_ctr, cudaStream_t st);

}  // namespace axpic
