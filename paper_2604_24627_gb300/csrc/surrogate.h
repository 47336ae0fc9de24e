// The spectral surrogate's target function on the host (internal to libaxpic).
#pragma once
#include <cstdint>
#include <vector>

namespace axpic {

constexpr double kSurXLo = 0.05, kSurXHi = 20.0;     // x = omega / T
constexpr double kSurKtLo = 0.012, kSurKtHi = 41.0;  // kappa / T
constexpr double kSurTLo = 0.5, kSurTHi = 10.0;      // keV
constexpr double kSurNeLo = 1e23, kSurNeHi = 1e26;   // cm^-3
constexpr int kSurOut = 96;

struct SurCell {
  double T, ne, Z, a, kappa, Q_C, Q_B, Gamma0_P;
  double bZ, bE;  // the bremsstrahlung fit's [1 - c eta] brackets before the 1e-3 floor
};

double sur_temperature(double kT, double ne, double Z);
double sur_kappa_over_T(double T, double ne, double Z);
SurCell sur_cell(double T, double ne, double Z, double brems_shape);
// dQ_c/dx at unit coupling (c: 0 Primakoff, 1 Compton-like, 2 bremsstrahlung)
double sur_emissivity(int ch, double x, const SurCell& c);
// quantiles x(u_j), j = 1..31, of channel c's number spectrum on [0.05, 20]
void sur_quantiles(int ch, const SurCell& c, double* out31);
// all 93 quantiles of a cell; universal (from sur_universal_knots, or NULL)
// supplies the cell-independent Compton-like and bremsstrahlung ones
void sur_knots(const SurCell& c, double* knots93, const double* universal = nullptr);
void sur_universal_knots(double brems_shape, double* knots93);
void sur_targets(double x, const SurCell& c, const double* knots93, double* out96);
void sur_features(double x, double kT, double ne, double Z, float* f4);
// x and kappa/T back from the features (inverse of the maps of sur_features)
void sur_feature_xkt(const float* f4, double* x, double* kT);
// The fixed part of output o of the network's model: for the ln-emissivity
// outputs (o = 0, 32, 64) the channel's exact x-dependence at fixed cell,
// zero for the quantiles:
//   Primakoff      3 ln x - ln(e^x - 1) + ln F(s), s = 4 x^2 / (kappa/T)^2
//   Compton-like   5 ln x - ln(e^x - 1)
//   bremsstrahlung a ln x - x
// with F the screening function of Sec. II.F. What is left of each
// ln-emissivity is a function of the cell alone.
double sur_shape(int o, double x, double kT, double a);
// Whether output o of the model does not depend on the cell: the
// Compton-like and bremsstrahlung quantiles (o = 33..63, 65..95).
inline bool sur_universal_output(int o) { return o > 32 && o % 32 != 0; }
// ncells random cells of the domain (T uniform, n_e log-uniform, Z in {1, 2};
// only where both bremsstrahlung brackets are at least kSurBracketMin) with
// xpc log-uniform x each: features X (rows x 4) and targets Y (rows x 96)
constexpr double kSurBracketMin = 0.05;
void sur_training_set(int ncells, int xpc, uint64_t seed, double brems_shape, std::vector<float>& X,
                      std::vector<double>& Y);

}  // namespace axpic
