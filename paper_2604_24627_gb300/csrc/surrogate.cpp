// The function the spectral surrogate stands in for, in binary64 on the host,
// and the training-data generator built on it.
//
// For a single-ion plasma of charge Z (n_i = n_e / Z, hydrogen or helium-4
// masses), Debye screening, ions as Primakoff targets and unit couplings
// (g_agg = 1 GeV^-1, g_ae = 1), at x = omega / T, per channel c in
// (Primakoff, Compton-like, bremsstrahlung):
//   slot 0: ln(dQ_c/dx) [erg cm^-3 s^-1 per unit x]:
//     Compton-like  Q_C x^5 / (e^x - 1) / (Gamma(6) zeta(6))        (Sec. II.G)
//     brems         Q_B x^a e^-x / Gamma(a + 1), [1 - c eta] >= 1e-3  (Sec. II.H)
//     Primakoff     E Gamma(E) n_gamma(E) T                          (Sec. II.F)
//   slots 1..31: quantiles x(u_j), u_j = j / 32, of the number spectrum
//     dQ_c/dx / x on [0.05, 20].
// The cell's (T, n_e, Z) follows from (kappa/T, n_e, Z) through the Debye
// screening length: T^3 = 4 pi alpha (hbar c)^3 n_e (1 + Z) / (kappa/T)^2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include "surrogate.h"
#include "tables.h"

namespace axpic {

namespace {
constexpr double kHc = 1.973269804e-8;       // hbar c [keV cm]
constexpr double kHcGeV = 1.973269804e-14;   // hbar c [GeV cm]
constexpr double kAl = 1.0 / 137.035999084;  // fine-structure constant
constexpr double kAmu = 1.66053906660e-24;   // atomic mass unit [g]
constexpr double kCl = 2.99792458e10;        // c [cm/s]
constexpr double kBoltz = 8.617333262e-8;    // k_B [keV/K]
constexpr double kErg = 1.602176634e-9;      // erg per keV
constexpr double kPI = 3.14159265358979323846;
}  // namespace

double sur_temperature(double kT, double ne, double Z) {
  return std::cbrt(4.0 * kPI * kAl * kHc * kHc * kHc * ne * (1.0 + Z) / (kT * kT));
}

double sur_kappa_over_T(double T, double ne, double Z) {
  return std::sqrt(4.0 * kPI * kAl * kHc * kHc * kHc * ne * (1.0 + Z) / (T * T * T));
}

SurCell sur_cell(double T, double ne, double Z, double brems_shape) {
  SurCell c;
  c.T = T;
  c.ne = ne;
  c.Z = Z;
  c.a = brems_shape;
  const double A = Z == 1.0 ? 1.00794 : 4.002602;
  const double ni = ne / Z;
  const double rho = ni * A * kAmu;
  const double XH = Z == 1.0 ? 1.0 : 0.0;
  const double zsq = Z * Z * ni;
  c.kappa = std::sqrt(4.0 * kPI * kAl * (ne + zsq) * kHc * kHc * kHc / T);
  const double T7 = T / (kBoltz * 1e7);
  const double rho2 = rho / 100.0;
  const double eta = (3.0 + XH) * rho2 / (T7 * T7);
  const double afac = (1.0 / (4.0 * kPI)) / 1.60e-23;
  const double epsC = 2.67e-2 * (1.0 + XH) * std::pow(T7, 6.0) * afac;
  c.bZ = 1.0 - 6.98e-2 * eta;
  c.bE = 1.0 - 0.140 * eta;
  const double epsZ = 0.150 * std::pow(T7, 2.5) * rho2 * (1.0 + XH) * afac * std::max(1e-3, c.bZ);
  const double epsE = 0.150 * std::pow(T7, 2.5) * rho2 * (1.0 + XH) * (1.0 + XH) / (2.0 * std::sqrt(2.0)) * afac *
                      std::max(1e-3, c.bE);
  c.Q_C = rho * epsC;
  c.Q_B = rho * (epsZ + epsE);
  c.Gamma0_P = kAl * kHcGeV * kHcGeV / 8.0 * zsq * kCl;
  return c;
}

// F(s) = (1 + 1/s) ln(1 + s) - 1; its series below s = 1e-3.
static double prim_F(double s) {
  if (s < 1e-3) {
    double acc = 0.0, p = s;
    for (int n = 1; n <= 8; ++n, p *= s) acc += ((n & 1) ? 1.0 : -1.0) * p / (n * (n + 1.0));
    return acc;
  }
  return (1.0 + 1.0 / s) * std::log1p(s) - 1.0;
}

double sur_emissivity(int ch, double x, const SurCell& c) {
  if (ch == 1) return c.Q_C * std::pow(x, 5.0) / std::expm1(x) / (120.0 * zeta(6.0));
  if (ch == 2) return c.Q_B * std::exp(c.a * std::log(x) - x - std::lgamma(c.a + 1.0));
  const double E = x * c.T;
  const double n_gamma = E * E / (kPI * kPI * kHc * kHc * kHc) / std::expm1(x);
  const double rate = c.Gamma0_P * prim_F(4.0 * E * E / (c.kappa * c.kappa));
  return E * rate * n_gamma * c.T * kErg;
}

template <class Cdf>
static void truncated_quantiles(Cdf cdf, double* out) {
  const double lo = cdf(kSurXLo), hi = cdf(kSurXHi);
  for (int j = 1; j <= 31; ++j) {
    const double target = lo + (j / 32.0) * (hi - lo);
    double a = std::log(kSurXLo), b = std::log(kSurXHi);
    for (int it = 0; it < 64; ++it) {
      const double m = 0.5 * (a + b);
      if (cdf(std::exp(m)) < target) a = m;
      else b = m;
    }
    out[j - 1] = std::exp(0.5 * (a + b));
  }
}

void sur_quantiles(int ch, const SurCell& c, double* out) {
  if (ch == 1) {
    truncated_quantiles([](double x) {
      double p, q;
      bose_cdf(4, x, &p, &q);
      return p;
    }, out);
    return;
  }
  if (ch == 2) {
    const double a = c.a;
    truncated_quantiles([a](double x) {
      double p, q;
      gamma_pq(a, x, &p, &q);
      return p;
    }, out);
    return;
  }
  // Primakoff: cumulative trapezoid of the number spectrum in ln x, inverted
  const int n = 8001;
  const double t0 = std::log(kSurXLo), t1 = std::log(kSurXHi), h = (t1 - t0) / (n - 1);
  std::vector<double> cum(n, 0.0);
  double prev = sur_emissivity(0, kSurXLo, c);  // d(number)/d(ln x) = dQ/dx
  for (int i = 1; i < n; ++i) {
    const double f = sur_emissivity(0, std::exp(t0 + i * h), c);
    cum[i] = cum[i - 1] + 0.5 * (prev + f) * h;
    prev = f;
  }
  int k = 0;
  for (int j = 1; j <= 31; ++j) {
    const double target = (j / 32.0) * cum[n - 1];
    while (k + 1 < n - 1 && cum[k + 1] < target) ++k;
    const double w = (target - cum[k]) / (cum[k + 1] - cum[k]);
    out[j - 1] = std::exp(t0 + (k + w) * h);
  }
}

void sur_targets(double x, const SurCell& c, const double* knots93, double* out96) {
  for (int ch = 0; ch < 3; ++ch) {
    out96[32 * ch] = std::log(sur_emissivity(ch, x, c));
    for (int j = 0; j < 31; ++j) out96[32 * ch + 1 + j] = knots93[31 * ch + j];
  }
}

void sur_knots(const SurCell& c, double* knots93, const double* universal) {
  sur_quantiles(0, c, knots93);
  if (universal) {
    for (int q = 31; q < 93; ++q) knots93[q] = universal[q];
    return;
  }
  for (int ch = 1; ch < 3; ++ch) sur_quantiles(ch, c, knots93 + 31 * ch);
}

void sur_universal_knots(double brems_shape, double* knots93) {
  // the Compton-like and bremsstrahlung number spectra in x do not depend on
  // the cell: any cell gives their quantiles
  sur_knots(sur_cell(1.0, 1e24, 1.0, brems_shape), knots93, nullptr);
}

void sur_features(double x, double kT, double ne, double Z, float* f) {
  f[0] = (float)(std::log(x / kSurXLo) / std::log(kSurXHi / kSurXLo) * 2.0 - 1.0);
  f[1] = (float)(std::log(kT / kSurKtLo) / std::log(kSurKtHi / kSurKtLo) * 2.0 - 1.0);
  f[2] = (float)((std::log10(ne) - 24.5) / 1.5);
  f[3] = (float)(Z - 1.5);
}

void sur_feature_xkt(const float* f, double* x, double* kT) {
  *x = kSurXLo * std::pow(kSurXHi / kSurXLo, 0.5 * ((double)f[0] + 1.0));
  *kT = kSurKtLo * std::pow(kSurKtHi / kSurKtLo, 0.5 * ((double)f[1] + 1.0));
}

double sur_shape(int o, double x, double kT, double a) {
  if (o == 0) return 3.0 * std::log(x) - std::log(std::expm1(x)) + std::log(prim_F(4.0 * x * x / (kT * kT)));
  if (o == 32) return 5.0 * std::log(x) - std::log(std::expm1(x));
  if (o == 64) return a * std::log(x) - x;
  return 0.0;
}

// splitmix64: a seeded stream for the training-set draws
static uint64_t mix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double unif(uint64_t& s) { return ((mix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

void sur_training_set(int ncells, int xpc, uint64_t seed, double brems_shape, std::vector<float>& X,
                      std::vector<double>& Y) {
  struct Draw {
    double T, ne, Z;
    std::vector<double> x;
  };
  std::vector<Draw> cells(ncells);
  uint64_t s = seed;
  for (auto& d : cells) {
    // the network is trained where the bremsstrahlung fit holds (both of its
    // brackets well above their floor); cells beyond fail validation there
    // and keep the table
    do {
      d.T = kSurTLo + (kSurTHi - kSurTLo) * unif(s);
      d.ne = std::pow(10.0, 23.0 + 3.0 * unif(s));
      d.Z = (mix(s) & 1) ? 2.0 : 1.0;
      const SurCell c = sur_cell(d.T, d.ne, d.Z, brems_shape);
      if (std::min(c.bZ, c.bE) >= kSurBracketMin) break;
    } while (true);
    d.x.resize(xpc);
    for (int k = 0; k < xpc; ++k) d.x[k] = kSurXLo * std::pow(kSurXHi / kSurXLo, unif(s));
  }
  X.assign((size_t)ncells * xpc * 4, 0.f);
  Y.assign((size_t)ncells * xpc * 96, 0.0);
  double uni[93];
  sur_universal_knots(brems_shape, uni);
  const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) {
    th.emplace_back([&, t]() {
      double knots[93];
      for (int i = t; i < ncells; i += nth) {
        const Draw& d = cells[i];
        const SurCell c = sur_cell(d.T, d.ne, d.Z, brems_shape);
        sur_knots(c, knots, uni);
        const double kT = c.kappa / d.T;
        for (int k = 0; k < xpc; ++k) {
          const size_t r = (size_t)i * xpc + k;
          sur_features(d.x[k], kT, d.ne, d.Z, &X[r * 4]);
          sur_targets(d.x[k], c, knots, &Y[r * 96]);
        }
      }
    });
  }
  for (auto& x : th) x.join();
}

}  // namespace axpic

// ---------------------------------------------------------------- C ABI
#include "axpic.h"

extern "C" {

axpic_status axpic_surrogate_targets(const double* in, int32_t n, double brems_shape, double* out) {
  if (n < 0 || (n > 0 && (!in || !out)) || !(brems_shape > 0)) return AXPIC_E_INVALID;
  double knots[93], uni[93];
  if (n > 0) axpic::sur_universal_knots(brems_shape, uni);
  for (int32_t r = 0; r < n; ++r) {
    const double x = in[4 * r], kT = in[4 * r + 1], ne = in[4 * r + 2], Z = in[4 * r + 3];
    if (!(x > 0) || !(kT > 0) || !(ne > 0) || (Z != 1.0 && Z != 2.0)) return AXPIC_E_INVALID;
    const axpic::SurCell c = axpic::sur_cell(axpic::sur_temperature(kT, ne, Z), ne, Z, brems_shape);
    axpic::sur_knots(c, knots, uni);
    axpic::sur_targets(x, c, knots, out + 96 * (size_t)r);
  }
  return AXPIC_OK;
}

axpic_status axpic_surrogate_features(const double* in, int32_t n, float* out) {
  if (n < 0 || (n > 0 && (!in || !out))) return AXPIC_E_INVALID;
  for (int32_t r = 0; r < n; ++r) axpic::sur_features(in[4 * r], in[4 * r + 1], in[4 * r + 2], in[4 * r + 3], out + 4 * r);
  return AXPIC_OK;
}

}  // extern "C"
