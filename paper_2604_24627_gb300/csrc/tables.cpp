// Inverse-CDF tables of the energy-sampling kernels, built on the host in
// binary64 and stored as binary32 ln x on a uniform grid of y = logit(u):
//   Compton-like: number pdf x^4/(e^x-1) (power spectrum E^5/(e^{E/T}-1),
//                 Sec. II.G, Eq. compton_kernel)
//   bremsstrahlung: Gamma(a), pdf x^(a-1) e^-x / Gamma(a) (Sec. II.H)
//   Planck photons: x^2/(e^x-1) (blackbody bath at T_e, Sec. II.G)
//   MB-equilibrium axions: Gamma(3) (Sec. II.I, MB target)
// The CDFs come from their series definitions: for the Bose-type integrals
// I_n(x) = int_0^x t^n/(e^t-1) dt a Bernoulli series below x = 1 and
// n! sum_k k^-(n+1) Q(n+1, kx) above; for Gamma(a) the lower series of the
// regularized incomplete gamma below x = a+1 and Legendre's continued
// fraction for the upper function above. Each node is inverted by bisection.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <map>
#include <vector>

#include "tables.h"

namespace axpic {

double zeta(double s) {
  const int N = 64;
  double sum = 0.0;
  for (int k = 1; k < N; ++k) sum += std::pow((double)k, -s);
  const double n = N;
  // Euler-Maclaurin remainder of sum_{k>=N} k^-s
  sum += std::pow(n, 1.0 - s) / (s - 1.0) + 0.5 * std::pow(n, -s) + s * std::pow(n, -s - 1.0) / 12.0 -
         s * (s + 1.0) * (s + 2.0) * std::pow(n, -s - 3.0) / 720.0;
  return sum;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Bernoulli numbers B_0..B_20 (B_1 = -1/2); odd ones above 1 vanish.
static const double kBern[21] = {1.0, -0.5, 1.0 / 6, 0, -1.0 / 30, 0, 1.0 / 42, 0, -1.0 / 30, 0, 5.0 / 66, 0,
                                 -691.0 / 2730, 0, 7.0 / 6, 0, -3617.0 / 510, 0, 43867.0 / 798, 0,
                                 -174611.0 / 330};

// CDF and complementary CDF of the number pdf x^n/(e^x-1)/(n! zeta(n+1)).
void bose_cdf(int n, double x, double* cdf, double* ccdf) {
  const double total = factorial(n) * zeta(n + 1.0);
  if (x < 1.0) {
    double acc = 0.0, fm = 1.0;
    for (int m = 0; m <= 20; ++m) {
      if (m > 0) fm *= m;
      if (kBern[m] == 0.0) continue;
      acc += kBern[m] / fm * std::pow(x, n + m) / (n + m);
    }
    *cdf = acc / total;
    *ccdf = 1.0 - *cdf;
    return;
  }
  double tail = 0.0;
  const int kmax = (int)std::ceil(80.0 / x) + 1;
  for (int k = 1; k <= kmax; ++k) {
    const double y = k * x;
    double q = 0.0, term = 1.0;
    for (int j = 0; j <= n; ++j) {
      if (j > 0) term *= y / j;
      q += term;
    }
    q *= std::exp(-y);
    tail += factorial(n) * std::pow((double)k, -(n + 1.0)) * q;
  }
  *ccdf = tail / total;
  *cdf = 1.0 - *ccdf;
}

// Regularized incomplete gamma: P(a,x) and Q(a,x) = 1 - P.
void gamma_pq(double a, double x, double* P, double* Q) {
  if (x <= 0.0) {
    *P = 0.0;
    *Q = 1.0;
    return;
  }
  const double lpre = -x + a * std::log(x) - std::lgamma(a);
  if (x < a + 1.0) {
    double ap = a, del = 1.0 / a, sum = del;
    for (int i = 0; i < 1000; ++i) {
      ap += 1.0;
      del *= x / ap;
      sum += del;
      if (std::fabs(del) < std::fabs(sum) * 1e-17) break;
    }
    *P = sum * std::exp(lpre);
    *Q = 1.0 - *P;
    return;
  }
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 1000; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (std::fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (std::fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (std::fabs(del - 1.0) < 1e-17) break;
  }
  *Q = std::exp(lpre) * h;
  *P = 1.0 - *Q;
}

template <class F>
static void build(F cdfs, float* out) {
  const double h = (double)(kTableY1 - kTableY0) / (kTableN - 1);
  for (int i = 0; i < kTableN; ++i) {
    const double y = kTableY0 + i * h;
    double u, v;
    if (y < 0) {
      const double e = std::exp(y);
      u = e / (1.0 + e);
    } else {
      u = 1.0 / (1.0 + std::exp(-y));
    }
    v = 1.0 / (1.0 + std::exp(y));
    double lo = std::log(1e-12), hi = std::log(400.0);
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      double c, cc;
      cdfs(std::exp(mid), &c, &cc);
      const bool below = (u < 0.5) ? (c < u) : (cc > v);
      if (below) lo = mid;
      else hi = mid;
    }
    out[i] = (float)(0.5 * (lo + hi));
  }
}

void build_tables(double brems_shape, float* out) {
  static std::mutex mu;
  static std::vector<float> fixed;             // Compton, Planck, MB (parameter free)
  static std::map<double, std::vector<float>> brems;
  std::lock_guard<std::mutex> lock(mu);
  if (fixed.empty()) {
    fixed.resize(3 * (size_t)kTableN);
    build([](double x, double* c, double* cc) { bose_cdf(4, x, c, cc); }, fixed.data());
    build([](double x, double* c, double* cc) { bose_cdf(2, x, c, cc); }, fixed.data() + kTableN);
    build([](double x, double* c, double* cc) { gamma_pq(3.0, x, c, cc); }, fixed.data() + 2 * kTableN);
  }
  auto it = brems.find(brems_shape);
  if (it == brems.end()) {
    std::vector<float> t(kTableN);
    build([brems_shape](double x, double* c, double* cc) { gamma_pq(brems_shape, x, c, cc); }, t.data());
    it = brems.emplace(brems_shape, std::move(t)).first;
  }
  for (int i = 0; i < kTableN; ++i) {
    out[TAB_COMPTON * kTableN + i] = fixed[i];
    out[TAB_PLANCK * kTableN + i] = fixed[kTableN + i];
    out[TAB_MBAXION * kTableN + i] = fixed[2 * kTableN + i];
    out[TAB_BREMS * kTableN + i] = it->second[i];
  }
}

}  // namespace axpic
