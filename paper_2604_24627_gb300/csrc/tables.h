// Host-side sampling tables (internal to libaxpic).
#pragma once

namespace axpic {

constexpr int kTableN = 8192;
constexpr float kTableY0 = -17.0f;
constexpr float kTableY1 = 17.0f;
enum { TAB_COMPTON = 0, TAB_BREMS = 1, TAB_PLANCK = 2, TAB_MBAXION = 3, kNumTables = 4 };

double zeta(double s);
// CDF and complementary CDF of the number pdf x^n/(e^x-1)/(n! zeta(n+1)).
void bose_cdf(int n, double x, double* cdf, double* ccdf);
// Regularized incomplete gamma P(a, x) and Q(a, x) = 1 - P.
void gamma_pq(double a, double x, double* P, double* Q);
// out: kNumTables * kTableN binary32 values of ln x(logit^-1(y_i)).
void build_tables(double brems_shape, float* out);

}  // namespace axpic
