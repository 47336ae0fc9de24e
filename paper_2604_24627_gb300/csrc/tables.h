// Host-side sampling tables (internal to libaxpic).
#pragma once

namespace axpic {

constexpr int kTableN = 8192;
constexpr float kTableY0 = -17.0f;
constexpr float kTableY1 = 17.0f;
enum { TAB_COMPTON = 0, TAB_BREMS = 1, TAB_PLANCK = 2, TAB_MBAXION = 3, kNumTables = 4 };

double zeta(double s);
// out: kNumTables * kTableN binary32 values of ln x(logit^-1(y_i)).
void build_tables(double brems_shape, float* out);

}  // namespace axpic
