// Auxiliary kernels of libaxpic: the synthetic initial plasma, per-cell rate
// records and cached electron moments, deterministic rate evaluation for
// checking, and the reductions behind the tallies.
#include "common.cuh"
#include "misc.h"

namespace axpic {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// ---------------------------------------------------------------- records
__global__ void record_kernel(int ncells, int nspecies, CellConst cc, const double* __restrict__ T,
                              const double* __restrict__ n_ion, float* rec, int* err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  float r[kRecLen];
#pragma unroll
  for (int i = 0; i < kRecLen; ++i) r[i] = 0.f;
  compute_composition(cc, n_ion + (size_t)c * nspecies, r);
  const float Tc = (float)T[c];
  if (!(Tc > 0.f) || !isfinite(Tc)) atomicOr(err, ERR_NUMERIC);
  compute_temperature(cc, Tc, r);
  float4* o = reinterpret_cast<float4*>(rec + (size_t)c * kRecLen);
#pragma unroll
  for (int i = 0; i < kRecLen / 4; ++i) o[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
}

cudaError_t launch_records(int ncells, int nspecies, const CellConst& cc, const double* T, const double* n_ion,
                           float* rec, int* err, cudaStream_t st) {
  if (ncells == 0) return cudaSuccess;
  record_kernel<<<(ncells + 127) / 128, 128, 0, st>>>(ncells, nspecies, cc, T, n_ion, rec, err);
  return cudaGetLastError();
}

// FP64 view of a cell's parameters (for checking): from the record, with the
// temperature-dependent extras recomputed exactly as the step kernels do.
__global__ void info_kernel(int first, int count, CellConst cc, double k_gamma, const float* __restrict__ rec_all,
                            double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int c = first + i;
  float r[kRecLen];
  for (int k = 0; k < kRecLen; ++k) r[k] = rec_all[(size_t)c * kRecLen + k];
  const CellExtras ex = compute_temperature(cc, r[R_T], r);
  double* o = out + (size_t)i * AXPIC_CELL_INFO_LEN;
  for (int k = 0; k < AXPIC_CELL_INFO_LEN; ++k) o[k] = 0.0;
  o[AXPIC_CI_RHO] = r[R_RHO];
  o[AXPIC_CI_XH] = r[R_XH];
  o[AXPIC_CI_NE] = (double)r[R_NE] * 1e24;
  o[AXPIC_CI_NEFF] = (double)r[R_NEFF] * 1e24;
  o[AXPIC_CI_SZ] = (double)r[R_SZ] * 1e24;
  o[AXPIC_CI_KAPPA] = ex.kappa;
  o[AXPIC_CI_QC] = ex.QC;
  o[AXPIC_CI_QB] = ex.QB;
  // k_gamma = 1 / (dt w_a^-1): recover Gamma from lambda per unit weight
  o[AXPIC_CI_GAMMA_C] = (double)r[R_CC] * k_gamma;
  o[AXPIC_CI_GAMMA_B] = (double)r[R_CB] * k_gamma;
  o[AXPIC_CI_ETA] = ex.eta;
  o[AXPIC_CI_T] = r[R_T];
  o[AXPIC_CI_GAMMA0_P] = (double)r[R_AP];  // Gamma_0 dt; the host divides by dt
}

cudaError_t launch_info(int first, int count, const CellConst& cc, double k_gamma, const float* rec, double* out,
                        cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  info_kernel<<<(count + 127) / 128, 128, 0, st>>>(first, count, cc, k_gamma, rec, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- deposit
// Composition from the deposited electron density (Sec. II.E, Eqs. rho_def,
// qn_def): n_e = sum w / V over the cell's electron macroparticles, then
// n_i = n_e * coef_i: the host's coefficients hold coef_i / V, so the device
// does no FP64 division. One warp per cell, the
// sum kept as an unevaluated binary32 pair (hi, lo): Knuth's TwoSum gives
// the exact rounding error of each hi + w, accumulated in lo, so the pair is
// within about (terms) 2^-48 of the exact sum without the FP64 pipe. The
// lanes' pairs are combined the same way; one FP64 add per cell evaluates
// the pair.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float w) {
  const float s = __fadd_rn(hi, w);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(w, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

__global__ void deposit_kernel(int ncells, int nspecies, SpeciesPtrs e, DepositCoef k, double* __restrict__ n_ion) {
  constexpr int kU = 4;  // quads in flight per lane
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncells) return;
  const int n = min(max(e.count[c], 0), e.cap);
  // quads of slots (cap is a multiple of 4); the weight is the first word of
  // each slot's record
  const float* wr = reinterpret_cast<const float*>(e.wp + (long)c * e.cap);
  float hi = 0.f, lo = 0.f;
  for (int q0 = lane; 4 * q0 < n; q0 += 32 * kU) {
    float4 v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = q0 + 32 * u;
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * q < n) {
        const float* p = wr + 16 * q;
        v[u] = make_float4(__ldcs(p), __ldcs(p + 4), __ldcs(p + 8), __ldcs(p + 12));
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int j = 4 * (q0 + 32 * u);  // slots past the count add +0
      two_sum_add(hi, lo, v[u].x);
      two_sum_add(hi, lo, j + 1 < n ? v[u].y : 0.f);
      two_sum_add(hi, lo, j + 2 < n ? v[u].z : 0.f);
      two_sum_add(hi, lo, j + 3 < n ? v[u].w : 0.f);
    }
  }
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(kFullMask, hi, o), l2 = __shfl_xor_sync(kFullMask, lo, o);
    two_sum_add(hi, lo, h2);
    lo = __fadd_rn(lo, l2);
  }
  // lane 0's pair for every species (the lanes combined in different orders)
  hi = __shfl_sync(kFullMask, hi, 0);
  lo = __shfl_sync(kFullMask, lo, 0);
  if (lane < nspecies) {  // the FP64 work, in these lanes only
    double cf = 0.0;      // coef[lane], read with constant indices (no local copy)
#pragma unroll
    for (int i = 0; i < kMaxSpecies; ++i)
      if (lane == i) cf = k.coef[i];
    n_ion[(size_t)c * nspecies + lane] = ((double)hi + (double)lo) * cf;
  }
}

cudaError_t launch_deposit(int ncells, int nspecies, const SpeciesPtrs& e, const DepositCoef& k, double* n_ion,
                           cudaStream_t st) {
  if (ncells == 0) return cudaSuccess;
  deposit_kernel<<<(ncells + 7) / 8, 256, 0, st>>>(ncells, nspecies, e, k, n_ion);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- moments
// Cached electron moments W, P, U2 and var = U2 - |P|^2 / W (Eqs.
// cell_moments, var_unnormalized), one warp per cell.
__global__ void moments_kernel(int ncells, SpeciesPtrs e, float* mom) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncells) return;
  const int n = min(max(e.count[c], 0), e.cap);
  const long b = (long)c * e.cap;
  float W = 0.f, Px = 0.f, Py = 0.f, Pz = 0.f, U2 = 0.f;
  float wmin = 3.0e38f, wmax = -3.0e38f;
  for (int i = lane; i < n; i += 32) {
    const float4 r = e.wp[b + i];
    const float w = r.x, px = r.y, py = r.z, pz = r.w;
    wmin = fminf(wmin, w);
    wmax = fmaxf(wmax, w);
    W += w;
    Px += w * px;
    Py += w * py;
    Pz += w * pz;
    U2 += w * (px * px + py * py + pz * pz);
  }
  for (int o = 16; o; o >>= 1) {
    W += __shfl_xor_sync(kFullMask, W, o);
    Px += __shfl_xor_sync(kFullMask, Px, o);
    Py += __shfl_xor_sync(kFullMask, Py, o);
    Pz += __shfl_xor_sync(kFullMask, Pz, o);
    U2 += __shfl_xor_sync(kFullMask, U2, o);
    wmin = fminf(wmin, __shfl_xor_sync(kFullMask, wmin, o));
    wmax = fmaxf(wmax, __shfl_xor_sync(kFullMask, wmax, o));
  }
  if (lane == 0) {
    float* m = mom + (size_t)c * kMomLen;
    m[M_W] = W;
    m[M_PX] = Px;
    m[M_PY] = Py;
    m[M_PZ] = Pz;
    m[M_U2] = U2;
    m[M_VAR] = W > 0.f ? fmaxf(0.f, U2 - (Px * Px + Py * Py + Pz * Pz) / W) : 0.f;
    m[M_WU] = (n > 0 && wmin == wmax && wmin > 0.f) ? wmin : 0.f;
    m[7] = 0.f;
  }
}

cudaError_t launch_moments(int ncells, const SpeciesPtrs& e, float* mom, cudaStream_t st) {
  if (ncells == 0) return cudaSuccess;
  moments_kernel<<<(ncells + 7) / 8, 256, 0, st>>>(ncells, e, mom);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sampler
// Synthetic initial plasma: per cell, NR-Maxwellian electrons (Box-Muller on
// block sub 0, positions on sub 1), Planck photons and MB-equilibrium axions
// (energy from word 0 through the inverse-CDF tables, direction from words 1
// and 2, positions on sub 1). One warp per cell.
__global__ void sample_kernel(SampleArgs S) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= S.ncells) return;
  const uint32_t gcell = S.cell_base + (uint32_t)c;
  const float* rec = S.rec + (size_t)c * kRecLen;
  const float T = rec[R_T];
  const float sigma = sqrtf(T * kInvMeC2f);
  const float we = rec[R_NE] * S.k_we;             // n_e V / n_el
  const float wg = T * T * T * S.k_wg;             // n_gamma V / n_ph
  for (int sp = 0; sp < 3; ++sp) {
    const SpeciesPtrs& P = sp == 0 ? S.e : (sp == 1 ? S.g : S.a);
    const int n = sp == 0 ? S.n_el : (sp == 1 ? S.n_ph : S.n_ax);
    const uint32_t stream = sp == 0 ? S_INIT_E : (sp == 1 ? S_INIT_G : S_INIT_A);
    const long b = (long)c * P.cap;
    for (int i = lane; i < n; i += 32) {
      const uint4 b0 = philox4x32_10(make_uint4(kInitStep, gcell, (uint32_t)i, stream << 24), S.key0, S.key1);
      const uint4 b1 = philox4x32_10(make_uint4(kInitStep, gcell, (uint32_t)i, (stream << 24) | 1u), S.key0, S.key1);
      float w, px, py, pz;
      if (sp == 0) {
        const float r1 = sqrtf(-2.0f * logf(u23(b0.x)));
        const float r2 = sqrtf(-2.0f * logf(u23(b0.z)));
        float s1, c1, s2, c2;
        sincospif(2.0f * u23(b0.y), &s1, &c1);
        sincospif(2.0f * u23(b0.w), &s2, &c2);
        px = sigma * r1 * c1;
        py = sigma * r1 * s1;
        pz = sigma * r2 * c2;
        w = we;
      } else {
        const float* tab = S.tables + (sp == 1 ? TAB_PLANCK : TAB_MBAXION) * kTableN;
        const float pm = icdf_lookup(tab, u23(b0.x)) * T * kInvMeC2f;
        const float3 d = iso_dir(u23(b0.y), u23(b0.z));
        px = pm * d.x;
        py = pm * d.y;
        pz = pm * d.z;
        w = sp == 1 ? wg : S.w_a;
      }
      P.wp[b + i] = make_float4(w, px, py, pz);
      P.xyz[b + i] = make_float4(u23(b1.x), u23(b1.y), u23(b1.z), 0.f);
    }
    if (lane == 0) P.count[c] = n;
  }
}

cudaError_t launch_sample(const SampleArgs& S, cudaStream_t st) {
  if (S.ncells == 0) return cudaSuccess;
  sample_kernel<<<(S.ncells + 7) / 8, 256, 0, st>>>(S);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- rates
__global__ void rates_kernel(const float* __restrict__ rec_all, int cell, const float* __restrict__ E, int n,
                             int eq_stats, float am3, float prim_mult, float mu2, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float rec[kRecLen];
  for (int k = 0; k < kRecLen; ++k) rec[k] = rec_all[(size_t)cell * kRecLen + k];
  const float om = E[i];
  const float x = om * rec[R_INVT];
  // gamma->a of a massive axion: beta(omega) times the rate (1 when massless)
  const float beta = mu2 > 0.f ? axion_beta(om * kInvMeC2f, mu2) : 1.0f;
  out[4 * i + 0] = prim_prob(rec, om, beta * rec[R_AP]);
  out[4 * i + 1] = prim_prob(rec, om, prim_mult * rec[R_AP]);
  out[4 * i + 2] = tau_compton(rec, x, eq_stats);
  out[4 * i + 3] = tau_brems(rec, x, am3, eq_stats);
}

cudaError_t launch_rates(const float* rec, int cell, const float* E, int n, int eq_stats, float am3, float prim_mult,
                         float mu2, float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  rates_kernel<<<(n + 255) / 256, 256, 0, st>>>(rec, cell, E, n, eq_stats, am3, prim_mult, mu2, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions
// Column sums of the per-CTA counters.
__global__ void counters_kernel(const unsigned long long* __restrict__ ctr, int rows, double* out) {
  const int col = blockIdx.x;
  unsigned long long s = 0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += ctr[(size_t)r * kNumCounters + col];
  __shared__ unsigned long long buf[256];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[col] = (double)buf[0];
}

// Alive totals: sum w and sum w E for axions and photons, electron NR
// kinetic energy, macroparticle counts and carried energy. One warp per cell,
// FP64 atomics once per warp.
__global__ void totals_kernel(int ncells, SpeciesPtrs e, SpeciesPtrs g, SpeciesPtrs a, const double* __restrict__ res,
                              double* out) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncells) return;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int na = min(max(a.count[c], 0), a.cap), ng = min(max(g.count[c], 0), g.cap),
            ne = min(max(e.count[c], 0), e.cap);
  for (int i = lane; i < na; i += 32) {
    const long k = (long)c * a.cap + i;
    const float4 r = a.wp[k];
    v[0] += r.x;
    v[1] += (double)r.x * sqrtf(r.y * r.y + r.z * r.z + r.w * r.w);
  }
  for (int i = lane; i < ng; i += 32) {
    const long k = (long)c * g.cap + i;
    const float4 r = g.wp[k];
    v[2] += r.x;
    v[3] += (double)r.x * sqrtf(r.y * r.y + r.z * r.z + r.w * r.w);
  }
  for (int i = lane; i < ne; i += 32) {
    const long k = (long)c * e.cap + i;
    const float4 r = e.wp[k];
    v[4] += 0.5 * (double)r.x * (double)(r.y * r.y + r.z * r.z + r.w * r.w);
  }
  if (lane == 0) {
    v[5] = na;
    v[6] = ng;
    v[7] = res[(size_t)c * 4];
  }
  for (int j = 0; j < 8; ++j) {
    double x = v[j];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
    if (lane == 0 && x != 0.0) atomicAdd(out + j, x);
  }
}

cudaError_t launch_totals(int ncells, const SpeciesPtrs& e, const SpeciesPtrs& g, const SpeciesPtrs& a,
                          const double* res, const unsigned long long* ctr, int ctr_rows, double* out8,
                          double* out_ctr, cudaStream_t st) {
  if (ncells > 0) {
    totals_kernel<<<(ncells + 7) / 8, 256, 0, st>>>(ncells, e, g, a, res, out8);
    cudaError_t err = cudaGetLastError();
    if (err) return err;
  }
  if (ctr_rows > 0) counters_kernel<<<kNumCounters, 256, 0, st>>>(ctr, ctr_rows, out_ctr);
  return cudaGetLastError();
}

}  // namespace axpic
