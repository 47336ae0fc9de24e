// Per-cell spectral records for the table and surrogate rate models.
//
// Table model: the exact targets tabulated on the host over (ln kappa/T,
// log10 n_e, Z) and interpolated bilinearly per cell. Surrogate model: the
// network evaluated per cell at the 32 grid points x_k in one fused kernel
// (features and layer 1 on the CUDA cores, layers 2 and 3 as tcgen05 MMAs
// with FP32 accumulators in tensor memory, output affine in FP32), written
// over the table record of every cell whose (T, n_e, Z) lies in the region
// where the network's validated error is within the bound.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "mlp.h"
#include "sr.h"
#include "surrogate.h"
#include "tc.cuh"

namespace axpic {

void build_sr_table(int nkt, int nne, double brems_shape, float* out) {
  const int nodes = 2 * nne * nkt;
  const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) {
    th.emplace_back([=]() {
      double knots[93], y[96];
      for (int node = t; node < nodes; node += nth) {
        const int i = node % nkt, j = (node / nkt) % nne, z = node / (nkt * nne);
        const double kT = std::exp(std::log(kSurKtLo) + std::log(kSurKtHi / kSurKtLo) * i / (nkt - 1));
        const double ne = std::pow(10.0, 23.0 + 3.0 * j / (nne - 1));
        const double Z = z + 1.0;
        const SurCell c = sur_cell(sur_temperature(kT, ne, Z), ne, Z, brems_shape);
        sur_knots(c, knots);
        float* o = out + (size_t)node * kSrTabOut;
        for (int k = 0; k < kSrGrid; ++k) {
          const double x = std::exp(std::log(kSurXLo) + std::log(kSurXHi / kSurXLo) / 29.0 * (k - 1));
          sur_targets(x, c, knots, y);
          for (int ch = 0; ch < 3; ++ch) o[ch * 32 + k] = (float)(y[32 * ch] + x);
        }
        for (int q = 0; q < 93; ++q) o[96 + q] = (float)knots[q];
      }
    });
  }
  for (auto& x : th) x.join();
}

// Cell quantities the records need: T, kappa/T, n_e.
__device__ __forceinline__ void sr_cell(const SrArgs& a, int cell, float* T, float* kT, float* ne) {
  const float* rec = a.rec + (size_t)cell * kRecLen;
  *T = rec[R_T];
  *kT = 2.0f * rsqrtf(rec[R_FOURK2]) / *T;
  *ne = rec[R_NE] * 1e24f;
}

// A CTA takes 32 cells: warp 0 forms each cell's interpolation constants
// (lane per cell) in shared memory, then the CTA's threads stream the 32 x
// 192 record entries (consecutive threads, consecutive entries of a cell):
// bilinear in (ln kappa/T, log10 n_e) at the cell's Z, plus the per-cell
// constants.
constexpr int kSrTableThreads = 256;
__global__ void __launch_bounds__(kSrTableThreads) sr_table_kernel(SrArgs a) {
  struct Interp {
    const float* t00;
    float fu, fv, lnKP, lnKA, T;
  };
  __shared__ Interp ip[32];
  const int c0 = blockIdx.x * 32;
  const int nc = min(32, a.ncells - c0);
  if (threadIdx.x < 32 && (int)threadIdx.x < nc) {
    float T, kT, ne;
    sr_cell(a, c0 + threadIdx.x, &T, &kT, &ne);
    float u = (__logf(kT) - kSrLnKt0) / kSrLnKtSpan * (a.nkt - 1);
    float v = (log10f(ne) - 23.0f) / 3.0f * (a.nne - 1);
    u = fminf(fmaxf(u, 0.f), (float)(a.nkt - 1));
    v = fminf(fmaxf(v, 0.f), (float)(a.nne - 1));
    const int i = min((int)u, a.nkt - 2), j = min((int)v, a.nne - 2);
    const int z = a.Z > 1.5f ? 1 : 0;
    Interp& q = ip[threadIdx.x];
    q.t00 = a.tab + ((size_t)(z * a.nne + j) * a.nkt + i) * kSrTabOut;
    q.fu = u - i;
    q.fv = v - j;
    q.lnKP = a.ln_gP - 4.0f * __logf(T);
    q.lnKA = a.ln_gA - 4.0f * __logf(T);
    q.T = T;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * kSrLen; e += kSrTableThreads) {
    const int c = e / kSrLen, o = e - c * kSrLen;
    const Interp& q = ip[c];
    float* out = a.sr + (size_t)(c0 + c) * kSrLen;
    if (o < kSrTabOut) {
      const float* t01 = q.t00 + (size_t)a.nkt * kSrTabOut;  // j + 1
      const float v00 = q.t00[o], v10 = q.t00[kSrTabOut + o], v01 = t01[o], v11 = t01[kSrTabOut + o];
      out[o] = (1.f - q.fv) * ((1.f - q.fu) * v00 + q.fu * v10) + q.fv * ((1.f - q.fu) * v01 + q.fu * v11);
    } else {
      out[o] = o == SR_LNKP ? q.lnKP : (o == SR_LNKA ? q.lnKA : q.T);
    }
  }
}

cudaError_t launch_sr_table(const SrArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  sr_table_kernel<<<(a.ncells + 31) / 32, kSrTableThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- fused network
// CTA = 4 cells x 32 grid points = 128 rows (thread = row). Shared memory:
// A1, A2 (128 x 64 bfloat16, core-matrix layout), W2^T (64 x 64), W3^T
// (96 x 64); tensor memory: 64 columns for layer 2, 96 for layer 3.
constexpr int kSrMlpThreads = 128;
constexpr size_t kSrMlpSmem = (size_t)(128 * 64 * 2 + 64 * 64 + 96 * 64) * sizeof(__nv_bfloat16);

__device__ __forceinline__ bool sr_trusted(const SrArgs& a, float T, float ne, float Z) {
  float fu = (T - (float)kSurTLo) / (float)(kSurTHi - kSurTLo) * (a.tnT - 1);
  float fv = (log10f(ne) - 23.0f) / 3.0f * (a.tnne - 1);
  // inside the validated grid (binary32 rounding at its edges tolerated)
  const float tol = 1e-4f;
  if (!(fu >= -tol && fu <= (float)(a.tnT - 1) + tol && fv >= -tol && fv <= (float)(a.tnne - 1) + tol)) return false;
  fu = fminf(fmaxf(fu, 0.f), (float)(a.tnT - 1));
  fv = fminf(fmaxf(fv, 0.f), (float)(a.tnne - 1));
  const int i = min((int)fu, a.tnT - 2), j = min((int)fv, a.tnne - 2);
  const int z = Z > 1.5f ? 1 : 0;
  const uint8_t* t = a.trust + (size_t)(z * a.tnne + j) * a.tnT + i;
  return t[0] && t[1] && t[a.tnT] && t[a.tnT + 1];
}

// The fixed x-shape of channel ch's ln-emissivity output (Primakoff: the
// Planck factor and min(s/2, ln(1 + s)), an upper bound of the screening
// function; Compton-like: x^5 / (e^x - 1); bremsstrahlung: x^a e^-x).
__device__ __forceinline__ float sr_shape(int ch, float x, float kT, float a) {
  if (ch == 0) {
    const float s = 4.0f * x * x / (kT * kT);
    return 3.0f * logf(x) - logf(expm1f(x)) + logf(fminf(0.5f * s, log1pf(s)));
  }
  if (ch == 1) return 5.0f * logf(x) - logf(expm1f(x));
  return a * logf(x) - x;
}

// Layers 2 and 3 as B^T (N x K = 64) bfloat16 in the core-matrix layout, laid
// out once per network: W2^T (64 x 64) then W3^T (96 x 64).
__global__ void sr_weights_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 64 * 64) {
    const int n = i >> 6, kk = i & 63;
    out[core_off(n, kk, 64)] = __float2bfloat16_rn(P[kOffW2 + kk * 64 + n]);
  } else if (i < 64 * 64 + 96 * 64) {
    const int j = i - 64 * 64, n = j >> 6, kk = j & 63;
    out[64 * 64 + core_off(n, kk, 64)] = __float2bfloat16_rn(P[kOffW3 + kk * 96 + n]);
  }
}

cudaError_t launch_sr_weights(const float* P, void* out, cudaStream_t st) {
  sr_weights_kernel<<<(64 * 64 + 96 * 64 + 255) / 256, 256, 0, st>>>(P, static_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kSrMlpThreads) sr_mlp_kernel(SrArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int any_trusted;
  __nv_bfloat16* sA1 = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* sA2 = sA1 + 128 * 64;
  __nv_bfloat16* sW2 = sA2 + 128 * 64;
  __nv_bfloat16* sW3 = sW2 + 64 * 64;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cell = blockIdx.x * 4 + warp, k = lane;
  const bool valid = cell < a.ncells;
  float T = 1.f, kT = 1.f, ne = 1e24f;
  if (valid) sr_cell(a, cell, &T, &kT, &ne);
  const bool trusted = valid && sr_trusted(a, T, ne, a.Z);
  if (tid == 0) any_trusted = 0;
  __syncthreads();
  if (trusted) any_trusted = 1;
  __syncthreads();
  if (!any_trusted) return;  // the table record stays: nothing to evaluate here
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the pre-laid-out weights: 20 KB of 16-byte copies
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.W16);
    uint4* dst = reinterpret_cast<uint4*>(sW2);
    for (int i = tid; i < (64 * 64 + 96 * 64) / 8; i += kSrMlpThreads) dst[i] = src[i];
  }
  // features of row (cell, k) and layer 1 on the CUDA cores
  float f[4];
  {
    f[0] = 2.0f * (k - 1) / 29.0f - 1.0f;  // ln x_k on the feature scale (x_1 -> -1, x_30 -> 1)
    f[1] = (__logf(kT) - kSrLnKt0) / kSrLnKtSpan * 2.0f - 1.0f;
    f[2] = (log10f(ne) - 24.5f) / 1.5f;
    f[3] = a.Z - 1.5f;
    for (int j = 0; j < 64; ++j) {
      float s = a.P[kOffB1 + j];
#pragma unroll
      for (int q = 0; q < 4; ++q) s = fmaf(f[q], a.P[kOffW1 + q * 64 + j], s);
      sA1[core_off(tid, j, 64)] = __float2bfloat16_rn(tanhf(s));
    }
  }
  smem_to_async_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t lbo = 128, sbo = 8 * 128;
  bool ok = true;
  if (any_trusted) {
    // layer 2: D[0, 64) = A1 . W2
    if (tid == 0) {
      for (int s = 0; s < 4; ++s)
        mma_bf16(tmem, mma_desc(smem_u32(sA1) + s * 256, lbo, sbo), mma_desc(smem_u32(sW2) + s * 256, lbo, sbo),
                 mma_idesc(128, 64), s > 0);
      tc_commit(&bar);
    }
    ok = mbar_wait(&bar, 0);
    tc_fence_after();
    if (ok) {
      const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tmem_ld16(row + c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          sA2[core_off(tid, c0 + j, 64)] = __float2bfloat16_rn(tanhf(v[j] + a.P[kOffB2 + c0 + j]));
      }
    }
    smem_to_async_proxy();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 3: D[64, 160) = A2 . W3
    if (ok && tid == 0) {
      for (int s = 0; s < 4; ++s)
        mma_bf16(tmem + 64, mma_desc(smem_u32(sA2) + s * 256, lbo, sbo),
                 mma_desc(smem_u32(sW3) + s * 256, lbo, sbo), mma_idesc(128, 96), s > 0);
      tc_commit(&bar);
    }
    bool issued3 = ok;
    if (ok) ok = mbar_wait(&bar, 1);
    tc_fence_after();
    if (!ok) {
      // flag it and give the tensor core a second bounded wait on whatever
      // it may still be doing before the tensor memory is released
      if (tid == 0) atomicOr(a.err, 2);
      mbar_wait(&bar, issued3 ? 1u : 0u);
    } else {
      const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16) + 64;
      float* out = a.sr + (size_t)cell * kSrLen;
      const float xk = __expf(kSrLnX0 + kSrH * (float)k);
      for (int c0 = 0; c0 < 96; c0 += 16) {
        float v[16];
        tmem_ld16(row + c0, v);
        if (trusted) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int o = c0 + j;
            float y = a.mu[o] + a.sigma[o] * (v[j] + a.P[kOffB3 + o]);
#pragma unroll
            for (int i = 0; i < 4; ++i) y = fmaf(a.skip[o * 4 + i], f[i], y);
            const int ch = o >> 5, slot = o & 31;
            if (slot == 0) out[ch * 32 + k] = y + sr_shape(ch, xk, kT, a.brems_a) + xk;
            else if (k == 0) out[96 + ch * 31 + slot - 1] = y;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tmem, 256);
}

cudaError_t sr_init_kernels() {
  return cudaFuncSetAttribute(sr_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSrMlpSmem);
}

cudaError_t launch_sr_mlp(const SrArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  sr_mlp_kernel<<<(a.ncells + 3) / 4, kSrMlpThreads, kSrMlpSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace axpic
