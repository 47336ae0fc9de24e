// The spectral surrogate's network evaluated for a CTA of 128 cells, one
// tensor-core row per cell (internal to libaxpic; used by the record kernel
// of rate model 2, sr_cells_kernel).
//
// The model's ln-emissivity outputs are y_c(x) = shape_c(x, kappa/T) + c_c,
// with shape_c each channel's exact x-dependence and c_c = mu + S f + sigma z
// a function of the cell alone (z the network at the cell features f). So a
// cell's three constants c_P, c_C, c_B are all the step needs from the
// network: with them the channels' rates keep their closed functional forms
// (Eqs. prim_rate, GammaC, gamma_abs) and only the prefactors change,
//   Gamma_{gamma->a} dt = exp(c_P + ln_gP - 4 ln T) F(s),
//   tau_C = exp(c_C + ln_gA - 4 ln T) x^2 e^x / (e^x - 1),
//   tau_B = exp(c_B + ln_gA - 4 ln T) x^(a-3),
//   lambda_C / w_e = exp(c_C + lnK_CC) / (n_e' T) (Q_C = g_ae^2 e^c_C Gamma(6) zeta(6)),
//   lambda_B / w_e = exp(c_B + lnK_CB) / (n_e' T) (Q_B = g_ae^2 e^c_B Gamma(a + 1)).
// The Compton-like and bremsstrahlung quantiles do not depend on the cell:
// the model carries them in mu alone (their sigma and S are zero).
//
// Layer 1 (K = 4) runs on the CUDA cores; layer 2 (64 x 64) and layer 3
// (the three ln-emissivity columns, N = 16) are tcgen05.mma kind::f16 with
// bfloat16 operands in shared memory and FP32 accumulators in 64 columns of
// tensor memory, issued by one thread and committed to an mbarrier with a
// bounded wait.
#pragma once
#include <cuda_bf16.h>

#include "mlp.h"
#include "sr.h"
#include "tc.cuh"

namespace axpic {

// The network's image, laid out once per network (launch_net_image) and
// copied by each CTA into its shared memory as it is:
//   [kImgW2, +8192)   W2^T (64 x 64 bfloat16, core-matrix layout)
//   [kImgW3, +2048)   W3 columns 0, 32, 64 as rows 0..2 of a 16 x 64 B^T
//                     (bfloat16, core-matrix layout, rows 3..15 zero)
//   [kImgL1, +1024)   layer 1: 64 float4 {b1_j, W1[1][j], W1[2][j], W1[3][j]}
//   [kImgB2, +256)    b2
//   [kImgAff, +64)    per ln-emissivity output k (o = 32 k): float4 {mu + sigma b3,
//                     sigma, S_o1, S_o2}, then float4 {S_o3 for k = 0, 1, 2, 0}
constexpr int kImgW2 = 0, kImgW3 = 8192, kImgL1 = 10240, kImgB2 = 11264, kImgAff = 11520;
static_assert(kNetImgBytes == kImgAff + 64, "image size");
constexpr int kNetThreads = 128;
// shared memory of a CTA that runs the network: the activation tile (128 x 64
// bfloat16, 1024-aligned) then the image
constexpr int kNetActBytes = 128 * 64 * 2;
constexpr int kNetSmemBytes = kNetActBytes + kNetImgBytes;

// Eight activations (columns j0..j0+7 of row r) as bfloat16 into one 16-byte
// row of a core matrix.
__device__ __forceinline__ void net_store8(__nv_bfloat16* base, int r, int j0, const float* v) {
  uint4 u;
  uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  *reinterpret_cast<uint4*>(base + core_off(r, j0, 64)) = u;
}

// The network's input features of a cell (the ln x input held at zero):
// ln(kappa/T), log10 n_e and Z, each mapped onto [-1, 1] over the domain.
__device__ __forceinline__ float net_f1(float lkT) { return (lkT - kSrLnKt0) / kSrLnKtSpan * 2.0f - 1.0f; }
__device__ __forceinline__ float net_f2(float lne) { return (lne - 24.5f) / 1.5f; }

// The CTA's network state: the mbarrier the tensor-core products commit to,
// the tensor-memory columns, and whether a wait ever ran out (then the
// network is not used again by this CTA).
struct NetShared {
  uint64_t bar;
  uint32_t tmem;
  int broken;
};

// Set-up, once per CTA (all threads; blockDim.x == 128): 64 tensor-memory
// columns, the mbarrier, and the image copied into sm + kNetActBytes (sm:
// kNetSmemBytes of shared memory, 1024-byte aligned).
__device__ __forceinline__ void net_begin(NetShared* ns, unsigned char* sm, const unsigned char* __restrict__ img) {
  const int tid = threadIdx.x;
  if ((tid >> 5) == 0) tmem_alloc(&ns->tmem, 64);
  if (tid == 0) {
    mbar_init(&ns->bar, 1);
    ns->broken = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const uint4* s = reinterpret_cast<const uint4*>(img);
  uint4* d = reinterpret_cast<uint4*>(sm + kNetActBytes);
  for (int i = tid; i < kNetImgBytes / 16; i += kNetThreads) d[i] = __ldg(s + i);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Release, once per CTA (all threads).
__device__ __forceinline__ void net_end(NetShared* ns) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_free(ns->tmem, 64);
}

// The network for the CTA's 128 rows (thread t = row t; all threads call
// it). Returns, CTA-uniformly, whether the tensor-core waits completed; then
// c[0..2] hold this row's constants c_P, c_C, c_B. A wait that runs out sets
// bit 4 of *err, marks the CTA's network broken and returns false. Every
// call that returns true committed twice to the mbarrier (parities 0 then 1).
static __device__ __noinline__ bool net_rows(NetShared* ns, unsigned char* sm, float f1, float f2, float f3, float* c,
                                             int* err) {
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sm);
  unsigned char* si = sm + kNetActBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (ns->broken) return false;
  const float4* sL1 = reinterpret_cast<const float4*>(si + kImgL1);
  const float* sB2 = reinterpret_cast<const float*>(si + kImgB2);
  // layer 1 on the CUDA cores
#pragma unroll
  for (int j0 = 0; j0 < 64; j0 += 8) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 w = sL1[j0 + j];
      v[j] = act_tanh(fmaf(f3, w.w, fmaf(f2, w.z, fmaf(f1, w.y, w.x))));
    }
    net_store8(sA, tid, j0, v);
  }
  smem_to_async_proxy();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ns->tmem;
  const uint32_t row = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t lbo = 128, sbo = 8 * 128;
  const uint32_t a0 = smem_u32(sA), w2 = smem_u32(si + kImgW2), w3 = smem_u32(si + kImgW3);
  // layer 2: D[0, 64) = A1 . W2
  if (tid == 0) {
    for (int s = 0; s < 4; ++s)
      mma_bf16(tmem, mma_desc(a0 + s * 256, lbo, sbo), mma_desc(w2 + s * 256, lbo, sbo), mma_idesc(128, 64), s > 0);
    tc_commit(&ns->bar);
  }
  bool ok;
  {
    bool w = true;
    if (warp == 0) w = __all_sync(0xFFFFFFFFu, mbar_wait(&ns->bar, 0));
    ok = __syncthreads_and(w) != 0;
  }
  tc_fence_after();
  if (ok) {
    // layer 2's activations over layer 1's (the MMA that read them is done)
#pragma unroll
    for (int j0 = 0; j0 < 64; j0 += 16) {
      float v[16];
      tmem_ld16(row + j0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = act_tanh(v[j] + sB2[j0 + j]);
      net_store8(sA, tid, j0, v);
      net_store8(sA, tid, j0 + 8, v + 8);
    }
  }
  smem_to_async_proxy();
  tc_fence_before();
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  // layer 3, the three ln-emissivity columns: D[0, 16) = A2 . W3'
  if (ok && tid == 0) {
    for (int s = 0; s < 4; ++s)
      mma_bf16(tmem, mma_desc(a0 + s * 256, lbo, sbo), mma_desc(w3 + s * 256, lbo, sbo), mma_idesc(128, 16), s > 0);
    tc_commit(&ns->bar);
  }
  const bool issued3 = ok;
  if (ok) {
    bool w = true;
    if (warp == 0) w = __all_sync(0xFFFFFFFFu, mbar_wait(&ns->bar, 1));
    ok = __syncthreads_and(w) != 0;
  }
  tc_fence_after();
  if (ok) {
    float y[16];
    tmem_ld16(row, y);
    const float4* aff = reinterpret_cast<const float4*>(si + kImgAff);
    const float4 s3 = aff[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 q = aff[k];
      const float S3 = k == 0 ? s3.x : (k == 1 ? s3.y : s3.z);
      c[k] = fmaf(S3, f3, fmaf(q.w, f2, fmaf(q.z, f1, fmaf(q.y, y[k], q.x))));
    }
  } else if (warp == 0) {
    // flag it and give the tensor core a second bounded wait on whatever it
    // may still be doing before the tensor memory is read or released again
    if (lane == 0) {
      atomicOr(err, 4);
      ns->broken = 1;
    }
    mbar_wait(&ns->bar, issued3 ? 1u : 0u);
  }
  // every thread has read its rows out of tensor memory before the next
  // products write there
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return ok;
}

// The cell-record slots the network's constants c (c_P, c_C, c_B) give.
__device__ __forceinline__ void net_prefactors(const RecordArgs& a, const float* c, float T, float ne1e24,
                                               float* rec) {
  const float lT = __logf(T);
  const float lnT4 = 4.0f * lT;
  const float lnneT = __logf(ne1e24) + lT;
  rec[R_AP] = expf((c[0] + a.ln_gP) - lnT4);
  rec[R_BC] = expf((c[1] + a.ln_gA) - lnT4);
  rec[R_BB] = expf((c[2] + a.ln_gA) - lnT4);
  rec[R_CC] = expf((c[1] + a.lnK_CC) - lnneT);
  rec[R_CB] = expf((c[2] + a.lnK_CB) - lnneT);
}

}  // namespace axpic
