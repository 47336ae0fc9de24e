// Per-cell records of the table and surrogate rate models.
//
// Table model (rate model 1): the exact targets tabulated on the host over
// (ln kappa/T, log10 n_e, Z) and interpolated bilinearly per cell into a
// 192-float spectral record.
//
// Surrogate model (rate model 2): the network evaluated once per cell (its
// inputs are the cell features; every x-dependence is in the exact shapes),
// one tcgen05 row per cell, giving the cell's three ln-emissivity constants;
// they become the prefactors of the closed functional forms in the cell
// record (srnet.cuh). Cells whose (T, n_e, Z) lies outside the region where
// the network's validated error is within the bound get the table's
// spectral record instead, written by the same CTA. The kernel runs right
// after the feedback kernel of every evolved-T step (the records then hold
// the new temperature with closed-form prefactors), at set-up, and after the
// caller changes T or the composition.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "mlp.h"
#include "sr.h"
#include "srnet.cuh"
#include "step.h"
#include "surrogate.h"

namespace axpic {

void build_sr_table(int nkt, int nne, double brems_shape, float* out) {
  const int nodes = 2 * nne * nkt;
  double uni[93];
  sur_universal_knots(brems_shape, uni);
  const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) {
    th.emplace_back([=, &uni]() {
      double knots[93], y[96];
      for (int node = t; node < nodes; node += nth) {
        const int i = node % nkt, j = (node / nkt) % nne, z = node / (nkt * nne);
        const double kT = std::exp(std::log(kSurKtLo) + std::log(kSurKtHi / kSurKtLo) * i / (nkt - 1));
        const double ne = std::pow(10.0, 23.0 + 3.0 * j / (nne - 1));
        const double Z = z + 1.0;
        const SurCell c = sur_cell(sur_temperature(kT, ne, Z), ne, Z, brems_shape);
        sur_knots(c, knots, uni);
        // the bremsstrahlung brackets, (b_eZ + c_ee b_ee) / (1 + c_ee) with
        // the 1e-3 floor, divided out of that row
        const double XH = Z == 1.0 ? 1.0 : 0.0;
        const double cee = (1.0 + XH) / (2.0 * std::sqrt(2.0));
        const double lnbr = std::log((std::max(1e-3, c.bZ) + cee * std::max(1e-3, c.bE)) / (1.0 + cee));
        float* o = out + (size_t)node * kSrTabOut;
        for (int k = 0; k < kSrGrid; ++k) {
          const double x = std::exp(std::log(kSurXLo) + std::log(kSurXHi / kSurXLo) / 29.0 * (k - 1));
          sur_targets(x, c, knots, y);
          for (int ch = 0; ch < 3; ++ch) o[ch * 32 + k] = (float)(y[32 * ch] + x - (ch == 2 ? lnbr : 0.0));
        }
        for (int q = 0; q < 93; ++q) o[96 + q] = (float)knots[q];
      }
    });
  }
  for (auto& x : th) x.join();
}

// ---------------------------------------------------------------- table model
// A CTA takes 32 cells: warp 0 forms each cell's interpolation constants
// (lane per cell) in shared memory, then the CTA's threads stream the 32 x
// 192 record entries (consecutive threads, consecutive entries of a cell).
constexpr int kSrTableThreads = 256;
__global__ void __launch_bounds__(kSrTableThreads) sr_table_kernel(SrArgs a) {
  __shared__ SrInterp ip[32];
  const int c0 = a.cell0 + blockIdx.x * 32;
  const int nc = min(32, a.cell0 + a.ncells - c0);
  if (threadIdx.x < 32 && (int)threadIdx.x < nc)
    sr_interp(a.ra, sr_cell_from(a.rec + (size_t)(c0 + threadIdx.x) * kRecLen, a.ra.k_T7), &ip[threadIdx.x]);
  __syncthreads();
  for (int e = threadIdx.x; e < nc * kSrLen; e += kSrTableThreads) {
    const int c = e / kSrLen, o = e - c * kSrLen;
    a.ra.sr[(size_t)(c0 + c) * kSrLen + o] = sr_table_entry(a.ra, ip[c], o);
  }
}

cudaError_t launch_sr_table(const SrArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  sr_table_kernel<<<(a.ncells + 31) / 32, kSrTableThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- surrogate model
// A persistent grid: each CTA sets the network up once (tensor memory, the
// weights' image in shared memory) and takes tiles of 128 consecutive cells,
// thread t = cell t of the tile = tensor-core row t. The network runs for a
// tile that has a trusted cell; trusted cells get their rate prefactors,
// the others the table record (a warp per cell, after the network).
__global__ void __launch_bounds__(kNetThreads) sr_cells_kernel(SrArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ NetShared ns;
  __shared__ int list[kNetThreads];
  __shared__ int nlist;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (a.ncells + kNetThreads - 1) / kNetThreads;
  const bool net = a.ra.trust != nullptr;
  if (net) net_begin(&ns, sm, a.ra.img);
  // each thread's record one tile ahead: its load runs under this tile's network
  float4 nx[kRecLen / 4];
  {
    const int cell = a.cell0 + blockIdx.x * kNetThreads + tid;
    if (blockIdx.x < ntiles && cell < a.cell0 + a.ncells) {
      const float4* r4 = reinterpret_cast<const float4*>(a.rec + (size_t)cell * kRecLen);
#pragma unroll
      for (int i = 0; i < kRecLen / 4; ++i) nx[i] = r4[i];
    }
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int cell = a.cell0 + tile * kNetThreads + tid;
    const bool valid = cell < a.cell0 + a.ncells;
    if (tid == 0) nlist = 0;
    float r[kRecLen];
#pragma unroll
    for (int i = 0; i < kRecLen / 4; ++i) {
      r[4 * i] = nx[i].x;
      r[4 * i + 1] = nx[i].y;
      r[4 * i + 2] = nx[i].z;
      r[4 * i + 3] = nx[i].w;
    }
    {
      const int nt = tile + gridDim.x, ncell = a.cell0 + nt * kNetThreads + tid;
      if (nt < ntiles && ncell < a.cell0 + a.ncells) {
        const float4* r4 = reinterpret_cast<const float4*>(a.rec + (size_t)ncell * kRecLen);
#pragma unroll
        for (int i = 0; i < kRecLen / 4; ++i) nx[i] = r4[i];
      }
    }
    SrCellIn ci = {1.f, 1.f, 0.f, 24.f, 0.f};
    bool trusted = false;
    if (valid) {
      ci = sr_cell_from(r, a.ra.k_T7);
      trusted = net && sr_trusted(a.ra, ci.T, ci.lne);
    }
    if (__syncthreads_or(trusted)) {
      float c[3];
      const bool ok = net_rows(&ns, sm, net_f1(ci.lkT), net_f2(ci.lne), a.ra.Z - 1.5f, c, a.err);
      trusted = trusted && ok;
      if (trusted) {
        net_prefactors(a.ra, c, ci.T, r[R_NE], r);
        float4* o = reinterpret_cast<float4*>(a.rec + (size_t)cell * kRecLen);
        o[0] = make_float4(r[0], r[1], r[2], r[3]);
        o[1] = make_float4(r[4], r[5], r[6], r[7]);
      }
    }
    if (valid) {
      a.ra.src[cell] = trusted ? 0 : 1;
      if (!trusted) list[atomicAdd(&nlist, 1)] = tid;
    }
    __syncthreads();
    const int n = nlist;
    for (int k = warp; k < n; k += kNetThreads / 32) {
      const int c = a.cell0 + tile * kNetThreads + list[k];
      const SrCellIn cc = sr_cell_from(a.rec + (size_t)c * kRecLen, a.ra.k_T7);
      sr_table_record_warp(a.ra, cc, a.ra.sr + (size_t)c * kSrLen, lane);
    }
    __syncthreads();  // the list and nlist are reused by the next tile
  }
  if (net) net_end(&ns);
}

static int g_sr_cells_grid = 0;

cudaError_t launch_sr_cells(const SrArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  const int ntiles = (a.ncells + kNetThreads - 1) / kNetThreads;
  const int grid = std::max(1, std::min(ntiles, g_sr_cells_grid > 0 ? g_sr_cells_grid : ntiles));
  sr_cells_kernel<<<grid, kNetThreads, kNetSmemBytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sr_records(int model, const SrArgs& a, cudaStream_t st) {
  if (model == 1) return launch_sr_table(a, st);
  if (model == 2) return launch_sr_cells(a, st);
  return cudaSuccess;
}

// The persistent grid: as many CTAs as the device holds at once (worked out
// from the kernel's registers and shared memory: 7 an SM on a GB300), at
// most 8 an SM (64 of the 512 tensor-memory columns each).
cudaError_t sr_init_kernels() {
  const cudaError_t e =
      cudaFuncSetAttribute(sr_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kNetSmemBytes);
  if (e) return e;
  const int n = resident_ctas((const void*)sr_cells_kernel, kNetThreads, kNetSmemBytes, 8);
  if (n <= 0) return cudaErrorUnknown;
  g_sr_cells_grid = n;
  return cudaSuccess;
}

// ---------------------------------------------------------------- network image
// The image of srnet.cuh from the FP32 parameters and the output model.
__global__ void net_image_kernel(const float* __restrict__ P, const float* __restrict__ mu,
                                 const float* __restrict__ sigma, const float* __restrict__ skip,
                                 unsigned char* __restrict__ img) {
  __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(img + kImgW2);
  __nv_bfloat16* w3 = reinterpret_cast<__nv_bfloat16*>(img + kImgW3);
  float4* l1 = reinterpret_cast<float4*>(img + kImgL1);
  float* b2 = reinterpret_cast<float*>(img + kImgB2);
  float4* aff = reinterpret_cast<float4*>(img + kImgAff);
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
    const int n = i >> 6, k = i & 63;
    w2[core_off(n, k, 64)] = __float2bfloat16_rn(P[kOffW2 + k * 64 + n]);
  }
  for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
    const int n = i >> 6, k = i & 63;
    w3[core_off(n, k, 64)] = __float2bfloat16_rn(n < 3 ? P[kOffW3 + k * 96 + 32 * n] : 0.f);
  }
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    l1[j] = make_float4(P[kOffB1 + j], P[kOffW1 + 64 + j], P[kOffW1 + 128 + j], P[kOffW1 + 192 + j]);
    b2[j] = P[kOffB2 + j];
  }
  if (threadIdx.x < 3) {
    const int o = 32 * threadIdx.x;
    aff[threadIdx.x] = make_float4(fmaf(sigma[o], P[kOffB3 + o], mu[o]), sigma[o], skip[o * 4 + 1], skip[o * 4 + 2]);
  }
  if (threadIdx.x == 0) aff[3] = make_float4(skip[0 * 4 + 3], skip[32 * 4 + 3], skip[64 * 4 + 3], 0.f);
}

cudaError_t launch_net_image(const float* P, const float* mu, const float* sigma, const float* skip, void* img,
                             cudaStream_t st) {
  net_image_kernel<<<1, 256, 0, st>>>(P, mu, sigma, skip, static_cast<unsigned char*>(img));
  return cudaGetLastError();
}

}  // namespace axpic
