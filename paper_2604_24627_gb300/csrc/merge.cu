// Axion merging for population control: in every cell holding more than
// n_target axions, each group of three or more axions of one momentum
// octant and |p|^2 bin becomes two, with the group's weight, momentum and
// energy (the N -> 2 merging of Vranic et al., Comput. Phys. Commun. 191, 65
// (2015), for massless particles; the method merges axions as a species of
// the PIC code, Sec. II.A, and names no algorithm).
//
// A warp per cell:
// * each slot's group (comparisons of binary32 |p|^2 with the thresholds,
//   and the sign bits) and the group sizes;
// * the groups of three or more in a list, and their members' slots in
//   shared memory, grouped and in slot order (a stable counting sort);
// * a lane per listed group forms the binary32 compensated sums over its
//   members in slot order, every rounding explicit (the results match the
//   oracle bit for bit), writes the two new axions into the group's first
//   two slots and frees the others;
// * the tail fill closes the freed slots.
#include "merge.h"

#include <algorithm>

namespace axpic {

namespace {

constexpr int kWarpsMax = 2;  // small blocks: a cell that finishes early frees its slot
constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kGroupsMax = (kMergeMaxEdges + 1) * 8;

__device__ __forceinline__ float fsum3(float a, float b, float c) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
}

// A compensated (Kahan) binary32 sum, every step rounded as written.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
};

// The two axions replacing the group whose m member slots, ascending, are
// mem[0..m) of the cell at base: binary32 compensated sums in slot order,
// then p_a and p_b on either side of P at cos theta = |P| / E. Members after
// the first two are freed.
__device__ void merge_group(const MergeArgs& a, long base, const uint16_t* mem, int m) {
  const SpeciesPtrs& s = a.s;
  Kahan W, Px, Py, Pz, E, X, Y, Z;
  // member k + 1's fields are loaded before member k's sums (m >= 3)
  long q = base + mem[0];
  float4 r = s.wp[q], u = s.xyz[q];
  float w = r.x, px = r.y, py = r.z, pz = r.w, x = u.x, y = u.y, z = u.z;
  for (int k = 0; k < m; ++k) {
    const long qn = base + mem[min(k + 1, m - 1)];
    r = s.wp[qn];
    u = s.xyz[qn];
    const float wn = r.x, pxn = r.y, pyn = r.z, pzn = r.w, xn = u.x, yn = u.y, zn = u.z;
    W.add(w);
    Px.add(__fmul_rn(w, px));
    Py.add(__fmul_rn(w, py));
    Pz.add(__fmul_rn(w, pz));
    E.add(__fmul_rn(w, __fsqrt_rn(fsum3(px, py, pz))));
    X.add(__fmul_rn(w, x));
    Y.add(__fmul_rn(w, y));
    Z.add(__fmul_rn(w, z));
    if (k >= 2) a.grp[q] = kMergeFreed;
    q = qn, w = wn, px = pxn, py = pyn, pz = pzn, x = xn, y = yn, z = zn;
  }
  const int sa = mem[0], sb = mem[1];
  const float pm = __fdiv_rn(E.s, W.s);
  const float Pn = __fsqrt_rn(fsum3(Px.s, Py.s, Pz.s));
  float e0, e1, e2, ct;
  if (Pn > 0.f) {
    e0 = __fdiv_rn(Px.s, Pn);
    e1 = __fdiv_rn(Py.s, Pn);
    e2 = __fdiv_rn(Pz.s, Pn);
    ct = fminf(__fdiv_rn(Pn, E.s), 1.0f);
  } else {
    e0 = 0.f, e1 = 0.f, e2 = 1.f;
    ct = 0.f;
  }
  const float st = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(ct, ct)));
  // the axis of e_P's smallest |component|, the lowest index on ties
  int k = 0;
  float amin = fabsf(e0);
  if (fabsf(e1) < amin) k = 1, amin = fabsf(e1);
  if (fabsf(e2) < amin) k = 2;
  const float ax0 = k == 0 ? 1.f : 0.f, ax1 = k == 1 ? 1.f : 0.f, ax2 = k == 2 ? 1.f : 0.f;
  const float u0 = __fsub_rn(__fmul_rn(e1, ax2), __fmul_rn(e2, ax1));
  const float u1 = __fsub_rn(__fmul_rn(e2, ax0), __fmul_rn(e0, ax2));
  const float u2 = __fsub_rn(__fmul_rn(e0, ax1), __fmul_rn(e1, ax0));
  const float un = __fsqrt_rn(fsum3(u0, u1, u2));
  const float e[3] = {e0, e1, e2};
  const float qv[3] = {__fdiv_rn(u0, un), __fdiv_rn(u1, un), __fdiv_rn(u2, un)};
  const float wh = __fmul_rn(W.s, 0.5f);
  const float mx = __fdiv_rn(X.s, W.s), my = __fdiv_rn(Y.s, W.s), mz = __fdiv_rn(Z.s, W.s);
  float pa[3], pb[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    pa[j] = __fmul_rn(pm, __fadd_rn(__fmul_rn(ct, e[j]), __fmul_rn(st, qv[j])));
    pb[j] = __fmul_rn(pm, __fsub_rn(__fmul_rn(ct, e[j]), __fmul_rn(st, qv[j])));
  }
  const long qa = base + sa, qb = base + sb;
  s.wp[qa] = make_float4(wh, pa[0], pa[1], pa[2]);
  s.xyz[qa] = make_float4(mx, my, mz, 0.f);
  s.wp[qb] = make_float4(wh, pb[0], pb[1], pb[2]);
  s.xyz[qb] = make_float4(mx, my, mz, 0.f);
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Dynamic shared memory: cap slot indices (u16) per warp.
__global__ void __launch_bounds__(kWarpsMax * 32, 20) merge_kernel(MergeArgs a) {
  extern __shared__ uint16_t smem_members[];
  __shared__ int gcnt[kWarpsMax][kGroupsMax];  // group sizes
  __shared__ int gpos[kWarpsMax][kGroupsMax];  // next member position of a listed group
  __shared__ uint8_t glist[kWarpsMax][kGroupsMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const SpeciesPtrs& s = a.s;
  uint16_t* mem = smem_members + (size_t)wid * s.cap;
  const int ngroups = (a.nedges + 1) * 8;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = blockIdx.x * nw + wid; c < a.ncells; c += gridDim.x * nw) {
    const int n = min(max(s.count[c], 0), s.cap);
    if (n <= a.n_target) continue;
    const long base = (long)c * s.cap;
    for (int g = lane; g < ngroups; g += 32) gcnt[wid][g] = 0;
    __syncwarp();
    // each slot's group: the number of thresholds at or below |p|^2, times
    // 8, plus the octant of p; the other fields' lines go to L1 meanwhile
    for (int s0 = 0; s0 < n; s0 += 32) {
      const int slot = s0 + lane;
      if (slot < n) {
        const long q = base + slot;
        prefetch_l1(s.xyz + q);
        const float4 r = s.wp[q];
        const float px = r.y, py = r.z, pz = r.w;
        const float p2 = __fadd_rn(__fadd_rn(__fmul_rn(px, px), __fmul_rn(py, py)), __fmul_rn(pz, pz));
        int e = 0;
        for (int k = 0; k < a.nedges; ++k) e += p2 >= a.edges[k] ? 1 : 0;
        const int g = e * 8 + (px < 0.f ? 1 : 0) + (py < 0.f ? 2 : 0) + (pz < 0.f ? 4 : 0);
        a.grp[q] = (uint8_t)g;
        atomicAdd(&gcnt[wid][g], 1);
      }
    }
    __syncwarp();
    // the groups of three or more: a list, and each one's first member
    // position (exclusive prefix of their sizes)
    int nm = 0, run = 0;
    for (int g0 = 0; g0 < ngroups; g0 += 32) {
      const int g = g0 + lane;
      const int m = g < ngroups ? gcnt[wid][g] : 0;
      const bool listed = m >= 3;
      const int v = listed ? m : 0;
      int incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(kAll, incl, d);
        if (lane >= d) incl += t;
      }
      const unsigned bm = __ballot_sync(kAll, listed);
      if (listed) {
        gpos[wid][g] = run + incl - v;
        glist[wid][nm + __popc(bm & lt)] = (uint8_t)g;
      }
      nm += __popc(bm);
      run += __shfl_sync(kAll, incl, 31);
    }
    if (nm == 0) continue;
    __syncwarp();
    // members of listed groups in slot order: rank among the chunk's lanes
    // of the same group, after the group's members of earlier chunks
    for (int s0 = 0; s0 < n; s0 += 32) {
      const int slot = s0 + lane;
      const int g = slot < n ? a.grp[base + slot] : 0;
      const bool take = slot < n && gcnt[wid][g] >= 3;
      const unsigned peers = __match_any_sync(kAll, take ? g : kGroupsMax + lane);
      const int rank = __popc(peers & lt);
      const int p0 = take ? gpos[wid][g] : 0;
      __syncwarp();
      if (take) {
        mem[p0 + rank] = (uint16_t)slot;
        if (rank == 0) gpos[wid][g] = p0 + __popc(peers);
      }
      __syncwarp();
    }
    // a lane per listed group
    int removed = 0;
    for (int t = lane; t < nm; t += 32) {
      const int g = glist[wid][t];
      const int m = gcnt[wid][g];
      merge_group(a, base, mem + (gpos[wid][g] - m), m);
      removed += m - 2;
    }
    __syncwarp();
#pragma unroll
    for (int d = 16; d; d >>= 1) removed += __shfl_xor_sync(kAll, removed, d);
    // the tail fill: the freed slots below the new count ns take, in
    // ascending order, the kept slots at or beyond it, in ascending order
    const int ns = n - removed;
    for (int j0 = 0;; j0 += 32) {
      const int j = j0 + lane;
      int from = -1, to = -1, runTo = 0, runFrom = 0;
      for (int s0 = 0; s0 < n; s0 += 32) {
        const int slot = s0 + lane;
        const bool freed = slot < n && a.grp[base + slot] == kMergeFreed;
        const unsigned tm = __ballot_sync(kAll, freed && slot < ns);
        const unsigned fm = __ballot_sync(kAll, slot < n && slot >= ns && !freed);
        int k = j - runTo;
        if (k >= 0 && k < __popc(tm)) to = s0 + (int)__fns(tm, 0, k + 1);
        k = j - runFrom;
        if (k >= 0 && k < __popc(fm)) from = s0 + (int)__fns(fm, 0, k + 1);
        runTo += __popc(tm);
        runFrom += __popc(fm);
      }
      if (j < runTo && from >= 0 && to >= 0) {
        const long qf = base + from, qt = base + to;
        const float4 r = s.wp[qf], u = s.xyz[qf];
        s.wp[qt] = r;
        s.xyz[qt] = u;
      }
      if (j0 + 32 >= runTo) break;
    }
    if (lane == 0) {
      s.count[c] = ns;
      atomicAdd(a.removed, (double)removed);
    }
  }
}

}  // namespace

constexpr int kDynMax = 160 * 1024;  // the members' dynamic shared memory, at most

cudaError_t merge_init_kernels() {
  return cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynMax);
}

cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  if (a.s.cap > kMergeMaxCap) return cudaErrorInvalidValue;
  // warps per CTA: as many as fit the members' shared memory, at most 2
  const size_t per_warp = (size_t)std::max(a.s.cap, 1) * sizeof(uint16_t);
  const int nw = (int)std::max<size_t>(1, std::min<size_t>(kWarpsMax, kDynMax / per_warp));
  merge_kernel<<<(a.ncells + nw - 1) / nw, nw * 32, per_warp * nw, st>>>(a);
  return cudaGetLastError();
}

}  // namespace axpic
