// Axion free streaming and cell migration: x += (p / E) c dt with E =
// sqrt(p^2 + m_a^2) (Sec. II.B: massless axions at c, massive ones
// sub-luminal; the transport of the axion macroparticles between steps) on
// the cell-sorted slabs, positions being fractions of the cell.
//
// Two kernels, a warp per cell each (grid-stride):
//  * stream_move_kernel moves every axion of its cell, in binary32 with each
//    rounding fixed (the result decides the destination cell), writes the
//    new position in place, the direction of each slot and the count per
//    direction, and copies the leaving axions into the cell's staging rows,
//    grouped by direction in slot order.
//  * stream_place_kernel takes the arrivals from its neighbours' staging
//    rows, ordered by the neighbour's position relative to it, (dz, dy, dx)
//    ascending, then by source slot, into the slots its own leavers freed
//    (ascending), then after the old count; freed slots left over are closed
//    by the tail fill. Staying axions keep their slots unless the tail fill
//    moves them. Slots beyond the capacity are dropped, counted, and latch
//    ERR_CAPACITY.
// The first kernel writes only its own cell's slots and rows; the second
// reads the neighbours' rows and writes only its own slab, so neither needs
// a barrier across cells.
#include "stream.h"

namespace axpic {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr float kBelowOne = 0x1.fffffep-1f;

// New fraction of one position component and the cell shift in {-1, 0, 1}:
// t = q + d, s = floor(t), t - s (the largest binary32 below 1 where that
// rounds up to 1).
__device__ __forceinline__ float advance(float q, float d, int* shift) {
  const float t = __fadd_rn(q, d);
  const float s = floorf(t);
  float r = __fsub_rn(t, s);
  if (r >= 1.0f) r = kBelowOne;
  // in {-1, 0, 1} for positions in [0, 1) and kappa < 1; clamped so that no
  // input can index beyond the 27 directions
  *shift = max(-1, min(1, (int)s));
  return r;
}

__global__ void __launch_bounds__(kThreads) stream_move_kernel(StreamArgs a) {
  __shared__ int cnt[kWarps][32];
  __shared__ int run[kWarps][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = blockIdx.x * kWarps + wid; c < a.ncells; c += gridDim.x * kWarps) {
    cnt[wid][lane] = 0;
    run[wid][lane] = 0;
    __syncwarp();
    const int n = min(max(a.s.count[c], 0), a.s.cap);
    const long base = (long)c * a.s.cap;
    const int ci = c % a.nx, cj = (c / a.nx) % a.ny, ck = c / (a.nx * a.ny);
    // two chunks of 32 slots per pass: both chunks' loads are issued before
    // either is stored
    for (int s0 = 0; s0 < n; s0 += 64) {
      float w[2], px[2], py[2], pz[2], x[2], y[2], z[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int slot = s0 + 32 * hh + lane;
        w[hh] = px[hh] = py[hh] = pz[hh] = x[hh] = y[hh] = z[hh] = 0.f;
        if (slot < n) {
          const long q = base + slot;
          const float4 r = a.s.wp[q], u = a.s.xyz[q];
          w[hh] = r.x, px[hh] = r.y, py[hh] = r.z, pz[hh] = r.w;
          x[hh] = u.x, y[hh] = u.y, z[hh] = u.z;
        }
      }
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int slot = s0 + 32 * hh + lane;
        if (slot >= n) continue;
        const long q = base + slot;
        // E = sqrt(p^2 + mu^2): v = p / E in units of c
        const float en = __fsqrt_rn(__fadd_rn(
            __fadd_rn(__fadd_rn(__fmul_rn(px[hh], px[hh]), __fmul_rn(py[hh], py[hh])), __fmul_rn(pz[hh], pz[hh])),
            __fmul_rn(a.mu, a.mu)));
        int sx = 0, sy = 0, sz = 0;
        if (en > 0.f) {
          const float k = __fdiv_rn(a.kappa, en);
          float4 u = make_float4(x[hh], y[hh], z[hh], 0.f);
          if (a.nx > 1) u.x = advance(x[hh], __fmul_rn(k, px[hh]), &sx);
          if (a.ny > 1) u.y = advance(y[hh], __fmul_rn(k, py[hh]), &sy);
          if (a.nz > 1) u.z = advance(z[hh], __fmul_rn(k, pz[hh]), &sz);
          a.s.xyz[q] = u;
        }
        int o = (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1);
        if (!a.periodic) {
          const int ii = ci + sx, jj = cj + sy, kk = ck + sz;
          if (ii < 0 || ii >= a.nx || jj < 0 || jj >= a.ny || kk < 0 || kk >= a.nz) {
            o = kStreamEscaped;
            const double wd = (double)w[hh];
            const double pm = sqrt((double)px[hh] * px[hh] + (double)py[hh] * py[hh] + (double)pz[hh] * pz[hh] +
                                   (double)a.mu * a.mu);
            atomicAdd(a.stats + 0, 1.0);
            atomicAdd(a.stats + 1, wd);
            atomicAdd(a.stats + 2, wd * pm * kMeC2);
          }
        }
        a.dir[q] = (uint8_t)o;
        atomicAdd(&cnt[wid][o], 1);
      }
    }
    __syncwarp();
    if (lane < kStreamDirs) a.cnt[(size_t)c * kStreamDirs + lane] = cnt[wid][lane];
    // staging offset of each direction's group: the leavers of the lower
    // directions (13 stays and 27 escaped hold none)
    const int v = (lane < kStreamDirs && lane != kStreamStay) ? cnt[wid][lane] : 0;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(kAll, incl, d);
      if (lane >= d) incl += t;
    }
    const int off = incl - v;
    if (lane < kStreamDirs) a.goff[(size_t)c * kStreamDirs + lane] = off;
    for (int s0 = 0; s0 < n; s0 += 32) {
      const int slot = s0 + lane;
      const int o = slot < n ? (int)a.dir[base + slot] : 31;
      const bool leave = o < kStreamDirs && o != kStreamStay;
      const unsigned m = __match_any_sync(kAll, o);
      const int goff = __shfl_sync(kAll, off, o);
      if (leave) {
        const int pos = goff + run[wid][o] + __popc(m & lt);
        const long q = base + slot;
        float4* dst = reinterpret_cast<float4*>(a.buf + ((size_t)c * a.s.cap + pos) * 8);
        dst[0] = a.s.wp[q];
        dst[1] = a.s.xyz[q];
      }
      __syncwarp();
      if (leave && (m & lt) == 0) run[wid][o] += __popc(m);  // the group's first lane
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kThreads) stream_place_kernel(StreamArgs a) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const SpeciesPtrs& s = a.s;
  for (int c = blockIdx.x * kWarps + wid; c < a.ncells; c += gridDim.x * kWarps) {
    const int n = min(max(s.count[c], 0), s.cap);
    const long base = (long)c * s.cap;
    const int ci = c % a.nx, cj = (c / a.nx) % a.ny, ck = c / (a.nx * a.ny);
    // freed slots: every slot of the cell that did not stay
    const int H = n - a.cnt[(size_t)c * kStreamDirs + kStreamStay];
    // arrivals: lane r (r < 27, r != 13) takes the neighbour at (dz, dy, dx)
    // = r's digits - 1, lanes ascending in r; that neighbour's axions that
    // moved here have the shift -(dz, dy, dx), direction 26 - r. Every
    // lane's group is found at once; a scan orders the groups by r.
    int m = 0, src = 0, g = 0;
    if (lane < kStreamDirs && lane != kStreamStay) {
      const int r = lane;
      const int dz = r / 9 - 1, dy = (r / 3) % 3 - 1, dx = r % 3 - 1;
      int si = ci + dx, sj = cj + dy, sk = ck + dz;
      bool ok = !((dx && a.nx == 1) || (dy && a.ny == 1) || (dz && a.nz == 1));
      if (a.periodic) {
        si = (si + a.nx) % a.nx;
        sj = (sj + a.ny) % a.ny;
        sk = (sk + a.nz) % a.nz;
      } else if (si < 0 || si >= a.nx || sj < 0 || sj >= a.ny || sk < 0 || sk >= a.nz) {
        ok = false;
      }
      if (ok) {
        src = (sk * a.ny + sj) * a.nx + si;
        const size_t k = (size_t)src * kStreamDirs + (kStreamDirs - 1 - r);
        m = a.cnt[k];
        g = a.goff[k];
      }
    }
    int incl = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(kAll, incl, d);
      if (lane >= d) incl += t;
    }
    const int A = __shfl_sync(kAll, incl, 31);
    const int excl = incl - m;
    // arrival t takes freed slot t (ascending) while there are any, then
    // slot n + (t - H)
    for (int t0 = 0; t0 < A; t0 += 32) {
      const int t = t0 + lane;
      int sel = 0;
#pragma unroll
      for (int r = 1; r < kStreamDirs; ++r) {
        const int e = __shfl_sync(kAll, excl, r), mr = __shfl_sync(kAll, m, r);
        if (mr > 0 && e <= t) sel = r;
      }
      const int e = __shfl_sync(kAll, excl, sel);
      const int gs = __shfl_sync(kAll, g, sel), ss = __shfl_sync(kAll, src, sel);
      int dst = n + (t - H);
      const int need = min(t0 + 32, H);  // freed slots of this pass: indices t0 .. need - 1
      if (t0 < need) {
        int run = 0;
        for (int s0 = 0; s0 < n && run < need; s0 += 32) {
          const int slot = s0 + lane;
          const unsigned hm = __ballot_sync(kAll, slot < n && a.dir[base + slot] != kStreamStay);
          const int k = t - run;
          if (t < H && k >= 0 && k < __popc(hm)) dst = s0 + (int)__fns(hm, 0, k + 1);
          run += __popc(hm);
        }
      }
      if (t < A && dst < s.cap) {
        const float* row = a.buf + ((size_t)ss * s.cap + gs + (t - e)) * 8;
        const float4 u0 = reinterpret_cast<const float4*>(row)[0];
        const float4 u1 = reinterpret_cast<const float4*>(row)[1];
        const long q = base + dst;
        s.wp[q] = u0;
        s.xyz[q] = u1;
      }
    }
    __syncwarp();
    // fewer arrivals than freed slots: the freed slots left over (indices A
    // .. H - 1) below the new count ns take, in ascending order, the kept
    // slots at or beyond ns (stayers and filled slots), in ascending order
    if (A < H) {
      const int ns = n - (H - A);
      for (int j0 = 0;; j0 += 32) {
        const int j = j0 + lane;
        int from = -1, to = -1, runH = 0, runTo = 0, runFrom = 0;
        for (int s0 = 0; s0 < n; s0 += 32) {
          const int slot = s0 + lane;
          const bool freed = slot < n && a.dir[base + slot] != kStreamStay;
          const unsigned hm = __ballot_sync(kAll, freed);
          const bool left = freed && runH + __popc(hm & lt) >= A;  // freed and not filled
          const unsigned tm = __ballot_sync(kAll, left && slot < ns);
          const unsigned fm = __ballot_sync(kAll, slot < n && slot >= ns && !left);
          int k = j - runTo;
          if (k >= 0 && k < __popc(tm)) to = s0 + (int)__fns(tm, 0, k + 1);
          k = j - runFrom;
          if (k >= 0 && k < __popc(fm)) from = s0 + (int)__fns(fm, 0, k + 1);
          runH += __popc(hm);
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
    }
    const int total = n - H + A;
    if (lane == 0) {
      s.count[c] = min(total, s.cap);
      if (total > s.cap) {
        atomicAdd(a.stats + 3, (double)(total - s.cap));
        atomicOr(a.err, ERR_CAPACITY);
      }
    }
  }
}

}  // namespace

cudaError_t launch_stream(const StreamArgs& a, cudaStream_t st) {
  if (a.ncells <= 0) return cudaSuccess;
  const int grid = (a.ncells + kWarps - 1) / kWarps;
  stream_move_kernel<<<grid, kThreads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  stream_place_kernel<<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace axpic
