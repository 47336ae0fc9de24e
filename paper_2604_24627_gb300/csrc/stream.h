// Axion free streaming and cell migration (internal to libaxpic).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace axpic {

// Direction of a slot after a move: the cell shift (sx, sy, sz) in {-1, 0, 1}^3
// as (sz + 1) 9 + (sy + 1) 3 + (sx + 1); 13 stays; 27 left an open box.
constexpr int kStreamDirs = 27, kStreamStay = 13, kStreamEscaped = 27;

struct StreamArgs {
  SpeciesPtrs s;       // the axion slabs (positions rewritten, slots re-binned)
  int ncells, nx, ny, nz;
  float kappa;         // binary32(c dt / h): the cell fraction moved at |v| = c
  float mu;            // binary32(m_a c^2 / m_e c^2): the axion mass in units of the momenta
  int periodic;        // 1 periodic, 0 open
  uint8_t* dir;        // [ncells * cap]: direction of each slot
  int32_t* cnt;        // [ncells * 27]: slots per direction
  int32_t* goff;       // [ncells * 27]: the direction's first row in the cell's staging rows
  float* buf;          // [ncells * cap * 8]: the cell's leaving axions, grouped by direction
  double* stats;       // [4]: escaped number, weight, weight x energy [keV]; dropped number
  int* err;            // latched error flags (ERR_CAPACITY)
};

cudaError_t launch_stream(const StreamArgs& a, cudaStream_t st);

}  // namespace axpic
