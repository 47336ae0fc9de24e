// Axion merging for population control (internal to libaxpic).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace axpic {

constexpr int kMergeMaxEdges = 30;  // |p|^2 thresholds: (30 + 1) bins x 8 octants = 248 groups
constexpr int kMergeFreed = 255;    // group byte of a freed slot
constexpr int kMergeMaxCap = 65535; // slots per cell, u16 member indices (slabs hold at most 65532)

struct MergeArgs {
  SpeciesPtrs s;     // the axion slabs
  int ncells;
  int n_target;      // cells holding more axions than this are merged
  int nedges;
  float edges[kMergeMaxEdges];  // ascending binary32 thresholds of |p|^2 (m_e c)^2
  uint8_t* grp;      // [ncells * cap]: each slot's group during the call
  double* removed;   // [1]: axions removed so far
};

// Sets the merge kernel's shared-memory limit; called before its first launch.
cudaError_t merge_init_kernels();
cudaError_t launch_merge(const MergeArgs& a, cudaStream_t st);

}  // namespace axpic
