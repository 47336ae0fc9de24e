// Launch interface of the step kernels (internal to libaxpic).
#pragma once
#include "common.cuh"
#include "sr.h"

namespace axpic {

enum { PH_ABSORB = 1, PH_EMIT = 2, PH_FEEDBACK = 4, PH_ALL = 7 };

size_t step_smem_per_warp(int acap, int gcap, int ecap);
// ev: NULL, or kStepKernels + 1 events recorded around the kernels of a
// PH_ALL step (the third interval covers the feedback kernel and, with a rate
// model, the records' rebuild). sra: the record kernels' arguments (rate
// models 1 and 2), else NULL.
cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st, cudaEvent_t* ev = nullptr,
                        const SrArgs* sra = nullptr);
constexpr int kStepKernels = 3;
// Comma-separated names of the kernels a PH_ALL step launches, in order.
const char* step_kernel_names();
// Raises (never lowers) the event kernels' dynamic shared-memory limit on the
// current device to at least `bytes`.
cudaError_t set_step_smem_limits(size_t bytes);
// CTAs of the decision kernel (chunk of 2, 4 or 8 cells) that the current
// device holds at once.
cudaError_t decide_resident_ctas(int chunk, int* out);
constexpr int kDefaultDecChunk = AXPIC_DEC_CHUNK;
// Writes v to the n device step counters p[0, n) (one thread).
cudaError_t launch_set_step(uint32_t* p, uint32_t v, int n, cudaStream_t st);

}  // namespace axpic
