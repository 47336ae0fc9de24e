// Launch interface of the step kernels (internal to libaxpic).
#pragma once
#include "common.cuh"
#include "sr.h"

namespace axpic {

enum { PH_ABSORB = 1, PH_EMIT = 2, PH_FEEDBACK = 4, PH_ALL = 7 };

size_t step_smem_per_warp(int acap, int gcap, int ecap);
// ev: NULL, or kStepKernels + 1 events recorded around the kernels of a
// PH_ALL step: decisions, events, feedback, and the rate model's record
// kernel (an empty interval when there is none). sra: the record kernels'
// arguments (rate models 1 and 2), else NULL.
cudaError_t launch_step(int phases, const StepArgs& A, int warps, cudaStream_t st, cudaEvent_t* ev = nullptr,
                        const SrArgs* sra = nullptr);
constexpr int kStepKernels = 4;
// Comma-separated names of the kernels a PH_ALL step launches, in order.
const char* step_kernel_names(int rate_model, int T_mode);
// CTAs of the kernel fn (threads a CTA, dyn_smem bytes of dynamic shared
// memory) that the current device holds at once: the SMs times what one SM
// holds by registers, shared memory (static, dynamic and the driver's
// reservation a CTA), threads and CTA slots, at most max_per_sm. 0 if a
// query fails. (On a GB300 the runtime's occupancy query gave 1 CTA an SM
// for a tensor-memory kernel that the SM holds 7 of.)
int resident_ctas(const void* fn, int threads, size_t dyn_smem, int max_per_sm = 32);
// Raises (never lowers) the event kernels' dynamic shared-memory limit on the
// current device to at least `bytes`.
cudaError_t set_step_smem_limits(size_t bytes);
// CTAs of the decision kernel (chunk of 4, 8, 16 or 32 cells) that the current
// device holds at once.
cudaError_t decide_resident_ctas(int chunk, int* out);
// The decision kernel's cells per chunk (requested, or 0 for the default:
// the largest of 32, 16 and 8 that still gives every resident decision warp
// a chunk of the ncells, else 4) and its persistent grid.
cudaError_t decide_shape(int requested, int ncells, int* chunk, int* grid);
constexpr int kDefaultDecChunk = AXPIC_DEC_CHUNK;
// Writes v to the n device step counters p[0, n) (one thread).
cudaError_t launch_set_step(uint32_t* p, uint32_t v, int n, cudaStream_t st);

}  // namespace axpic
