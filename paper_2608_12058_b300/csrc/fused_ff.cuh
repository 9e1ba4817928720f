// Fused float-float Clenshaw step of the FP64 path (fused_ff.cu).
#pragma once
#include <cuda_runtime.h>

#include "fused.cuh"
#include "kernels.cuh"

namespace cheb {

// Smallest n for the float-float fused step (the energy tables have 11-bit tiles).
constexpr int kFFMinQubits = 11;

// Split of the n bit flips of one float-float step: bits [0, 10) from the shared-memory
// tile, [10, 10 + l) from L2 partner tiles, the remaining h bits in strided passes.
bool ff_supported(int n);
bool ff_split_valid(int n, int l, int h);
bool ff_set_split(int n, int l, int h);  // l < 0 restores the default
FusedPlan ff_plan(int n);
// psi (complex128) -> float-float vector, in place.
cudaError_t launch_to_ff(int64_t N, void* psi, cudaStream_t s);
// dst = (cr + i ci) src, both float-float vectors.
cudaError_t launch_ff_scale(int64_t N, const void* src, void* dst, double cr, double ci, cudaStream_t s);
// One Clenshaw step on float-float vectors b1, b2, psi; out is float-float, or complex128
// when out_f64 (the final step).
// scratch (nullable): the fused scratch of the workspace (counters of the blocked pair).
cudaError_t launch_step_ff(const FusedPlan& plan, const StepArgs& a, void* scratch, int* flags, bool out_f64,
                           cudaStream_t s);
// The blocked strided pair applies to the float-float step (two strided passes of 6..9 bits).
bool ff_pair_eligible(const FusedPlan& plan);

}  // namespace cheb
