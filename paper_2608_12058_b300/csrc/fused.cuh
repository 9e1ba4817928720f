// Fused shared-memory Clenshaw step for the FP32 path (fused.cu).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cstddef>

#include "kernels.cuh"

namespace cheb {

// How the n bit flips of one step are split between passes over memory:
//   low pass:      bits [0, M) from the shared-memory tile, bits [M, M + l) from
//                  partner tiles that TMA fetches from L2;
//   strided passes: the remaining h = n - M - l bits, in npass ranges of 3..9 bits
//                  each, [lo[k], lo[k] + hb[k]), each from a strided shared-memory
//                  tile of 2^hb rows of 16 amplitudes.
struct FusedPlan {
    int n = 0;
    int prec = 0;
    int M = 0;
    int l = 0;
    int h = 0;
    int npass = 0;
    int lo[4] = {0, 0, 0, 0};
    int hb[4] = {0, 0, 0, 0};
};

size_t fused_scratch_bytes(int n, int prec);
// Number of SMs of the current device (cached).
int num_sms();
// L2-blocked launches: 0 off, 1 the step tail (the last strided pass and the low pass in
// one launch), 2 the strided pair (both strided passes of a two-pass plan in one launch),
// -1 automatic (the pair from n = 26 on for FP32, from n = 28 on for the float-float path).
void fused_set_blocking(int mode);
int fused_get_blocking();
// Choices of the autotuner: per (prec, n) the AUTO path (-1 = built-in rule) and, for
// FP32, the blocked tail (-1 = the process-wide switch).
void tuned_set(int prec, int n, int path, int blocking);
// The L2-blocked mode for (prec, n): the autotuner's choice, else the process-wide switch
// (the blocked tail, mode 1, is FP32 only).
int fused_blocking_for(int prec, int n);
// Lag of the blocked pair in groups for groups of `group_bytes` (b_{k+1} and q).
int pair_lag(size_t group_bytes);
int tuned_auto_path(int prec, int n);
bool fused_blocking_eligible(const FusedPlan& plan);
// The blocked strided pair applies (two strided passes of 6..9 bits, FP32).
bool fused_pair_eligible(const FusedPlan& plan);
// Kahan-compensated flip sums in the fused FP32 passes: on/off (process-wide).
void fused_set_compensated(int on);
int fused_get_compensated();
bool fused_split_valid(int n, int l, int h);
// Override the split for n (l < 0 restores the default); false if invalid.
bool fused_set_split(int n, int l, int h);
bool fused_supported(int n, int prec);
FusedPlan fused_plan(int n, int prec);
// cuTensorMapEncodeTiled through the runtime's driver entry point (null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
cudaError_t launch_step_fused(const FusedPlan& plan, const StepArgs& a, void* scratch, int* flags,
                              cudaStream_t s);

}  // namespace cheb
