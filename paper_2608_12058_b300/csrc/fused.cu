// Fused FP32 Clenshaw step (placeholder until the tiled kernels land).
#include "fused.cuh"

namespace cheb {

size_t fused_scratch_bytes(int, int) { return 0; }
bool fused_supported(int, int) { return false; }
FusedPlan fused_plan(int n, int prec) {
    FusedPlan p;
    p.n = n;
    p.prec = prec;
    return p;
}
cudaError_t launch_step_fused(const FusedPlan&, const StepArgs&, void*, int*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace cheb
