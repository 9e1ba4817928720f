// Launchers for the device kernels (kernels.cu, fused.cu). All launches are
// asynchronous on the given stream; none of them allocates memory.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <utility>

namespace cheb {

// Kernel kinds for launch counting and event timing (cheb_kernel_kind_t).
enum KernelKind : int {
    kKindTables = 0,
    kKindMinmax = 1,
    kKindScale = 2,
    kKindStepPlain = 3,
    kKindSmall = 4,
    kKindReduce = 5,
    kKindLow = 6,
    kKindHigh = 7,
    kKindMixed = 8,
    kKindPair = 9,
};
void note_launch(int kind);
// count kernels that run as part of a CUDA graph replay; whether event timing is on
void note_launches(long long count);
bool prof_enabled();
// Whether step kernels are launched with programmatic dependent launch (on by default;
// off while event profiling is on, so that per-kernel event times do not overlap).
bool pdl_enabled();
void pdl_set(bool on);
// Event-bracketed timing of one launch when profiling is on (prof_begin returns -1 otherwise).
int prof_begin(int kind, cudaStream_t s);
void prof_end(int idx, cudaStream_t s);

// Arguments of one Clenshaw step (Eq. recursion, Algorithm 2):
//   out = scale * (Dt .* b1 + g * sum_j X_j b1) + sgn * b2 + ck * psi,
// with Dt(z) = (E(z) - c) / r reconstructed from the fixed-point tables and
// g = gamma / r. scale = 2 for the inner steps and 1 for the final step;
// sgn = -1 normally and 0 when b_{k+2} is the zero vector. `out` may alias b2
// (in-place update) or psi (final step), never b1; when it is a buffer of its own,
// b2 and psi are left unchanged.
struct StepArgs {
    int n;
    int M;              // tile bits of the energy tables
    int Q;              // fixed-point scale: value = int * 2^-Q
    const int64_t* tiles;
    const int64_t* elow;
    const int64_t* jq;  // fixed-point couplings: J symmetric n*n, h[n], c
    const void* b1;
    const void* b2;
    const void* psi;
    void* out;
    double ck_re, ck_im;
    double scale;
    double sgn;
    double g;           // gamma / r (the FP32 kernels split it into hi + lo)
};

void launch_tables(int n, int M, const int64_t* jq, int64_t* tiles, int64_t* elow, cudaStream_t s);
void launch_minmax(int n, int M, const int64_t* tiles, const int64_t* elow, int64_t* part,
                   int64_t* out2, cudaStream_t s);
void launch_scale(int prec, int64_t N, const void* src, void* dst, double cr, double ci,
                  cudaStream_t s);
void launch_step_plain(int prec, const StepArgs& a, cudaStream_t s);
// Whole Clenshaw run for n <= kSmallMax*: one CTA keeps psi, b1, b2 in shared memory.
cudaError_t launch_small(int prec, int n, int K, const double* coef_dev, int Q,
                         const int64_t* tiles, const int64_t* elow, double g, void* psi,
                         cudaStream_t s);
// One small instance of a batch (whole run in one CTA's shared memory).
struct SmallDesc {
    int n;
    int K;                 // degree; K <= 0 skips the instance
    int Q;                 // fixed-point scale of its tables
    int pad;
    double g;              // gamma / r
    const double* coef;    // (K+1) complex doubles, device
    const int64_t* tiles;  // its energy tables
    const int64_t* elow;
    void* psi;             // its state, in/out
};
cudaError_t launch_small_batched(int prec, int count, int max_n, const SmallDesc* descs, cudaStream_t s);
// Whole runs of instances of one size n on thread-block clusters (cluster.cu): one
// cluster of 2^(n - SB) CTAs per instance, SB = cluster_slice_bits(prec), n - SB in
// 1..4. Returns cudaErrorNotSupported when no such cluster fits on the device.
int cluster_slice_bits(int prec);
cudaError_t launch_cluster_batched(int prec, int n, int count, const SmallDesc* descs, cudaStream_t s);
// Evaluation-bound norms (Sec. II.B.3): *out_b += ||b||^2 and, if want_c,
// *out_c += ||(cr + i ci) psi - b||^2, both FP64 (atomic adds; zero them first).
// prec: 0 complex64, 1 complex128, kFormatFF float-float vectors.
void launch_step_norms(int prec, int64_t N, const void* b, const void* psi, double cr, double ci, int want_c,
                       double* out_b, double* out_c, cudaStream_t s);
void launch_norm_energy(int prec, int n, int M, int Q, const int64_t* tiles, const int64_t* elow,
                        double c, double r, const void* psi, double* part, double* out2,
                        cudaStream_t s);

// Launches kern<<<grid, block, smem, s>>>(args...) with programmatic stream serialization
// when pdl_enabled(), else as an ordinary launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_step_kernel(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                               Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace cheb
