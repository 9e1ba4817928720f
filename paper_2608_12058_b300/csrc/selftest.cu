// Failure-detection self-test of both kinds of bounded wait, each with a short limit on a
// wait that nothing satisfies: an mbarrier that nothing arrives on (the wait of the TMA
// kernels) and a team barrier whose teammate never comes (the wait of the persistent
// batch kernel). Each gives up, records kFlagTimeout in its status word and lets the
// kernel return, so the host sees CHEB_ERR_TIMEOUT and the context stays usable. No
// fault, trap or hang.
#include <cuda_runtime.h>

#include "cheb_internal.h"
#include "kernels.cuh"
#include "mbar.cuh"
#include "pipeline.h"
#include "batch_team.cuh"

namespace cheb {
namespace {

__global__ void k_wait_selftest(int* flags, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // expects one arrival, which never comes
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, flags, (volatile int*)&abort_flag, limit);
    __syncthreads();
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" cheb_status_t cheb_wait_selftest(void* workspace, size_t workspace_bytes, void* stream) {
    if (!workspace || workspace_bytes < 4 * sizeof(int) || ((uintptr_t)workspace & 3)) return CHEB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int* flags = (int*)workspace;  // [0]: mbarrier wait, [1]: team barrier, [2]: its counter
    CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    note_launch(kKindReduce);
    k_wait_selftest<<<1, 32, 0, s>>>(flags, 2000000LL);  // ~1 ms at 2 GHz
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(launch_team_barrier_selftest((unsigned*)(flags + 2), flags + 1, 2000000LL, s));
    int f[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(f, flags, sizeof(f), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ((f[0] & kFlagTimeout) && (f[1] & kFlagTimeout)) ? CHEB_ERR_TIMEOUT : CHEB_OK;
}
