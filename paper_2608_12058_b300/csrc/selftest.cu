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
#include "pair.cuh"

#include <vector>

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

// The blocked pair's work order (pairk::decode), checked on the host: the items
// 0 .. G (NA + NB) - 1 are every A-tile and every B-tile of the G groups exactly once,
// the next index is the end marker, and every B-tile of a group comes after all of that
// group's A-tiles (so an item only waits on items taken before it).
extern "C" int cheb_pair_schedule_check(int gbits, int HA, int HB, int lag, long long* min_gap) {
    if (gbits < 0 || gbits > 16 || HA < 1 || HA > 9 || HB < 1 || HB > 9 || lag < 1 || lag > (1 << gbits))
        return -1;
    const long long G = 1LL << gbits, NA = 1LL << HB, NB = 1LL << HA;
    const unsigned long long total = (unsigned long long)(G * (NA + NB));
    std::vector<unsigned char> seen_a((size_t)(G * NA), 0), seen_b((size_t)(G * NB), 0);
    std::vector<long long> last_a((size_t)G, -1), first_b((size_t)G, -1);
    for (unsigned long long i = 0; i < total; ++i) {
        const pairk::Item it = pairk::decode(i, gbits, HA, HB, lag);
        if (it.g < 0 || it.g >= G) return 1;
        if (it.kind == pairk::kItemA) {
            if (it.idx < 0 || it.idx >= NA) return 1;
            unsigned char& f = seen_a[(size_t)(it.g * NA + it.idx)];
            if (f) return 2;
            f = 1;
            last_a[(size_t)it.g] = (long long)i;
        } else if (it.kind == pairk::kItemB) {
            if (it.idx < 0 || it.idx >= NB) return 1;
            unsigned char& f = seen_b[(size_t)(it.g * NB + it.idx)];
            if (f) return 2;
            f = 1;
            if (first_b[(size_t)it.g] < 0) first_b[(size_t)it.g] = (long long)i;
        } else {
            return 5;  // the end marker before the last item
        }
    }
    if (pairk::decode(total, gbits, HA, HB, lag).kind != pairk::kItemEnd) return 5;
    long long gap = -1;
    for (long long g = 0; g < G; ++g) {
        if (last_a[(size_t)g] < 0 || first_b[(size_t)g] < 0) return 3;
        const long long d = first_b[(size_t)g] - last_a[(size_t)g];
        if (d <= 0) return 4;
        if (gap < 0 || d < gap) gap = d;
    }
    for (unsigned char f : seen_a)
        if (!f) return 3;
    for (unsigned char f : seen_b)
        if (!f) return 3;
    if (min_gap) *min_gap = gap;
    return 0;
}
