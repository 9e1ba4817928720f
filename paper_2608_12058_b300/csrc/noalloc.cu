// cheb_expmv_noalloc: exp(-itH) psi for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or an
// allocator that forbids foreign allocations, plugins that are handed only the
// buffers they work on, and host programs that must not grow the device footprint
// after start-up. The regular entry points need a caller-supplied device workspace
// for the two Clenshaw vectors and the energy tables. This entry point instead uses
// one fixed scratch array that is part of the library image.
//
// The scratch is a file-scope __device__ array of kNoAllocBytes (10 MiB). Every GPU
// on which the library's device code is loaded holds it until the process exits.
// In host code the array's name is only a host-side stand-in, so the first call on
// each device (with that device current) looks up its device address with
// cudaGetSymbolAddress and caches it; that first call should come before any stream
// capture. The cache is keyed on the device's current context (its unique id), so a
// context reset (cudaDeviceReset, or a primary context released and retained again)
// makes the next call look the address up again instead of using a stale one. All calls share the one array and it keeps the last call's contents:
// the status word is cleared and the tables are rebuilt on every call, and the first
// Clenshaw step never reads the vector it overwrites. Calls that overlap on the GPU
// (different streams, or different host threads on one device) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cheb_expmv.h"
#include "cheb_internal.h"

namespace cheb {

cheb_status_t expmv_impl(int n, const double* h, const double* J, double gamma, double t, void* psi, int prec,
                         double tol, int method, int splits, int path, void* ws, size_t ws_bytes, void* stream,
                         cheb_info_t* info);

namespace {

constexpr size_t kNoAllocBytes = (size_t)10 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

std::mutex g_mu;
struct Cached {
    unsigned long long ctx_id = 0;  // context the address belongs to (0 = none yet)
    void* addr = nullptr;
};
Cached g_addr[kMaxDevices];

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the library
// does not link libcuda).
using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);

bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)p;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)p;
    }
    if (!get_current || !get_id) return false;
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0 && *id != 0;
}

// Device address of g_scratch in the current device's current context (looked up
// once per device and context).
cheb_status_t scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHEB_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CHEB_ERR_UNSUPPORTED;
    // make the device's primary context current (cudaSetDevice initialises it)
    if (cudaSetDevice(dev) != cudaSuccess) return CHEB_ERR_CUDA;
    unsigned long long id = 0;
    if (!current_context_id(&id)) return CHEB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev].ctx_id != id || !g_addr[dev].addr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CHEB_ERR_CUDA;
        g_addr[dev].addr = p;
        g_addr[dev].ctx_id = id;
    }
    *out = g_addr[dev].addr;
    return CHEB_OK;
}

}  // namespace
}  // namespace cheb

extern "C" cheb_status_t cheb_expmv_noalloc(int n, const double* h, const double* J, double gamma, double t,
                                            void* psi, cheb_precision_t precision, double tol,
                                            cheb_method_t method, int time_splits, void* stream,
                                            cheb_info_t* info) {
    using namespace cheb;
    if (n < 1 || n > kMaxQubits) return CHEB_ERR_INVALID_ARG;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (make_layout(n, precision).total > kNoAllocBytes) return CHEB_ERR_UNSUPPORTED;
    void* ws = nullptr;
    cheb_status_t st = scratch_address(&ws);
    if (st != CHEB_OK) return st;
    return expmv_impl(n, h, J, gamma, t, psi, precision, tol, method, time_splits, CHEB_PATH_AUTO, ws,
                      kNoAllocBytes, stream, info);
}
