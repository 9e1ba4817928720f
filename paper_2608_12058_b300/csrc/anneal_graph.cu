// A piecewise-constant schedule (the segments of cheb_anneal_general, Sec. III.B)
// captured once into a CUDA graph and replayed: every host-side step (spectral scan,
// fixed-point couplings, series and degrees) runs at capture; a replay is the device
// work alone. Per segment the graph copies that segment's fixed-point couplings from
// the graph's own store into the working tables, rebuilds the tables on the device and
// runs the segment's Clenshaw steps on the same kernels (and launch attributes) as
// cheb_anneal_general, so a replay gives the same state bit for bit.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "kernels.cuh"
#include "pipeline.h"

using namespace cheb;

struct cheb_anneal_graph {
    cudaGraphExec_t exec = nullptr;
    int device = -1;
    long long kernels = 0;  // library kernels per replay (for cheb_launch_count)
};

namespace {

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

size_t jq_bytes(int n) { return ((size_t)n * n + n + 1) * sizeof(int64_t); }

// Per segment the store keeps the fixed-point couplings and, where the whole run is one
// kernel that reads its coefficients from device memory (n <= 13 FP32, 12 FP64), the
// coefficients of one time slice (at most kMaxK + 1).
size_t seg_bytes(int n, int prec) {
    const bool small = n <= (prec == CHEB_FP32 ? kSmallMaxF32 : kSmallMaxF64);
    return a256(jq_bytes(n)) + (small ? a256((size_t)(kMaxK + 1) * 2 * sizeof(double)) : 0);
}

struct Seg {
    FixedOp F;
    std::vector<std::complex<double>> coef;
    int slices = 1;
    double g = 0.0;
};

// Ends a capture that failed part way, drops its graph and the capture stream.
cheb_status_t abandon(cudaStream_t s, cheb_status_t st) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(s);
    cudaGetLastError();
    return st == CHEB_OK ? CHEB_ERR_CUDA : st;
}

}  // namespace

extern "C" size_t cheb_anneal_graph_workspace_bytes(int n, cheb_precision_t precision, int S) {
    if (n < 1 || n > kMaxQubits || S < 1) return 0;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return 0;
    return a256(make_layout(n, precision).total) + (size_t)S * seg_bytes(n, precision);
}

extern "C" cheb_status_t cheb_anneal_graph_create(int n, const double* h, const double* J, int S, const double* a_s,
                                                  const double* b_s, const double* t_s, void* psi,
                                                  cheb_precision_t precision, double tol, cheb_method_t method,
                                                  void* boundaries, void* workspace, size_t ws_bytes, void* stream,
                                                  cheb_anneal_graph_t* graph) {
    if (!graph) return CHEB_ERR_INVALID_ARG;
    *graph = nullptr;
    cheb_status_t st = check_common(n, h, J, precision, workspace, ws_bytes);
    if (st != CHEB_OK) return st;
    if (S < 1 || !a_s || !t_s || !psi || ((uintptr_t)psi & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (boundaries && ((uintptr_t)boundaries & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(a_s, S) || !finite_all(t_s, S) || (b_s && !finite_all(b_s, S)) || !(tol > 0) ||
        !std::isfinite(tol))
        return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    if (ws_bytes < cheb_anneal_graph_workspace_bytes(n, precision, S)) return CHEB_ERR_WORKSPACE;
    // per-kernel event timing records host-side events at launch time, which a replay
    // would not renew
    if (prof_enabled()) return CHEB_ERR_UNSUPPORTED;
    cudaStream_t s0 = (cudaStream_t)stream;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, s0};
    unsigned char* store = C.ws + a256(C.L.total);
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
    double emin = 0, emax = 0;
    st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    // host side of every segment, as cheb_anneal_general does it
    const double tol_s = tol / S;
    std::vector<Seg> segs(S);
    std::vector<double> hb(n), Jb((size_t)n * n);
    for (int s = 0; s < S; ++s) {
        const double b = b_s ? b_s[s] : 1.0;
        const double c = b * 0.5 * (emax + emin);
        double r = std::fabs(b) * 0.5 * (emax - emin) + std::fabs(a_s[s]) * n;
        if (!(r > 0)) r = 1.0;
        for (int i = 0; i < n; ++i) hb[i] = b * h[i];
        for (size_t q = 0; q < (size_t)n * n; ++q) Jb[q] = b * J[q];
        Seg& G = segs[s];
        G.F = make_fixed(n, hb.data(), Jb.data(), c, r, precision == CHEB_FP32 ? kMaxQF32 : 62);
        if (G.F.Q < 24) return CHEB_ERR_UNSUPPORTED;
        int K = -1;
        double err = 0.0;
        st = slice_coefficients(t_s[s], c, r, tol_s, method, 0, G.coef, &K, &G.slices, &err);
        if (st != CHEB_OK) return st;
        G.g = a_s[s] / r;
        unsigned char* seg = store + (size_t)s * seg_bytes(n, precision);
        CUDA_TRY(cudaMemcpyAsync(seg, G.F.jq.data(), jq_bytes(n), cudaMemcpyHostToDevice, s0));
        if (seg_bytes(n, precision) > a256(jq_bytes(n)))
            CUDA_TRY(cudaMemcpyAsync(seg + a256(jq_bytes(n)), G.coef.data(),
                                     G.coef.size() * sizeof(std::complex<double>), cudaMemcpyHostToDevice, s0));
    }
    CUDA_TRY(cudaStreamSynchronize(s0));  // the host copies above are done before capture
    st = read_flags(C);
    if (st != CHEB_OK) return st;
    const size_t vbytes = ((size_t)1 << n) * C.L.cbytes;
    // capture on a private stream (the caller's may be the legacy default stream, which
    // cannot be captured); the graph itself is launched on the caller's stream
    cudaStream_t cs = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    C.s = cs;
    const long long launches0 = cheb_launch_count();
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return CHEB_ERR_CUDA;
    }
    for (int s = 0; s < S; ++s) {
        const Seg& G = segs[s];
        if (boundaries &&
            cudaMemcpyAsync((unsigned char*)boundaries + (size_t)s * vbytes, psi, vbytes, cudaMemcpyDeviceToDevice,
                            cs) != cudaSuccess)
            return abandon(cs, CHEB_ERR_CUDA);
        unsigned char* seg = store + (size_t)s * seg_bytes(n, precision);
        if (cudaMemcpyAsync(C.ws + C.L.jq, seg, jq_bytes(n), cudaMemcpyDeviceToDevice, cs) != cudaSuccess)
            return abandon(cs, CHEB_ERR_CUDA);
        C.dev_coef = seg_bytes(n, precision) > a256(jq_bytes(n)) ? seg + a256(jq_bytes(n)) : nullptr;
        launch_tables(n, C.L.M, (const int64_t*)(C.ws + C.L.jq), C.tiles(), C.elow(), cs);
        if (cudaGetLastError() != cudaSuccess) return abandon(cs, CHEB_ERR_CUDA);
        for (int q = 0; q < G.slices; ++q) {
            st = clenshaw_run(C, CHEB_PATH_AUTO, psi, G.coef, G.F.Q, G.g);
            if (st != CHEB_OK) return abandon(cs, st);
        }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess || !g) {
        cudaGetLastError();
        return CHEB_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CHEB_ERR_CUDA;
    }
    cheb_anneal_graph* G = new cheb_anneal_graph;
    G->exec = exec;
    G->kernels = cheb_launch_count() - launches0;
    cudaGetDevice(&G->device);
    *graph = G;
    return CHEB_OK;
}

extern "C" cheb_status_t cheb_anneal_graph_launch(cheb_anneal_graph_t graph, void* stream) {
    if (!graph || !graph->exec) return CHEB_ERR_INVALID_ARG;
    note_launches(graph->kernels);
    CUDA_TRY(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
    return CHEB_OK;
}

extern "C" void cheb_anneal_graph_destroy(cheb_anneal_graph_t graph) {
    if (!graph) return;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    delete graph;
}
