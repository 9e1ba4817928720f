// Host-side pieces of the exp(-itH) psi pipeline shared by the entry points
// (api.cu: single expmv; anneal.cu: schedules; batched.cu; adjoint.cu).
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <vector>

#include "../../include/cheb_expmv.h"
#include "cheb_internal.h"

namespace cheb {

// Couplings in fixed point: value = integer * 2^-Q.
struct FixedOp {
    int Q = 0;
    std::vector<int64_t> jq;  // J symmetric n*n, then h[n], then c
};

// One call's view of a workspace.
struct Ctx {
    int n;
    int prec;
    Layout L;
    unsigned char* ws;
    cudaStream_t s;
    // when set, the whole-run kernel takes the run's coefficients from this device copy
    // (a captured graph must not read host memory at replay)
    const void* dev_coef = nullptr;
    int64_t* tiles() const { return (int64_t*)(ws + L.tiles); }
    int64_t* elow() const { return (int64_t*)(ws + L.elow); }
    int* flags() const { return (int*)(ws + L.status); }
    int64_t* i64out() const { return (int64_t*)(ws + L.status + 64); }
    double* f64out() const { return (double*)(ws + L.status + 128); }
    double* part() const { return (double*)(ws + L.part); }
};

#define CUDA_TRY(x)                                   \
    do {                                              \
        if ((x) != cudaSuccess) return CHEB_ERR_CUDA; \
    } while (0)

bool finite_all(const double* p, size_t k);
// J/scale, h/scale, center/scale quantised at the largest safe Q (<= max_q).
FixedOp make_fixed(int n, const double* h, const double* J, double center, double scale, int max_q = 62);
cheb_status_t upload_tables(const Ctx& C, const FixedOp& F);
cheb_status_t check_common(int n, const double* h, const double* J, int prec, void* ws, size_t ws_bytes);
// Exact E_min, E_max of the Ising diagonal (synchronises the stream).
cheb_status_t bounds_impl(Ctx& C, const double* h, const double* J, double* emin, double* emax);
// One Clenshaw run of coefficients c over psi in place, with the tables already uploaded.
// step_norms (device, nullable): 2(K+1) zeroed doubles that receive, per k, ||b_k||^2 at
// [2k] and ||c_k psi - b_{k+2}||^2 at [2k+1] (k <= K-2) for the evaluation bound of
// Sec. II.B.3; the run then uses the step-by-step kernels (b_k must be visible).
cheb_status_t clenshaw_run(Ctx& C, int path, void* psi, const std::vector<std::complex<double>>& c, int Q,
                           double g, double* step_norms = nullptr);
// Applies the autotuner cache named by CHEB_AUTOTUNE_CACHE (once per process).
void autotune_cache_once();
// Synchronises and maps the device status word to a status code.
cheb_status_t read_flags(const Ctx& C);
// Segments s < s_end (s_end < 0: all S) of a schedule H_s = b_s H_P + a_s sum_j X_j
// (b_s = 1 when b_s is null), each with tolerance tol / S (cheb_anneal_general).
cheb_status_t anneal_run(int n, const double* h, const double* J, int S, const double* b_s, const double* a_s,
                         const double* t_s, void* psi, cheb_precision_t precision, double tol,
                         cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes, void* stream,
                         cheb_info_t* infos, int s_end = -1);
// Coefficients of exp(-i a x) * exp(-i ts c) for one slice, slicing t automatically
// (splits = 0) when the degree would exceed the coefficient table.
cheb_status_t slice_coefficients(double t, double c, double r, double tol, int method, int splits,
                                 std::vector<std::complex<double>>& coef, int* K, int* s_out, double* err);

}  // namespace cheb
