// cheb_anneal: a piecewise-constant annealing schedule H_s = H_P + gamma_s sum_j X_j
// applied segment by segment, psi <- exp(-i t_s H_s) psi for s = 0..S-1 (the
// constant-segment building block of the time-dependent evolution of Sec. III.B).
// The Ising diagonal, and hence the spectral centre c, is shared by all segments;
// only the radius r_s = (Emax - Emin)/2 + |gamma_s| n and the series change.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <vector>

#include "kernels.cuh"
#include "pipeline.h"

using namespace cheb;

extern "C" cheb_status_t cheb_anneal(int n, const double* h, const double* J, int S, const double* gamma_s,
                                     const double* t_s, void* psi, cheb_precision_t precision, double tol,
                                     cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes,
                                     void* stream, cheb_info_t* infos) {
    cheb_status_t st = check_common(n, h, J, precision, workspace, ws_bytes);
    if (st != CHEB_OK) return st;
    if (S < 1 || !gamma_s || !t_s || !psi || ((uintptr_t)psi & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (boundaries && ((uintptr_t)boundaries & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(gamma_s, S) || !finite_all(t_s, S) || !(tol > 0) || !std::isfinite(tol))
        return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, (cudaStream_t)stream};
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), C.s));
    double emin = 0, emax = 0;
    st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    const double c = 0.5 * (emax + emin);
    const size_t vbytes = ((size_t)1 << n) * C.L.cbytes;
    const double tol_s = tol / S;
    for (int s = 0; s < S; ++s) {
        double r = 0.5 * (emax - emin) + std::fabs(gamma_s[s]) * n;
        if (!(r > 0)) r = 1.0;
        FixedOp F = make_fixed(n, h, J, c, r, precision == CHEB_FP32 ? kMaxQF32 : 62);
        if (F.Q < 24) return CHEB_ERR_UNSUPPORTED;
        st = upload_tables(C, F);
        if (st != CHEB_OK) return st;
        std::vector<std::complex<double>> coef;
        int K = -1, slices = 1;
        double err = 0.0;
        st = slice_coefficients(t_s[s], c, r, tol_s, method, 0, coef, &K, &slices, &err);
        if (st != CHEB_OK) return st;
        if (boundaries)
            CUDA_TRY(cudaMemcpyAsync((unsigned char*)boundaries + (size_t)s * vbytes, psi, vbytes,
                                     cudaMemcpyDeviceToDevice, C.s));
        const double g = gamma_s[s] / r;
        for (int q = 0; q < slices; ++q) {
            st = clenshaw_run(C, CHEB_PATH_AUTO, psi, coef, F.Q, g);
            if (st != CHEB_OK) return st;
        }
        if (infos) {
            cheb_info_t& in = infos[s];
            launch_norm_energy(precision, n, C.L.M, F.Q, C.tiles(), C.elow(), c, r, psi, C.part(), C.f64out(), C.s);
            CUDA_TRY(cudaGetLastError());
            double ne[2];
            CUDA_TRY(cudaMemcpyAsync(ne, C.f64out(), sizeof(ne), cudaMemcpyDeviceToHost, C.s));
            st = read_flags(C);
            if (st != CHEB_OK) return st;
            in.K = K;
            in.time_splits = slices;
            in.matvecs = (int64_t)K * slices;
            in.emin = emin;
            in.emax = emax;
            in.center = c;
            in.radius = r;
            in.a = (t_s[s] / slices) * r;
            in.trunc_bound = err * slices;
            in.norm = std::sqrt(ne[0]);
            in.energy = ne[1];
            if (!std::isfinite(ne[0]) || !std::isfinite(ne[1])) return CHEB_ERR_NONFINITE;
        }
    }
    return CHEB_OK;
}
