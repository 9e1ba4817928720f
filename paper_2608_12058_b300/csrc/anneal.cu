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

namespace {

// Segments H_s = b_s H_P + a_s sum_j X_j (b_s = 1 when b is null), psi <- exp(-i t_s H_s) psi
// in order. b_s H_P has energies b_s E(z): its centre is b_s c and its half-width
// |b_s| (Emax - Emin)/2, so one bounds scan serves every segment; the fixed-point
// tables are rebuilt per segment from the scaled couplings.
cheb_status_t anneal_impl(int n, const double* h, const double* J, int S, const double* b_s, const double* a_s,
                          const double* t_s, void* psi, cheb_precision_t precision, double tol,
                          cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes, void* stream,
                          cheb_info_t* infos) {
    cheb_status_t st = check_common(n, h, J, precision, workspace, ws_bytes);
    if (st != CHEB_OK) return st;
    if (S < 1 || !a_s || !t_s || !psi || ((uintptr_t)psi & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (boundaries && ((uintptr_t)boundaries & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(a_s, S) || !finite_all(t_s, S) || (b_s && !finite_all(b_s, S)) || !(tol > 0) ||
        !std::isfinite(tol))
        return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, (cudaStream_t)stream};
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), C.s));
    double emin = 0, emax = 0;
    st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    const size_t vbytes = ((size_t)1 << n) * C.L.cbytes;
    const double tol_s = tol / S;
    std::vector<double> hb(n), Jb((size_t)n * n);
    for (int s = 0; s < S; ++s) {
        const double b = b_s ? b_s[s] : 1.0;
        const double c = b * 0.5 * (emax + emin);
        double r = std::fabs(b) * 0.5 * (emax - emin) + std::fabs(a_s[s]) * n;
        if (!(r > 0)) r = 1.0;
        for (int i = 0; i < n; ++i) hb[i] = b * h[i];
        for (size_t q = 0; q < (size_t)n * n; ++q) Jb[q] = b * J[q];
        FixedOp F = make_fixed(n, hb.data(), Jb.data(), c, r, precision == CHEB_FP32 ? kMaxQF32 : 62);
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
        const double g = a_s[s] / r;
        for (int q = 0; q < slices; ++q) {
            st = clenshaw_run(C, CHEB_PATH_AUTO, psi, coef, F.Q, g);
            if (st != CHEB_OK) return st;
        }
        if (infos) {
            cheb_info_t& in = infos[s];
            // energy of the segment's diagonal part b_s H_P (the tables hold b_s E)
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

}  // namespace

extern "C" cheb_status_t cheb_anneal(int n, const double* h, const double* J, int S, const double* gamma_s,
                                     const double* t_s, void* psi, cheb_precision_t precision, double tol,
                                     cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes,
                                     void* stream, cheb_info_t* infos) {
    return anneal_impl(n, h, J, S, nullptr, gamma_s, t_s, psi, precision, tol, method, boundaries, workspace,
                       ws_bytes, stream, infos);
}

extern "C" cheb_status_t cheb_anneal_general(int n, const double* h, const double* J, int S, const double* a_s,
                                             const double* b_s, const double* t_s, void* psi,
                                             cheb_precision_t precision, double tol, cheb_method_t method,
                                             void* boundaries, void* workspace, size_t ws_bytes, void* stream,
                                             cheb_info_t* infos) {
    if (!b_s) return CHEB_ERR_INVALID_ARG;
    return anneal_impl(n, h, J, S, b_s, a_s, t_s, psi, precision, tol, method, boundaries, workspace, ws_bytes,
                       stream, infos);
}

// Fourth-order commutator-free Magnus step (the exponential integrator for
// time-dependent H cited in Sec. III.B, built from two exponentials of linear
// combinations of H at the Gauss-Legendre nodes t1,2 = t + (1/2 -+ sqrt(3)/6) dt):
//   psi <- exp(-i dt (w1 H(t1) + w2 H(t2))) exp(-i dt (w2 H(t1) + w1 H(t2))) psi,
//   w1 = 1/4 - sqrt(3)/6, w2 = 1/4 + sqrt(3)/6,
// with H(t) = A(t) sum_j X_j + B(t) H_P, so that every factor is one segment
// b H_P + a sum_j X_j of cheb_anneal_general.
extern "C" cheb_status_t cheb_magnus4(int n, const double* h, const double* J, int steps, const double* dt,
                                      const double* nodes, void* psi, cheb_precision_t precision, double tol,
                                      cheb_method_t method, void* workspace, size_t ws_bytes, void* stream,
                                      cheb_info_t* infos) {
    if (steps < 1 || !dt || !nodes) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(dt, steps) || !finite_all(nodes, (size_t)4 * steps)) return CHEB_ERR_INVALID_ARG;
    const double w1 = 0.25 - std::sqrt(3.0) / 6.0, w2 = 0.25 + std::sqrt(3.0) / 6.0;
    std::vector<double> a(2 * (size_t)steps), b(2 * (size_t)steps), t(2 * (size_t)steps);
    for (int m = 0; m < steps; ++m) {
        const double A1 = nodes[4 * m + 0], B1 = nodes[4 * m + 1], A2 = nodes[4 * m + 2], B2 = nodes[4 * m + 3];
        // applied first: w2 H(t1) + w1 H(t2); then w1 H(t1) + w2 H(t2)
        a[2 * m] = w2 * A1 + w1 * A2;
        b[2 * m] = w2 * B1 + w1 * B2;
        a[2 * m + 1] = w1 * A1 + w2 * A2;
        b[2 * m + 1] = w1 * B1 + w2 * B2;
        t[2 * m] = t[2 * m + 1] = dt[m];
    }
    return anneal_impl(n, h, J, 2 * steps, b.data(), a.data(), t.data(), psi, precision, tol, method, nullptr,
                       workspace, ws_bytes, stream, infos);
}
