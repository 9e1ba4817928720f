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

// Segments H_s = b_s H_P + a_s sum_j X_j (b_s = 1 when b is null), psi <- exp(-i t_s H_s) psi
// in order for s < s_end (s_end < 0: all S). b_s H_P has energies b_s E(z): its centre is
// b_s c and its half-width |b_s| (Emax - Emin)/2, so one bounds scan serves every segment;
// the fixed-point tables are rebuilt per segment from the scaled couplings. Every segment
// takes the tolerance tol / S.
cheb_status_t cheb::anneal_run(int n, const double* h, const double* J, int S, const double* b_s,
                               const double* a_s, const double* t_s, void* psi, cheb_precision_t precision,
                               double tol, cheb_method_t method, void* boundaries, void* workspace,
                               size_t ws_bytes, void* stream, cheb_info_t* infos, int s_end) {
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
    const int S_run = (s_end < 0 || s_end > S) ? S : s_end;
    for (int s = 0; s < S_run; ++s) {
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
            in.eval_bound = -1.0;
            if (!std::isfinite(ne[0]) || !std::isfinite(ne[1])) return CHEB_ERR_NONFINITE;
        }
    }
    return CHEB_OK;
}

extern "C" cheb_status_t cheb_anneal(int n, const double* h, const double* J, int S, const double* gamma_s,
                                     const double* t_s, void* psi, cheb_precision_t precision, double tol,
                                     cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes,
                                     void* stream, cheb_info_t* infos) {
    return anneal_run(n, h, J, S, nullptr, gamma_s, t_s, psi, precision, tol, method, boundaries, workspace,
                      ws_bytes, stream, infos);
}

extern "C" cheb_status_t cheb_anneal_general(int n, const double* h, const double* J, int S, const double* a_s,
                                             const double* b_s, const double* t_s, void* psi,
                                             cheb_precision_t precision, double tol, cheb_method_t method,
                                             void* boundaries, void* workspace, size_t ws_bytes, void* stream,
                                             cheb_info_t* infos) {
    if (!b_s) return CHEB_ERR_INVALID_ARG;
    return anneal_run(n, h, J, S, b_s, a_s, t_s, psi, precision, tol, method, boundaries, workspace, ws_bytes,
                      stream, infos);
}

// Fourth-order commutator-free Magnus step (the exponential integrator for
// time-dependent H cited in Sec. III.B, built from two exponentials of linear
// combinations of H at the Gauss-Legendre nodes t1,2 = t + (1/2 -+ sqrt(3)/6) dt):
//   psi <- exp(-i dt (w1 H(t1) + w2 H(t2))) exp(-i dt (w2 H(t1) + w1 H(t2))) psi,
//   w1 = 1/4 - sqrt(3)/6, w2 = 1/4 + sqrt(3)/6,
// with H(t) = A(t) sum_j X_j + B(t) H_P, so that every factor is one segment
// b H_P + a sum_j X_j of cheb_anneal_general.
namespace {

const double kW1 = 0.25 - std::sqrt(3.0) / 6.0, kW2 = 0.25 + std::sqrt(3.0) / 6.0;

// Segments (a_s, b_s, t_s) of the 2*steps exponentials; segment 2m is applied first.
void magnus_segments(int steps, const double* dt, const double* nodes, std::vector<double>& a,
                     std::vector<double>& b, std::vector<double>& t) {
    a.resize(2 * (size_t)steps);
    b.resize(2 * (size_t)steps);
    t.resize(2 * (size_t)steps);
    for (int m = 0; m < steps; ++m) {
        const double A1 = nodes[4 * m + 0], B1 = nodes[4 * m + 1], A2 = nodes[4 * m + 2], B2 = nodes[4 * m + 3];
        a[2 * m] = kW2 * A1 + kW1 * A2;
        b[2 * m] = kW2 * B1 + kW1 * B2;
        a[2 * m + 1] = kW1 * A1 + kW2 * A2;
        b[2 * m + 1] = kW1 * B1 + kW2 * B2;
        t[2 * m] = t[2 * m + 1] = dt[m];
    }
}

bool magnus_args_ok(int steps, const double* dt, const double* nodes) {
    return steps >= 1 && dt && nodes && finite_all(dt, steps) && finite_all(nodes, (size_t)4 * steps);
}

}  // namespace

extern "C" cheb_status_t cheb_magnus4_nodes(double T, int steps, cheb_schedule_fn schedule, void* user, double* dt,
                                            double* nodes) {
    if (steps < 1 || !schedule || !dt || !nodes || !std::isfinite(T)) return CHEB_ERR_INVALID_ARG;
    const double h = T / steps;
    for (int m = 0; m < steps; ++m) {
        const double t1 = m * h + (0.5 - std::sqrt(3.0) / 6.0) * h;
        const double t2 = m * h + (0.5 + std::sqrt(3.0) / 6.0) * h;
        dt[m] = h;
        if (schedule(t1, &nodes[4 * m + 0], &nodes[4 * m + 1], user) != 0) return CHEB_ERR_INVALID_ARG;
        if (schedule(t2, &nodes[4 * m + 2], &nodes[4 * m + 3], user) != 0) return CHEB_ERR_INVALID_ARG;
    }
    return finite_all(nodes, (size_t)4 * steps) ? CHEB_OK : CHEB_ERR_INVALID_ARG;
}

extern "C" cheb_status_t cheb_magnus4(int n, const double* h, const double* J, int steps, const double* dt,
                                      const double* nodes, void* psi, cheb_precision_t precision, double tol,
                                      cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes,
                                      void* stream, cheb_info_t* infos) {
    if (!magnus_args_ok(steps, dt, nodes)) return CHEB_ERR_INVALID_ARG;
    std::vector<double> a, b, t;
    magnus_segments(steps, dt, nodes, a, b, t);
    return anneal_run(n, h, J, 2 * steps, b.data(), a.data(), t.data(), psi, precision, tol, method, boundaries,
                      workspace, ws_bytes, stream, infos);
}

extern "C" cheb_status_t cheb_magnus4_adjoint(int n, const double* h, const double* J, int steps, const double* dt,
                                              const double* nodes, const void* boundaries, const void* psi_T,
                                              void* grad, cheb_precision_t precision, double tol,
                                              cheb_method_t method, double* grad_dt, double* grad_nodes,
                                              double* grad_h, double* grad_J, void* workspace, size_t ws_bytes,
                                              void* stream) {
    if (!magnus_args_ok(steps, dt, nodes)) return CHEB_ERR_INVALID_ARG;
    std::vector<double> a, b, t;
    magnus_segments(steps, dt, nodes, a, b, t);
    const size_t S = 2 * (size_t)steps;
    std::vector<double> ga(S), gb(S), gt(S);
    cheb_status_t st = cheb_anneal_general_adjoint(n, h, J, (int)S, a.data(), b.data(), t.data(), boundaries, psi_T,
                                                   grad, precision, tol, method, ga.data(), gb.data(), gt.data(),
                                                   grad_h, grad_J, workspace, ws_bytes, stream);
    if (st != CHEB_OK) return st;
    // chain rule through the Gauss-node combinations of each step
    for (int m = 0; m < steps; ++m) {
        const size_t s0 = 2 * (size_t)m, s1 = s0 + 1;
        if (grad_dt) grad_dt[m] = gt[s0] + gt[s1];
        if (grad_nodes) {
            grad_nodes[4 * m + 0] = kW2 * ga[s0] + kW1 * ga[s1];
            grad_nodes[4 * m + 1] = kW2 * gb[s0] + kW1 * gb[s1];
            grad_nodes[4 * m + 2] = kW1 * ga[s0] + kW2 * ga[s1];
            grad_nodes[4 * m + 3] = kW1 * gb[s0] + kW2 * gb[s1];
        }
    }
    return CHEB_OK;
}

extern "C" size_t cheb_magnus4_adaptive_workspace_bytes(int n, cheb_precision_t precision) {
    const size_t base = cheb_workspace_bytes(n, precision);
    if (base == 0) return 0;
    const size_t vb = (((size_t)1 << n) * (precision == CHEB_FP32 ? 8 : 16) + 255) / 256 * 256;
    return base + 2 * vb;
}

// Step count chosen a posteriori: runs with M and 2M equal steps estimate the error of
// the 2M run as ||y_M - y_2M|| / 15 (fourth order: halving the step divides the error
// by 16), and a final run uses M' = ceil(2M (est / tol)^(1/4) * 1.1) steps when the
// estimate exceeds tol.
extern "C" cheb_status_t cheb_magnus4_adaptive(int n, const double* h, const double* J, double T,
                                               cheb_schedule_fn schedule, void* user, int steps0, double tol,
                                               void* psi, cheb_precision_t precision, cheb_method_t method,
                                               void* workspace, size_t ws_bytes, void* stream, int* steps_used,
                                               double* err_estimate) {
    if (steps0 < 1 || steps0 > (1 << 20) || !schedule || !(tol > 0) || !std::isfinite(tol) || !std::isfinite(T))
        return CHEB_ERR_INVALID_ARG;
    if (!psi || ((uintptr_t)psi & 15) != 0 || !steps_used) return CHEB_ERR_INVALID_ARG;
    const size_t base = cheb_workspace_bytes(n, precision);
    if (base == 0) return CHEB_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < cheb_magnus4_adaptive_workspace_bytes(n, precision))
        return CHEB_ERR_WORKSPACE;
    const size_t vbytes = ((size_t)1 << n) * (precision == CHEB_FP32 ? 8 : 16);
    const size_t vb = (vbytes + 255) / 256 * 256;
    unsigned char* y1 = (unsigned char*)workspace + base;
    unsigned char* y2 = y1 + vb;
    cudaStream_t s = (cudaStream_t)stream;
    // the series of every exponential at the precision's default budget
    const double tol_series = precision == CHEB_FP32 ? std::ldexp(1.0, -23) : 1e-12;
    auto run = [&](int M, void* y) -> cheb_status_t {
        std::vector<double> dt((size_t)M), nd(4 * (size_t)M);
        cheb_status_t st = cheb_magnus4_nodes(T, M, schedule, user, dt.data(), nd.data());
        if (st != CHEB_OK) return st;
        CUDA_TRY(cudaMemcpyAsync(y, psi, vbytes, cudaMemcpyDeviceToDevice, s));
        return cheb_magnus4(n, h, J, M, dt.data(), nd.data(), y, precision, tol_series, method, nullptr, workspace,
                            base, stream, nullptr);
    };
    cheb_status_t st = run(steps0, y1);
    if (st != CHEB_OK) return st;
    st = run(2 * steps0, y2);
    if (st != CHEB_OK) return st;
    // ||y1 - y2||^2 as ||1 * y1 - y2||^2 of the evaluation-bound reduction
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, s};
    double* d = C.f64out();
    CUDA_TRY(cudaMemsetAsync(d, 0, 2 * sizeof(double), s));
    launch_step_norms(precision, (int64_t)1 << n, y2, y1, 1.0, 0.0, 1, d, d + 1, s);
    double dd[2];
    CUDA_TRY(cudaMemcpyAsync(dd, d, sizeof(dd), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double est = std::sqrt(dd[1]) / 15.0;
    int M = 2 * steps0;
    double final_est = est;
    if (est > tol) {
        const int M2 = (int)std::ceil(M * std::pow(est / tol, 0.25) * 1.1);
        st = run(M2, y2);
        if (st != CHEB_OK) return st;
        final_est = est * std::pow((double)M / M2, 4.0);  // fourth-order scaling of the estimate
        M = M2;
    }
    CUDA_TRY(cudaMemcpyAsync(psi, y2, vbytes, cudaMemcpyDeviceToDevice, s));
    *steps_used = M;
    if (err_estimate) *err_estimate = final_est;
    return CHEB_OK;
}
