// C ABI entry points (include/cheb_expmv.h): argument checks, workspace layout,
// fixed-point operator tables, coefficient generation and the Clenshaw step loop.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/cheb_expmv.h"
#include "cheb_internal.h"
#include "fused.cuh"
#include "fused_ff.cuh"
#include "kernels.cuh"
#include "pipeline.h"

namespace cheb {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout make_layout(int n, int precision) {
    Layout L;
    L.n = n;
    L.M = n < kTileBits ? n : kTileBits;
    L.cbytes = precision == 0 ? 8 : 16;
    size_t off = 0;
    L.status = off;
    off += 256;
    L.part = off;
    off = align_up(off + 4 * kRedBlocks * sizeof(double), 256);
    L.jq = off;
    off = align_up(off + ((size_t)n * n + n + 1) * sizeof(int64_t), 256);
    L.tiles = off;
    off = align_up(off + ((size_t)1 << (n - L.M)) * (L.M + 1) * sizeof(int64_t), 256);
    L.elow = off;
    off = align_up(off + ((size_t)1 << L.M) * sizeof(int64_t), 256);
    L.coef = off;
    off = align_up(off + (size_t)(kMaxK + 1) * 2 * sizeof(double), 256);
    off += fused_scratch_bytes(n, precision);
    off = align_up(off, 256);
    L.b0 = off;
    off = align_up(off + ((size_t)1 << n) * L.cbytes, 256);
    L.b1 = off;
    off = align_up(off + ((size_t)1 << n) * L.cbytes, 256);
    L.total = off;
    return L;
}

bool finite_all(const double* p, size_t k) {
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Largest Q <= 62 with bound * 2^Q <= 2^61 (so every partial sum fits in int64).
static int choose_scale(long double bound) {
    if (!(bound > 0)) return 62;
    int e = (int)std::ceil(std::log2((double)bound));
    int Q = 61 - e;
    return Q > 62 ? 62 : Q;
}

// J/scale, h/scale, c/scale quantised at the largest safe Q.
FixedOp make_fixed(int n, const double* h, const double* J, double center, double scale, int max_q) {
    FixedOp F;
    long double bound = std::fabs((long double)center);
    for (int i = 0; i < n; ++i) {
        bound += std::fabs((long double)h[i]);
        for (int j = i + 1; j < n; ++j) bound += std::fabs((long double)J[(size_t)i * n + j]);
    }
    bound /= (long double)scale;
    F.Q = std::min(choose_scale(bound), max_q);
    const long double mul = std::ldexp(1.0L, F.Q) / (long double)scale;
    F.jq.assign((size_t)n * n + n + 1, 0);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            int64_t q = (int64_t)std::llroundl((long double)J[(size_t)i * n + j] * mul);
            F.jq[(size_t)i * n + j] = q;
            F.jq[(size_t)j * n + i] = q;
        }
    for (int i = 0; i < n; ++i) F.jq[(size_t)n * n + i] = (int64_t)std::llroundl((long double)h[i] * mul);
    F.jq[(size_t)n * n + n] = (int64_t)std::llroundl((long double)center * mul);
    return F;
}

cheb_status_t upload_tables(const Ctx& C, const FixedOp& F) {
    CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.jq, F.jq.data(), F.jq.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, C.s));
    launch_tables(C.n, C.L.M, (const int64_t*)(C.ws + C.L.jq), C.tiles(), C.elow(), C.s);
    CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status_t check_common(int n, const double* h, const double* J, int prec, void* ws, size_t ws_bytes) {
    if (n < 1 || n > kMaxQubits) return CHEB_ERR_INVALID_ARG;
    if (!h || !J) return CHEB_ERR_INVALID_ARG;
    if (prec != CHEB_FP32 && prec != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(h, n) || !finite_all(J, (size_t)n * n)) return CHEB_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255) != 0) return CHEB_ERR_WORKSPACE;
    if (ws_bytes < make_layout(n, prec).total) return CHEB_ERR_WORKSPACE;
    return CHEB_OK;
}

cheb_status_t bounds_impl(Ctx& C, const double* h, const double* J, double* emin, double* emax) {
    FixedOp F = make_fixed(C.n, h, J, 0.0, 1.0);
    cheb_status_t st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    launch_minmax(C.n, C.L.M, C.tiles(), C.elow(), (int64_t*)C.part(), C.i64out(), C.s);
    CUDA_TRY(cudaGetLastError());
    int64_t mm[2];
    CUDA_TRY(cudaMemcpyAsync(mm, C.i64out(), sizeof(mm), cudaMemcpyDeviceToHost, C.s));
    CUDA_TRY(cudaStreamSynchronize(C.s));
    *emin = std::ldexp((double)mm[0], -F.Q);
    *emax = std::ldexp((double)mm[1], -F.Q);
    return CHEB_OK;
}

// One Clenshaw run (Algorithm 2) of the coefficients c over psi, in place.
cheb_status_t clenshaw_run(Ctx& C, int path, void* psi, const std::vector<std::complex<double>>& c, int Q,
                           double g, double* step_norms) {
    autotune_cache_once();
    const int K = (int)c.size() - 1;
    const int64_t N = (int64_t)1 << C.n;
    if (K == 0) {
        launch_scale(C.prec, N, psi, psi, c[0].real(), c[0].imag(), C.s);
        CUDA_TRY(cudaGetLastError());
        if (step_norms) launch_step_norms(C.prec, N, psi, psi, 0, 0, 0, step_norms, nullptr, C.s);
        return CHEB_OK;
    }
    const int small_max = C.prec == 0 ? kSmallMaxF32 : kSmallMaxF64;
    // the evaluation bound needs every b_k in memory: the plain kernel replaces the
    // whole-run shared-memory kernel
    if (step_norms && path == CHEB_PATH_AUTO && C.n <= small_max) path = CHEB_PATH_PLAIN;
    // a choice measured by the autotuner replaces the built-in AUTO rule
    if (path == CHEB_PATH_AUTO && C.n > small_max) {
        const int tp = tuned_auto_path(C.prec, C.n);
        if (tp == CHEB_PATH_PLAIN || tp == CHEB_PATH_FUSED) path = tp;
    }
    if (path == CHEB_PATH_AUTO && C.n <= small_max) {
        static_assert(sizeof(std::complex<double>) == 2 * sizeof(double), "layout");
        if (C.dev_coef)
            CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.coef, C.dev_coef, c.size() * sizeof(std::complex<double>),
                                     cudaMemcpyDeviceToDevice, C.s));
        else
            CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.coef, c.data(), c.size() * sizeof(std::complex<double>),
                                     cudaMemcpyHostToDevice, C.s));
        CUDA_TRY(launch_small(C.prec, C.n, K, (const double*)(C.ws + C.L.coef), Q, C.tiles(), C.elow(), g,
                              psi, C.s));
        return CHEB_OK;
    }
    const int csb = cluster_slice_bits(C.prec);
    if (path == CHEB_PATH_CLUSTER && step_norms) return CHEB_ERR_UNSUPPORTED;
    if (path == CHEB_PATH_CLUSTER && C.n > csb && C.n <= csb + 4) {
        // whole run on one cluster; its descriptor goes to the reduction scratch, which
        // the run does not otherwise use
        CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.coef, c.data(), c.size() * sizeof(std::complex<double>),
                                 cudaMemcpyHostToDevice, C.s));
        SmallDesc d{};
        d.n = C.n;
        d.K = K;
        d.Q = Q;
        d.g = g;
        d.coef = (const double*)(C.ws + C.L.coef);
        d.tiles = C.tiles();
        d.elow = C.elow();
        d.psi = psi;
        SmallDesc* dd = (SmallDesc*)C.part();
        CUDA_TRY(cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, C.s));
        const cudaError_t e = launch_cluster_batched(C.prec, C.n, 1, dd, C.s);
        if (e == cudaSuccess) return CHEB_OK;
        (void)cudaGetLastError();
        return e == cudaErrorNotSupported ? CHEB_ERR_UNSUPPORTED : CHEB_ERR_CUDA;
    } else if (path == CHEB_PATH_CLUSTER) {
        return CHEB_ERR_UNSUPPORTED;
    }
    // AUTO: below 2^20 amplitudes (L2-resident vectors) a step is launch-bound and the
    // one-launch plain kernel is faster than the two-pass fused step (measured)
    bool fused = false;
    if (path == CHEB_PATH_FUSED || (path == CHEB_PATH_AUTO && C.n > kPlainMaxF32))
        fused = fused_supported(C.n, C.prec);
    // FP64: the float-float fused step (complex128 storage, arithmetic on the FP32 units)
    bool ff = false;
    if (C.prec == CHEB_FP64 && (path == CHEB_PATH_FUSED || (path == CHEB_PATH_AUTO && C.n >= kFFAutoMinF64)))
        ff = ff_supported(C.n);
    if (path == CHEB_PATH_FUSED && !fused && !ff) return CHEB_ERR_UNSUPPORTED;
    unsigned char* B[2] = {C.ws + C.L.b0, C.ws + C.L.b1};
    if (ff) {
        // the run works on float-float vectors: psi is converted in place, and the final
        // step writes y back as complex128
        CUDA_TRY(launch_to_ff(N, psi, C.s));
        CUDA_TRY(launch_ff_scale(N, psi, B[1], c[K].real(), c[K].imag(), C.s));
    } else {
        launch_scale(C.prec, N, psi, B[1], c[K].real(), c[K].imag(), C.s);
    }
    auto norms = [&](int k, const void* bk) {
        // ||b_k||^2, and ||c_{k-2} psi - b_k||^2 while b_k is still the b_{k+2} of step k - 2
        if (!step_norms) return;
        const bool wc = k >= 2;
        const std::complex<double> cc = wc ? c[k - 2] : std::complex<double>(0.0, 0.0);
        const int fmt = (ff && k > 0) ? kFormatFF : C.prec;
        launch_step_norms(fmt, N, bk, psi, cc.real(), cc.imag(), wc ? 1 : 0, step_norms + 2 * k,
                          wc ? step_norms + 2 * (k - 2) + 1 : nullptr, C.s);
    };
    norms(K, B[1]);
    FusedPlan plan;
    if (fused) plan = fused_plan(C.n, C.prec);
    if (ff) plan = ff_plan(C.n);
    int cur = 1;
    for (int k = K - 1; k >= 0; --k) {
        StepArgs a;
        a.n = C.n;
        a.M = C.L.M;
        a.Q = Q;
        a.tiles = C.tiles();
        a.elow = C.elow();
        a.jq = (const int64_t*)(C.ws + C.L.jq);
        a.b1 = B[cur];
        a.b2 = B[cur ^ 1];
        a.psi = psi;
        a.out = (k == 0) ? psi : (void*)B[cur ^ 1];
        a.ck_re = c[k].real();
        a.ck_im = c[k].imag();
        a.scale = (k == 0) ? 1.0 : 2.0;
        a.sgn = (k == K - 1) ? 0.0 : -1.0;
        a.g = g;
        if (ff) {
            if (launch_step_ff(plan, a, C.ws + C.L.coef + (size_t)(kMaxK + 1) * 2 * sizeof(double), C.flags(), k == 0,
                               C.s) != cudaSuccess)
                return CHEB_ERR_CUDA;
        } else if (fused) {
            cudaError_t e = launch_step_fused(plan, a, C.ws + C.L.coef + (size_t)(kMaxK + 1) * 2 * sizeof(double),
                                              C.flags(), C.s);
            if (e != cudaSuccess) return CHEB_ERR_CUDA;
        } else {
            launch_step_plain(C.prec, a, C.s);
        }
        norms(k, a.out);
        cur ^= 1;
    }
    CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status_t read_flags(const Ctx& C) {
    int f = 0;
    CUDA_TRY(cudaMemcpyAsync(&f, C.flags(), sizeof(int), cudaMemcpyDeviceToHost, C.s));
    CUDA_TRY(cudaStreamSynchronize(C.s));
    if (f & kFlagTimeout) return CHEB_ERR_TIMEOUT;
    if (f & kFlagBadLaunch) return CHEB_ERR_CUDA;
    return CHEB_OK;
}

cheb_status_t slice_coefficients(double t, double c, double r, double tol, int method, int splits,
                                 std::vector<std::complex<double>>& coef, int* K_out, int* s_out, double* err) {
    // coefficients, with automatic slicing when the degree exceeds the table
    int s = splits > 0 ? splits : 1;
    int K = -1;
    for (int attempt = 0; attempt < 24; ++attempt) {
        const double ts = t / s;
        const std::complex<double> phase = std::polar(1.0, -ts * c);
        K = make_coefficients(ts * r, phase, tol / s, method, kMaxK, coef, err);
        if (K >= 0 || splits > 0) break;
        s *= 2;
    }
    if (K < 0) return CHEB_ERR_UNSUPPORTED;
    *K_out = K;
    *s_out = s;
    return CHEB_OK;
}

// Unit roundoff of the arithmetic that a Clenshaw run of (n, prec, path) uses: FP32
// (operator constants in float-float, flip sums in FP32), the float-float FP64 path,
// or native FP64.
double unit_roundoff(int n, int prec, int path) {
    if (prec == CHEB_FP32) return std::ldexp(1.0, -24);
    if (path == CHEB_PATH_AUTO && n > kSmallMaxF64) {
        const int tp = tuned_auto_path(prec, n);
        if (tp == CHEB_PATH_PLAIN || tp == CHEB_PATH_FUSED) path = tp;
    }
    // float-float (about 48 significant bits): 2^-47 bounds the relative error of its
    // additions and products
    if (path == CHEB_PATH_FUSED || (path == CHEB_PATH_AUTO && n >= kFFAutoMinF64 && ff_supported(n)))
        return std::ldexp(1.0, -47);
    return std::ldexp(1.0, -53);
}

// The a-posteriori evaluation bound of Sec. II.B.3 for one Clenshaw run:
//   sum_{k=0}^{K} u ||b_k|| + u ||c_k psi - b_{k+2}|| + sqrt(d) gamma_d ||b_{k+1}||,
// d = n + 1 nonzeros per column of H, gamma_d = d u / (1 - d u), ||Ht||_2 <= 1,
// b_0 = y, b_{K+1} = b_{K+2} = 0. norms2 holds ||b_k||^2 at [2k] and
// ||c_k psi - b_{k+2}||^2 at [2k+1] for k <= K-2; for k = K-1, K, b_{k+2} = 0.
double evaluation_bound(int n, int prec, int path, const std::vector<std::complex<double>>& c,
                        const std::vector<double>& norms2, double psi_norm) {
    const int K = (int)c.size() - 1;
    const double u = unit_roundoff(n, prec, path);
    const double d = n + 1.0;
    const double gd = d * u / (1.0 - d * u);
    double sum = 0.0;
    for (int k = 0; k <= K; ++k) {
        const double bk = std::sqrt(norms2[2 * (size_t)k]);
        const double bk1 = k + 1 <= K ? std::sqrt(norms2[2 * (size_t)(k + 1)]) : 0.0;
        const double ck = k <= K - 2 ? std::sqrt(norms2[2 * (size_t)k + 1]) : std::abs(c[k]) * psi_norm;
        sum += u * bk + u * ck + std::sqrt(d) * gd * bk1;
    }
    return sum;
}

cheb_status_t expmv_impl(int n, const double* h, const double* J, double gamma, double t, void* psi,
                                int prec, double tol, int method, int splits, int path, void* ws,
                                size_t ws_bytes, void* stream, cheb_info_t* info) {
    cheb_status_t st = check_common(n, h, J, prec, ws, ws_bytes);
    if (st != CHEB_OK) return st;
    if (!psi || ((uintptr_t)psi & 15) != 0) return CHEB_ERR_INVALID_ARG;
    if (!std::isfinite(gamma) || !std::isfinite(t) || !(tol > 0) || !std::isfinite(tol)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    const bool want_bound = (path & CHEB_FLAG_EVAL_BOUND) != 0;
    path &= ~CHEB_FLAG_EVAL_BOUND;
    if (splits < 0 || path < 0 || path > 3) return CHEB_ERR_INVALID_ARG;
    if (want_bound && !info) return CHEB_ERR_INVALID_ARG;
    Ctx C{n, prec, make_layout(n, prec), (unsigned char*)ws, (cudaStream_t)stream};
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), C.s));
    double emin = 0, emax = 0;
    st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    const double c = 0.5 * (emax + emin);
    double r = 0.5 * (emax - emin) + std::fabs(gamma) * n;
    if (!(r > 0)) r = 1.0;  // H is the constant c: any radius is exact
    FixedOp F = make_fixed(n, h, J, c, r, prec == CHEB_FP32 ? kMaxQF32 : 62);
    if (F.Q < 24) return CHEB_ERR_UNSUPPORTED;
    st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    int s = 1, K = -1;
    std::vector<std::complex<double>> coef;
    double err = 0.0;
    st = slice_coefficients(t, c, r, tol, method, splits, coef, &K, &s, &err);
    if (st != CHEB_OK) return st;
    const double g = gamma / r;
    double ebound = -1.0;
    if (want_bound) ebound = 0.0;
    for (int q = 0; q < s; ++q) {
        if (!want_bound) {
            st = clenshaw_run(C, path, psi, coef, F.Q, g);
            if (st != CHEB_OK) return st;
            continue;
        }
        // the step norms go to the coefficient table (unused by the step-by-step
        // kernels), ||psi||^2 next to the reduction outputs
        double* dn = (double*)(C.ws + C.L.coef);
        double* dpsi = C.f64out() + 2;
        CUDA_TRY(cudaMemsetAsync(dn, 0, 2 * (size_t)(K + 1) * sizeof(double), C.s));
        CUDA_TRY(cudaMemsetAsync(dpsi, 0, sizeof(double), C.s));
        launch_step_norms(prec, (int64_t)1 << n, psi, psi, 0, 0, 0, dpsi, nullptr, C.s);
        std::vector<double> hn(2 * (size_t)(K + 1));
        double psi2 = 0;
        CUDA_TRY(cudaMemcpyAsync(&psi2, dpsi, sizeof(double), cudaMemcpyDeviceToHost, C.s));
        st = clenshaw_run(C, path, psi, coef, F.Q, g, dn);
        if (st != CHEB_OK) return st;
        CUDA_TRY(cudaMemcpyAsync(hn.data(), dn, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, C.s));
        CUDA_TRY(cudaStreamSynchronize(C.s));
        ebound += evaluation_bound(n, prec, path, coef, hn, std::sqrt(psi2));
    }
    if (info) {
        launch_norm_energy(prec, n, C.L.M, F.Q, C.tiles(), C.elow(), c, r, psi, C.part(), C.f64out(), C.s);
        CUDA_TRY(cudaGetLastError());
        double ne[2];
        CUDA_TRY(cudaMemcpyAsync(ne, C.f64out(), sizeof(ne), cudaMemcpyDeviceToHost, C.s));
        st = read_flags(C);
        if (st != CHEB_OK) return st;
        info->K = K;
        info->time_splits = s;
        info->matvecs = (int64_t)K * s;
        info->emin = emin;
        info->emax = emax;
        info->center = c;
        info->radius = r;
        info->a = (t / s) * r;
        info->trunc_bound = err * s;
        info->norm = std::sqrt(ne[0]);
        info->energy = ne[1];
        info->eval_bound = ebound;
        if (!std::isfinite(ne[0]) || !std::isfinite(ne[1])) return CHEB_ERR_NONFINITE;
    }
    return CHEB_OK;
}

}  // namespace cheb

using namespace cheb;

extern "C" {

const char* cheb_status_string(cheb_status_t s) {
    switch (s) {
        case CHEB_OK: return "ok";
        case CHEB_ERR_INVALID_ARG: return "invalid argument";
        case CHEB_ERR_WORKSPACE: return "workspace too small or misaligned";
        case CHEB_ERR_CUDA: return "CUDA runtime error";
        case CHEB_ERR_TIMEOUT: return "device wait timed out";
        case CHEB_ERR_NONFINITE: return "non-finite result";
        case CHEB_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* cheb_version(void) { return "cheb_expmv 0.1 (sm_103a)"; }

cheb_status_t cheb_coefficients(double a, double phase_re, double phase_im, double tol, cheb_method_t method,
                                int max_K, double* coeffs, int* K, double* err_bound) {
    if (!std::isfinite(a) || !(tol > 0) || !std::isfinite(tol) || !coeffs || !K || max_K < 0)
        return CHEB_ERR_INVALID_ARG;
    if (!std::isfinite(phase_re) || !std::isfinite(phase_im)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    std::vector<std::complex<double>> c;
    double err = 0;
    int k = make_coefficients(a, std::complex<double>(phase_re, phase_im), tol, method, max_K, c, &err);
    if (k < 0) return CHEB_ERR_UNSUPPORTED;
    for (int m = 0; m <= k; ++m) {
        coeffs[2 * m] = c[m].real();
        coeffs[2 * m + 1] = c[m].imag();
    }
    *K = k;
    if (err_bound) *err_bound = err;
    return CHEB_OK;
}

cheb_status_t cheb_monomial_to_chebyshev(int K, const double* monomial, double* chebyshev) {
    if (K < 0 || K > kMaxK || !monomial || !chebyshev) return CHEB_ERR_INVALID_ARG;
    std::vector<std::complex<double>> a(K + 1), c(K + 1);
    for (int m = 0; m <= K; ++m) {
        a[m] = std::complex<double>(monomial[2 * m], monomial[2 * m + 1]);
        if (!std::isfinite(monomial[2 * m]) || !std::isfinite(monomial[2 * m + 1])) return CHEB_ERR_INVALID_ARG;
    }
    monomial_to_chebyshev(K, a.data(), c.data());
    for (int k = 0; k <= K; ++k) {
        chebyshev[2 * k] = c[k].real();
        chebyshev[2 * k + 1] = c[k].imag();
    }
    return CHEB_OK;
}

size_t cheb_workspace_bytes(int n, cheb_precision_t precision) {
    if (n < 1 || n > kMaxQubits) return 0;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return 0;
    return make_layout(n, precision).total;
}

cheb_status_t cheb_ising_bounds(int n, const double* h, const double* J, void* workspace, size_t workspace_bytes,
                                void* stream, double* emin, double* emax) {
    cheb_status_t st = check_common(n, h, J, CHEB_FP32, workspace, workspace_bytes);
    if (st != CHEB_OK) return st;
    if (!emin || !emax) return CHEB_ERR_INVALID_ARG;
    Ctx C{n, 0, make_layout(n, 0), (unsigned char*)workspace, (cudaStream_t)stream};
    return bounds_impl(C, h, J, emin, emax);
}

cheb_status_t cheb_expmv(int n, const double* h, const double* J, double gamma, double t, void* psi,
                         cheb_precision_t precision, double tol, cheb_method_t method, int time_splits,
                         void* workspace, size_t workspace_bytes, void* stream, cheb_info_t* info) {
    return expmv_impl(n, h, J, gamma, t, psi, precision, tol, method, time_splits, CHEB_PATH_AUTO, workspace,
                      workspace_bytes, stream, info);
}

cheb_status_t cheb_expmv_path(int n, const double* h, const double* J, double gamma, double t, void* psi,
                              cheb_precision_t precision, double tol, cheb_method_t method, int time_splits,
                              int path, void* workspace, size_t workspace_bytes, void* stream,
                              cheb_info_t* info) {
    return expmv_impl(n, h, J, gamma, t, psi, precision, tol, method, time_splits, path, workspace,
                      workspace_bytes, stream, info);
}

cheb_status_t cheb_poly_apply(int n, const double* h, const double* J, double gamma, double center,
                              double radius, int K, const double* coeffs, void* psi, cheb_precision_t precision,
                              int path, void* workspace, size_t workspace_bytes, void* stream) {
    cheb_status_t st = check_common(n, h, J, precision, workspace, workspace_bytes);
    if (st != CHEB_OK) return st;
    if (!psi || ((uintptr_t)psi & 15) != 0 || !coeffs) return CHEB_ERR_INVALID_ARG;
    if (!std::isfinite(gamma) || !std::isfinite(center) || !(radius > 0) || !std::isfinite(radius))
        return CHEB_ERR_INVALID_ARG;
    if (K < 0 || K > kMaxK || path < 0 || path > 3) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(coeffs, 2 * (size_t)(K + 1))) return CHEB_ERR_INVALID_ARG;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, (cudaStream_t)stream};
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), C.s));
    FixedOp F = make_fixed(n, h, J, center, radius, precision == CHEB_FP32 ? kMaxQF32 : 62);
    if (F.Q < 24) return CHEB_ERR_UNSUPPORTED;
    st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    std::vector<std::complex<double>> c(K + 1);
    for (int m = 0; m <= K; ++m) c[m] = std::complex<double>(coeffs[2 * m], coeffs[2 * m + 1]);
    return clenshaw_run(C, path, psi, c, F.Q, gamma / radius);
}

cheb_status_t cheb_set_fused_split(int n, int l, int h) {
    return fused_set_split(n, l, h) ? CHEB_OK : CHEB_ERR_INVALID_ARG;
}

cheb_status_t cheb_set_fused_split_fp64(int n, int l, int h) {
    return ff_set_split(n, l, h) ? CHEB_OK : CHEB_ERR_INVALID_ARG;
}

cheb_status_t cheb_get_fused_split_fp64(int n, int* l, int* h) {
    if (!l || !h || !ff_supported(n)) return CHEB_ERR_INVALID_ARG;
    FusedPlan p = ff_plan(n);
    *l = p.l;
    *h = p.h;
    return CHEB_OK;
}

cheb_status_t cheb_set_fused_blocking(int on) {
    if (on < -1 || on > 2) return CHEB_ERR_INVALID_ARG;
    fused_set_blocking(on);
    return CHEB_OK;
}

int cheb_get_fused_blocking(void) { return fused_get_blocking(); }

cheb_status_t cheb_set_fused_compensated(int on) {
    if (on != 0 && on != 1) return CHEB_ERR_INVALID_ARG;
    fused_set_compensated(on);
    return CHEB_OK;
}

int cheb_get_fused_compensated(void) { return fused_get_compensated(); }

cheb_status_t cheb_get_fused_split(int n, int* l, int* h) {
    if (!l || !h || !fused_supported(n, 0)) return CHEB_ERR_INVALID_ARG;
    FusedPlan p = fused_plan(n, 0);
    *l = p.l;
    *h = p.h;
    return CHEB_OK;
}

cheb_status_t cheb_workspace_status(void* workspace, size_t workspace_bytes, void* stream) {
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < 256) return CHEB_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int* f = (int*)workspace;  // the status word sits at the start of every workspace layout
    int v = 0;
    CUDA_TRY(cudaMemcpyAsync(&v, f, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(int), s));
    if (v & kFlagTimeout) return CHEB_ERR_TIMEOUT;
    if (v & kFlagBadLaunch) return CHEB_ERR_CUDA;
    return CHEB_OK;
}

cheb_status_t cheb_energy(int n, const double* h, const double* J, const void* psi, cheb_precision_t precision,
                          void* workspace, size_t workspace_bytes, void* stream, double* energy, double* norm2) {
    cheb_status_t st = check_common(n, h, J, precision, workspace, workspace_bytes);
    if (st != CHEB_OK) return st;
    if (!psi || ((uintptr_t)psi & 15) != 0 || !energy || !norm2) return CHEB_ERR_INVALID_ARG;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, (cudaStream_t)stream};
    FixedOp F = make_fixed(n, h, J, 0.0, 1.0);
    st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    launch_norm_energy(precision, n, C.L.M, F.Q, C.tiles(), C.elow(), 0.0, 1.0, psi, C.part(), C.f64out(), C.s);
    CUDA_TRY(cudaGetLastError());
    double ne[2];
    CUDA_TRY(cudaMemcpyAsync(ne, C.f64out(), sizeof(ne), cudaMemcpyDeviceToHost, C.s));
    CUDA_TRY(cudaStreamSynchronize(C.s));
    *norm2 = ne[0];
    *energy = ne[1];
    return CHEB_OK;
}

}  // extern "C"
