// Oracle for exp(-itH)psi by a truncated Chebyshev (or Caratheodory-Fejer) series
// evaluated with the matrix Clenshaw recurrence.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, FP64 reference that the
// CUDA path is checked against. It shares no code, header, table or helper with
// the CUDA library, and the library never calls it. Only the tests, the smoke
// check and the CPU-baseline leg of the benchmark load it.
//
// Everything here is written for readability, not speed: every energy is a
// brute-force double loop over the couplings, every matvec is an explicit loop
// over elements and bit flips, and the Bessel values come from Miller's backward
// recurrence in x86 80-bit long double. The one concession to speed is an OpenMP
// parallel-for over the elements of a vector; the arithmetic done for each element
// (and its order) does not depend on the thread count, so results are deterministic.
//
// Problem (Sec. I): H = H_P + gamma * H_G on n qubits, N = 2^n,
//   H_G = sum_j X_j  (X_j flips bit j of the basis index z),
//   H_P = diag(E(z)),  E(z) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i,  s_i = 1 - 2*bit_i(z).
// Qubit i is bit i of z (least significant bit first); only the strict upper
// triangle (i<j) of the row-major n x n matrix J is read.
//
// Parity status of each function is listed in oracle.py's header.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

typedef std::complex<double> cplx;

extern "C" {

// ---------------------------------------------------------------------------
// Ising diagonal (Sec. I; the SK instances of Fig. 3 / Fig. 4).
// E(z) by the defining double sum, for one z.
static double energy_of(int n, const double* h, const double* J, uint64_t z) {
    double e = 0.0;
    for (int i = 0; i < n; ++i) {
        double si = ((z >> i) & 1) ? -1.0 : 1.0;
        e += h[i] * si;
        for (int j = i + 1; j < n; ++j) {
            double sj = ((z >> j) & 1) ? -1.0 : 1.0;
            e += J[(size_t)i * n + j] * si * sj;
        }
    }
    return e;
}

// All 2^n energies, brute force.
void oracle_energies(int n, const double* h, const double* J, double* E) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z) E[z] = energy_of(n, h, J, (uint64_t)z);
}

// Spectral interval of Sec. II.A: the induced L1 norm of the shifted H.
// The diagonal is shifted by c = (Emax+Emin)/2 so its range is symmetric; each
// column of the shifted H then has absolute sum |E(z)-c| + gamma*n, so
// ||H - c||_1 = (Emax-Emin)/2 + |gamma|*n = r.  out = {Emin, Emax, c, r}.
void oracle_bounds(int n, const double* h, const double* J, double gamma, double* out) {
    const int64_t N = (int64_t)1 << n;
    double emin = energy_of(n, h, J, 0), emax = emin;
    for (int64_t z = 1; z < N; ++z) {
        double e = energy_of(n, h, J, (uint64_t)z);
        emin = std::min(emin, e);
        emax = std::max(emax, e);
    }
    out[0] = emin;
    out[1] = emax;
    out[2] = 0.5 * (emax + emin);
    out[3] = 0.5 * (emax - emin) + std::fabs(gamma) * n;
}

// ---------------------------------------------------------------------------
// Bessel functions J_m(a), m = 0..mmax, by Miller's backward recurrence
// (Sec. II.B.1), in 80-bit long double.
// Start: an even index M well past both mmax and the turning point m ~ a, where
// J_m has decayed far below anything kept; set J_{M+1} = 0, J_M = tiny and run
// J_{m-1} = (2m/a) J_m - J_{m+1} down to m = 0. Normalise with the identity
// J_0 + 2 sum_{k>=1} J_{2k} = 1, which is Eq. cheb evaluated at x = 0
// (T_{2k}(0) = (-1)^k cancels i^{2k}, odd T_m(0) vanish); it holds for every real a.
void oracle_bessel_j(double a_in, int mmax, double* out) {
    long double a = (long double)std::fabs(a_in);
    if (a < 1e-8L) {
        // Leading term of the power series: J_m(a) = (a/2)^m / m! (1 + O(a^2)).
        long double term = 1.0L;
        for (int m = 0; m <= mmax; ++m) {
            out[m] = (double)term;
            term *= (a / 2.0L) / (long double)(m + 1);
        }
    } else {
        double ad = (double)a;
        int M = (int)std::ceil(std::max(ad + 20.0 * std::cbrt(ad) + 40.0, (double)mmax + 40.0));
        if (M % 2) M += 1;
        std::vector<long double> j(M + 2, 0.0L);
        j[M + 1] = 0.0L;
        j[M] = 1e-300L;
        for (int m = M; m >= 1; --m) {
            j[m - 1] = (2.0L * m / a) * j[m] - j[m + 1];
            if (std::fabs(j[m - 1]) > 1e300L) {  // rescale to stay in range
                for (int q = m - 1; q <= M; ++q) j[q] *= 1e-300L;
            }
        }
        long double norm = j[0];
        for (int k = 2; k <= M; k += 2) norm += 2.0L * j[k];
        for (int m = 0; m <= mmax; ++m) out[m] = (double)(j[m] / norm);
    }
    // J_m(-a) = (-1)^m J_m(a)
    if (a_in < 0)
        for (int m = 1; m <= mmax; m += 2) out[m] = -out[m];
}

// ---------------------------------------------------------------------------
// Chebyshev coefficients of f(x) = exp(-i a x) on [-1, 1] (Eq. cheb with a -> -a):
//   f(x) = J_0(a) + 2 sum_{m>=1} (-i)^m J_m(a) T_m(x),
// c_0 is the full J_0(a) (not halved), as in Eq. cheb and Algorithm 2.
// The returned coefficients are multiplied by the global phase `phase` (complex,
// e^{-itc} for the shifted spectrum of Sec. II.A).
// Degree K: the smallest k with sum_{m=k+1}^{M} |c_m| <= tol (Eq. TruncError with
// |T_m| <= 1), where M is the last index computed (the tail beyond it is
// below 1e-40 relative).
// coeffs: 2*(maxK+1) doubles (re, im). Returns K, or -1 if K would exceed maxK.
int oracle_cheb_coeffs(double a, double phase_re, double phase_im, double tol, int maxK,
                       double* coeffs, double* trunc_bound) {
    double aa = std::fabs(a);
    int mmax = (int)std::ceil(aa + 25.0 * std::cbrt(aa + 1.0) + 60.0);
    std::vector<double> jm(mmax + 1);
    oracle_bessel_j(a, mmax, jm.data());
    // |c_m| for the tail test
    std::vector<double> mag(mmax + 1);
    mag[0] = std::fabs(jm[0]);
    for (int m = 1; m <= mmax; ++m) mag[m] = 2.0 * std::fabs(jm[m]);
    // tail[k] = sum_{m>k} |c_m|, summed from the small end
    std::vector<double> tail(mmax + 1, 0.0);
    double s = 0.0;
    for (int k = mmax; k >= 0; --k) {
        tail[k] = s;
        s += mag[k];
    }
    int K = 0;
    while (K < mmax && tail[K] > tol) ++K;
    if (K > maxK) return -1;
    cplx phase(phase_re, phase_im);
    cplx mi_pow(1.0, 0.0);  // (-i)^m
    for (int m = 0; m <= K; ++m) {
        double w = (m == 0) ? 1.0 : 2.0;
        cplx c = w * jm[m] * mi_pow * phase;
        coeffs[2 * m] = c.real();
        coeffs[2 * m + 1] = c.imag();
        mi_pow *= cplx(0.0, -1.0);
    }
    if (trunc_bound) *trunc_bound = tail[K];
    return K;
}

// ---------------------------------------------------------------------------
// Caratheodory-Fejer near-minimax approximation (Sec. II.C) of a real function
// given by its Chebyshev coefficients a[0..M]: degree K.
// Steps, in the paper's order:
//  1. Hankel matrix of the tail coefficients, Hk[i][j] = a[K+1+i+j], 0 <= i,j < L,
//     L = M - K (entries past M are zero).
//  2. Eigenpair (lambda, u) of largest |lambda| (cyclic Jacobi here).
//  3. Laurent coefficients of the error function by the downward recurrence of
//     Eq. iter: b_j = a_j for j > K, then
//        b_j = -(1/u_0) sum_{k=1}^{L-1} u_k b_{j+k},   j = K, K-1, ..., -K.
//  4. Corrected coefficients p_0 = a_0 - b_0, p_j = a_j - b_j - b_{-j} (1 <= j <= K);
//     the error f - p is then the real part of a Blaschke product of modulus |lambda|.
// Returns lambda; p has K+1 entries.
static void jacobi_eigen(int L, std::vector<double>& A, std::vector<double>& V, std::vector<double>& w) {
    // Cyclic Jacobi rotations on the symmetric L x L matrix A (row-major).
    V.assign((size_t)L * L, 0.0);
    for (int i = 0; i < L; ++i) V[(size_t)i * L + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) {
                if (i != j) off += A[(size_t)i * L + j] * A[(size_t)i * L + j];
                else diag += A[(size_t)i * L + j] * A[(size_t)i * L + j];
            }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < L - 1; ++p)
            for (int q = p + 1; q < L; ++q) {
                double apq = A[(size_t)p * L + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * L + p], aqq = A[(size_t)q * L + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < L; ++k) {  // rotate columns p, q
                    double akp = A[(size_t)k * L + p], akq = A[(size_t)k * L + q];
                    A[(size_t)k * L + p] = c * akp - s * akq;
                    A[(size_t)k * L + q] = s * akp + c * akq;
                }
                for (int k = 0; k < L; ++k) {  // rotate rows p, q
                    double apk = A[(size_t)p * L + k], aqk = A[(size_t)q * L + k];
                    A[(size_t)p * L + k] = c * apk - s * aqk;
                    A[(size_t)q * L + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < L; ++k) {
                    double vkp = V[(size_t)k * L + p], vkq = V[(size_t)k * L + q];
                    V[(size_t)k * L + p] = c * vkp - s * vkq;
                    V[(size_t)k * L + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(L);
    for (int i = 0; i < L; ++i) w[i] = A[(size_t)i * L + i];
}

double oracle_cf_real(int M, const double* a, int K, double* p) {
    int L = M - K;
    if (L <= 0) {  // nothing to correct
        for (int j = 0; j <= K; ++j) p[j] = (j <= M) ? a[j] : 0.0;
        return 0.0;
    }
    std::vector<double> Hk((size_t)L * L, 0.0);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            int idx = K + 1 + i + j;
            Hk[(size_t)i * L + j] = (idx <= M) ? a[idx] : 0.0;
        }
    std::vector<double> V, w;
    jacobi_eigen(L, Hk, V, w);
    int best = 0;
    for (int i = 1; i < L; ++i)
        if (std::fabs(w[i]) > std::fabs(w[best])) best = i;
    double lambda = w[best];
    std::vector<double> u(L);
    for (int i = 0; i < L; ++i) u[i] = V[(size_t)i * L + best];
    // b_j stored at offset: index j in [-K, M] -> b[j + K]
    std::vector<double> b((size_t)(M + K + 1 + L), 0.0);
    auto B = [&](int j) -> double& { return b[(size_t)(j + K)]; };
    for (int j = K + 1; j <= M; ++j) B(j) = a[j];
    for (int j = K; j >= -K; --j) {
        double s = 0.0;
        for (int k = 1; k < L; ++k) s += u[k] * ((j + k <= M) ? B(j + k) : 0.0);
        B(j) = -s / u[0];
    }
    p[0] = a[0] - B(0);
    for (int j = 1; j <= K; ++j) p[j] = a[j] - B(j) - B(-j);
    return lambda;
}

// CF coefficients for f(x) = exp(-i a x) (times `phase`): cos(ax) and sin(ax) are
// real and handled separately (cos(ax) = J_0 + 2 sum (-1)^k J_{2k} T_{2k},
// sin(ax) = 2 sum (-1)^k J_{2k+1} T_{2k+1}), then combined as p = p_cos - i p_sin.
// Degree: the smallest K <= K_cheb (the Chebyshev degree for tol) whose error
// estimate sqrt(lambda_cos^2 + lambda_sin^2) is <= tol (the two real error curves
// are bounded by |lambda_cos| and |lambda_sin| pointwise, so the complex error
// |e_cos - i e_sin| is bounded by their root-sum-square). Returns K (or -1) and
// writes the estimate to err_est.
int oracle_cf_coeffs(double a, double phase_re, double phase_im, double tol, int maxK,
                     double* coeffs, double* err_est) {
    double aa = std::fabs(a);
    int M = (int)std::ceil(aa + 25.0 * std::cbrt(aa + 1.0) + 60.0);
    std::vector<double> jm(M + 1);
    oracle_bessel_j(a, M, jm.data());
    std::vector<double> ac(M + 1, 0.0), as(M + 1, 0.0);
    for (int m = 0; m <= M; ++m) {
        double sgn = ((m / 2) % 2) ? -1.0 : 1.0;  // (-1)^{floor(m/2)}
        double w = (m == 0) ? 1.0 : 2.0;
        if (m % 2 == 0) ac[m] = w * sgn * jm[m];
        else as[m] = w * sgn * jm[m];
    }
    // Chebyshev degree as the starting point
    std::vector<double> tmp(2 * (M + 1));
    int Kc = oracle_cheb_coeffs(a, 1.0, 0.0, tol, M, tmp.data(), nullptr);
    if (Kc < 0) return -1;
    std::vector<double> pc(M + 1), ps(M + 1);
    int K = Kc;
    double err = 0.0;
    {
        double lc = oracle_cf_real(M, ac.data(), K, pc.data());
        double ls = oracle_cf_real(M, as.data(), K, ps.data());
        err = std::hypot(lc, ls);
    }
    while (K > 0) {
        std::vector<double> qc(M + 1), qs(M + 1);
        double lc = oracle_cf_real(M, ac.data(), K - 1, qc.data());
        double ls = oracle_cf_real(M, as.data(), K - 1, qs.data());
        double e = std::hypot(lc, ls);
        if (e > tol) break;
        K -= 1;
        pc = qc;
        ps = qs;
        err = e;
    }
    if (K > maxK) return -1;
    cplx phase(phase_re, phase_im);
    for (int m = 0; m <= K; ++m) {
        cplx c = cplx(pc[m], -ps[m]) * phase;
        coeffs[2 * m] = c.real();
        coeffs[2 * m + 1] = c.imag();
    }
    if (err_est) *err_est = err;
    return K;
}

// ---------------------------------------------------------------------------
// Matrix-free application of the scaled operator (Sec. II.D):
//   (Ht v)(z) = D(z) v(z) + g * sum_{j<n} v(z xor 2^j),
// with D(z) = (E(z) - c)/r and g = gamma/r, so that ||Ht||_1 <= 1.
static void apply_ht(int n, const double* D, double g, const cplx* v, cplx* out) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; ++z) {
        cplx s(0.0, 0.0);
        for (int j = 0; j < n; ++j) s += v[z ^ ((int64_t)1 << j)];
        out[z] = D[z] * v[z] + g * s;
    }
}

// Matrix Clenshaw recurrence (Algorithm 2; Eq. recursion):
//   b_{K+1} = 0, b_K = c_K psi,
//   b_k = 2 Ht b_{k+1} - b_{k+2} + c_k psi,   k = K-1, ..., 1,
//   y   = Ht b_1 - b_2 + c_0 psi.
// K = 0 gives y = c_0 psi (the printed listing mishandles a single coefficient).
// If norms != nullptr it receives the A14 ingredients per step k = 0..K:
//   norms[3k+0] = ||b_k||, norms[3k+1] = ||c_k psi - b_{k+2}||, norms[3k+2] = ||b_{k+1}||.
void oracle_clenshaw(int n, const double* D, double g, int K, const double* coeffs,
                     const double* psi_in, double* y_out, double* norms) {
    const int64_t N = (int64_t)1 << n;
    const cplx* psi = reinterpret_cast<const cplx*>(psi_in);
    cplx* y = reinterpret_cast<cplx*>(y_out);
    std::vector<cplx> ck(K + 1);
    for (int m = 0; m <= K; ++m) ck[m] = cplx(coeffs[2 * m], coeffs[2 * m + 1]);
    auto nrm = [&](const std::vector<cplx>& v) {
        double s = 0.0;
        for (int64_t z = 0; z < N; ++z) s += std::norm(v[z]);
        return std::sqrt(s);
    };
    if (K == 0) {
        for (int64_t z = 0; z < N; ++z) y[z] = ck[0] * psi[z];
        if (norms) { norms[0] = nrm(std::vector<cplx>(y, y + N)); norms[1] = norms[0]; norms[2] = 0.0; }
        return;
    }
    std::vector<cplx> b1(N), b2(N, cplx(0.0, 0.0)), hb(N);   // b1 = b_{k+1}, b2 = b_{k+2}
    for (int64_t z = 0; z < N; ++z) b1[z] = ck[K] * psi[z];
    if (norms) { norms[3 * K + 0] = nrm(b1); norms[3 * K + 1] = norms[3 * K + 0]; norms[3 * K + 2] = 0.0; }
    std::vector<cplx> tmp(N);
    for (int k = K - 1; k >= 1; --k) {
        apply_ht(n, D, g, b1.data(), hb.data());
        std::vector<cplx> bk(N);
        for (int64_t z = 0; z < N; ++z) bk[z] = 2.0 * hb[z] - b2[z] + ck[k] * psi[z];
        if (norms) {
            for (int64_t z = 0; z < N; ++z) tmp[z] = ck[k] * psi[z] - b2[z];
            norms[3 * k + 0] = nrm(bk);
            norms[3 * k + 1] = nrm(tmp);
            norms[3 * k + 2] = nrm(b1);
        }
        b2.swap(b1);   // b2 <- b_{k+1}
        b1.swap(bk);   // b1 <- b_k
    }
    apply_ht(n, D, g, b1.data(), hb.data());
    for (int64_t z = 0; z < N; ++z) y[z] = hb[z] - b2[z] + ck[0] * psi[z];
    if (norms) {
        std::vector<cplx> yy(y, y + N);
        for (int64_t z = 0; z < N; ++z) tmp[z] = ck[0] * psi[z] - b2[z];
        norms[0] = nrm(yy);
        norms[1] = nrm(tmp);
        norms[2] = nrm(b1);
    }
}

// A polynomial given in the monomial basis (the other basis of Sec. II.B), by its
// definition: y = sum_{m=0}^{K} a_m Ht^m psi, with the powers formed by repeated
// matvecs (no basis change, no recurrence).
void oracle_monomial_apply(int n, const double* D, double g, int K, const double* a,
                           const double* psi_in, double* y_out) {
    const int64_t N = (int64_t)1 << n;
    const cplx* psi = reinterpret_cast<const cplx*>(psi_in);
    cplx* y = reinterpret_cast<cplx*>(y_out);
    std::vector<cplx> pw(psi, psi + N), nx(N);   // pw = Ht^m psi
    for (int64_t z = 0; z < N; ++z) y[z] = cplx(0.0, 0.0);
    for (int m = 0; m <= K; ++m) {
        const cplx am(a[2 * m], a[2 * m + 1]);
        for (int64_t z = 0; z < N; ++z) y[z] += am * pw[z];
        if (m == K) break;
        apply_ht(n, D, g, pw.data(), nx.data());
        pw.swap(nx);
    }
}

// Evaluation-error bound of Sec. II.B.3 for a run whose per-step norms are given:
//   sum_k  u ||b_k|| + u ||c_k psi - b_{k+2}|| + sqrt(d) gamma_d ||b_{k+1}||,
//   gamma_d = d u / (1 - d u),  d = n + 1 nonzeros per column (Sec. I).
double oracle_eval_bound(int n, int K, const double* norms, double u) {
    double d = n + 1.0;
    double gd = d * u / (1.0 - d * u);
    double s = 0.0;
    for (int k = 0; k <= K; ++k)
        s += u * norms[3 * k] + u * norms[3 * k + 1] + std::sqrt(d) * gd * norms[3 * k + 2];
    return s;
}

// ---------------------------------------------------------------------------
// Full pipeline: psi_out ~= exp(-i t H) psi_in.
//  1. energies E(z) and bounds c, r (Sec. II.A);
//  2. for each of `splits` equal time slices (exp(-itH) = exp(-i(t/s)H)^s):
//     a = (t/s) r, coefficients for exp(-i a x) times exp(-i (t/s) c) with
//     tolerance tol/s (Chebyshev: Eq. cheb + Eq. TruncError; CF: Sec. II.C),
//     then Clenshaw (Algorithm 2) with the scaled operator.
// info (12 doubles): {K (per slice), Emin, Emax, c, r, a (per slice), trunc bound
//  (summed), eval bound for u = 2^-53 (summed), ||y||, <y|H_P|y>, splits, 0}.
// Returns 0 on success, -1 on invalid input.
int oracle_expmv(int n, const double* h, const double* J, double gamma, double t,
                 double tol, int method, int splits, const double* psi_in, double* psi_out,
                 double* info) {
    if (n < 1 || n > 34 || !(tol > 0) || splits < 1 || (method != 0 && method != 1)) return -1;
    const int64_t N = (int64_t)1 << n;
    std::vector<double> E(N), D(N);
    oracle_energies(n, h, J, E.data());
    double emin = E[0], emax = E[0];
    for (int64_t z = 1; z < N; ++z) { emin = std::min(emin, E[z]); emax = std::max(emax, E[z]); }
    double c = 0.5 * (emax + emin);
    double r = 0.5 * (emax - emin) + std::fabs(gamma) * n;
    if (r <= 0) r = 1.0;  // H = 0 when gamma = 0 and E is constant; any r works
    for (int64_t z = 0; z < N; ++z) D[z] = (E[z] - c) / r;
    double g = gamma / r;
    double ts = t / splits;
    double a = ts * r;
    double phre = std::cos(-ts * c), phim = std::sin(-ts * c);
    int maxK = (int)std::ceil(std::fabs(a) + 25.0 * std::cbrt(std::fabs(a) + 1.0) + 60.0);
    std::vector<double> coeffs(2 * (maxK + 1));
    double tb = 0.0;
    int K = (method == 0) ? oracle_cheb_coeffs(a, phre, phim, tol / splits, maxK, coeffs.data(), &tb)
                          : oracle_cf_coeffs(a, phre, phim, tol / splits, maxK, coeffs.data(), &tb);
    if (K < 0) return -1;
    std::vector<double> cur(psi_in, psi_in + 2 * N), nxt(2 * N);
    std::vector<double> norms(3 * (K + 1));
    double eb = 0.0;
    for (int s = 0; s < splits; ++s) {
        oracle_clenshaw(n, D.data(), g, K, coeffs.data(), cur.data(), nxt.data(), norms.data());
        eb += oracle_eval_bound(n, K, norms.data(), std::ldexp(1.0, -53));
        cur.swap(nxt);
    }
    std::memcpy(psi_out, cur.data(), sizeof(double) * 2 * N);
    double nn = 0.0, en = 0.0;
    for (int64_t z = 0; z < N; ++z) {
        double p2 = cur[2 * z] * cur[2 * z] + cur[2 * z + 1] * cur[2 * z + 1];
        nn += p2;
        en += E[z] * p2;
    }
    if (info) {
        info[0] = K; info[1] = emin; info[2] = emax; info[3] = c; info[4] = r; info[5] = a;
        info[6] = tb * splits; info[7] = eb; info[8] = std::sqrt(nn); info[9] = en;
        info[10] = splits; info[11] = 0.0;
    }
    return 0;
}

// <psi|H_P|psi> and ||psi||^2 by brute force. out = {energy, norm^2}.
void oracle_energy_norm(int n, const double* h, const double* J, const double* psi, double* out) {
    const int64_t N = (int64_t)1 << n;
    double en = 0.0, nn = 0.0;
    for (int64_t z = 0; z < N; ++z) {
        double p2 = psi[2 * z] * psi[2 * z] + psi[2 * z + 1] * psi[2 * z + 1];
        nn += p2;
        en += energy_of(n, h, J, (uint64_t)z) * p2;
    }
    out[0] = en;
    out[1] = nn;
}

}  // extern "C"
