// Host coefficient generator: Chebyshev and Caratheodory-Fejer coefficients of
// exp(-i a x) on [-1, 1], and the degree K chosen from the truncation bound.
//
//  * Bessel values J_m(a) by Miller's backward recurrence (Sec. II.B.1) in x86
//    80-bit long double; normalised with the Parseval identity of Eq. cheb,
//    J_0^2 + 2 sum_{m>=1} J_m^2 = 1, the sign fixed by J_0 + 2 sum_k J_{2k} = 1 > 0.
//  * c_0 = J_0(a), c_m = 2 (-i)^m J_m(a) (Eq. cheb with a -> -a, c_0 not halved),
//    times a caller-given phase (exp(-i t c) for the spectral shift of Sec. II.A).
//  * K = the smallest k with sum_{m>k} |c_m| <= tol (Eq. TruncError, |T_m| <= 1).
//  * CF (Sec. II.C): Hankel matrix of the tail, dominant eigenpair (power
//    iteration on H^2, sign split, shifted inverse iteration), Laurent coefficients
//    of the Blaschke error function by the recurrence of Eq. iter with early exit,
//    corrected coefficients p_j = a_j - b_j - b_{-j}.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "cheb_internal.h"

namespace cheb {

// Deepest index needed so that the Miller start does not disturb J_0..J_mmax.
static int miller_start(double a, int mmax) {
    int top = std::max(mmax, (int)std::ceil(a));
    int M = top + 50 + 12 * (int)std::ceil(std::cbrt(a + 1.0));
    return M + (M & 1);
}

void bessel_jn(double a, int mmax, std::vector<double>& out) {
    out.assign(mmax + 1, 0.0);
    const long double x = std::fabs((long double)a);
    if (x == 0.0L) {
        out[0] = 1.0;
        return;
    }
    if (x < 1e-9L) {
        // J_m(x) = (x/2)^m / m! to relative O(x^2)
        long double v = 1.0L;
        for (int m = 0; m <= mmax; ++m) {
            out[m] = (double)v;
            v = v * (x * 0.5L) / (long double)(m + 1);
        }
    } else {
        const int M = miller_start((double)x, mmax);
        std::vector<long double> v(M + 2);
        long double hi = 0.0L, cur = 1e-320L;  // v_{m+1}, v_m
        v[M + 1] = 0.0L;
        v[M] = cur;
        const long double two_over_x = 2.0L / x;
        for (int m = M; m > 0; --m) {
            long double nxt = (long double)m * two_over_x * cur - hi;
            hi = cur;
            cur = nxt;
            v[m - 1] = cur;
            if (std::fabs(cur) > 1e2000L) {
                for (int q = m - 1; q <= M; ++q) v[q] *= 1e-2000L;
                hi *= 1e-2000L;
                cur *= 1e-2000L;
            }
        }
        long double sq = v[0] * v[0], ev = v[0];
        for (int m = 1; m <= M; ++m) {
            sq += 2.0L * v[m] * v[m];
            if ((m & 1) == 0) ev += 2.0L * v[m];
        }
        long double scale = 1.0L / std::sqrt(sq);
        if (ev < 0) scale = -scale;
        for (int m = 0; m <= mmax; ++m) out[m] = (double)(v[m] * scale);
    }
    if (a < 0)
        for (int m = 1; m <= mmax; m += 2) out[m] = -out[m];
}

static int table_length(double a) {
    double x = std::fabs(a);
    return (int)std::ceil(x + 30.0 * std::cbrt(x + 1.0) + 64.0);
}

// ---------------------------------------------------------------------------
// Dominant eigenpair (largest |lambda|) of a small symmetric matrix A (L x L,
// row-major):
//  1. power iteration on A^2, which converges to the span of the eigenvectors of
//     the largest |lambda| even when +|lambda| and -|lambda| are both present;
//  2. split v into its +|lambda| and -|lambda| parts, (|lambda| v +- A v)/2, and
//     keep the larger one;
//  3. polish with shifted inverse iteration (Gaussian elimination with partial
//     pivoting on A - rho I, rho the Rayleigh quotient).
static void matvec(int L, const std::vector<double>& A, const std::vector<double>& x,
                   std::vector<double>& y) {
    for (int i = 0; i < L; ++i) {
        double s = 0.0;
        for (int j = 0; j < L; ++j) s += A[(size_t)i * L + j] * x[j];
        y[i] = s;
    }
}

static double normalise(std::vector<double>& v) {
    double s = 0.0;
    for (double x : v) s += x * x;
    s = std::sqrt(s);
    if (s > 0)
        for (double& x : v) x /= s;
    return s;
}

static bool solve_shifted(int L, const std::vector<double>& A, double rho, std::vector<double> b,
                          std::vector<double>& x) {
    std::vector<double> M(A);
    for (int i = 0; i < L; ++i) M[(size_t)i * L + i] -= rho;
    std::vector<int> piv(L);
    for (int i = 0; i < L; ++i) piv[i] = i;
    double amax = 0.0;
    for (double v : A) amax = std::max(amax, std::fabs(v));
    for (int k = 0; k < L; ++k) {
        int p = k;
        for (int i = k + 1; i < L; ++i)
            if (std::fabs(M[(size_t)i * L + k]) > std::fabs(M[(size_t)p * L + k])) p = i;
        if (p != k) {
            for (int j = 0; j < L; ++j) std::swap(M[(size_t)k * L + j], M[(size_t)p * L + j]);
            std::swap(b[k], b[p]);
        }
        double piv_v = M[(size_t)k * L + k];
        if (std::fabs(piv_v) < 1e-300) piv_v = (piv_v < 0 ? -1.0 : 1.0) * 1e-30 * (amax + 1e-300);
        M[(size_t)k * L + k] = piv_v;
        for (int i = k + 1; i < L; ++i) {
            double f = M[(size_t)i * L + k] / piv_v;
            if (f == 0.0) continue;
            for (int j = k; j < L; ++j) M[(size_t)i * L + j] -= f * M[(size_t)k * L + j];
            b[i] -= f * b[k];
        }
    }
    x.assign(L, 0.0);
    for (int i = L - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < L; ++j) s -= M[(size_t)i * L + j] * x[j];
        x[i] = s / M[(size_t)i * L + i];
    }
    for (double v : x)
        if (!std::isfinite(v)) return false;
    return true;
}

static double dominant_eigenpair(int L, const std::vector<double>& A, std::vector<double>& u) {
    std::vector<double> v(L), t(L), w(L);
    for (int i = 0; i < L; ++i) v[i] = 1.0 / std::sqrt((double)L) * (1.0 + 0.01 * i);
    normalise(v);
    double mu = 0.0;  // estimate of lambda^2
    for (int it = 0; it < 5000; ++it) {
        matvec(L, A, v, t);
        matvec(L, A, t, w);
        double nm = normalise(w);
        double change = 0.0;
        for (int i = 0; i < L; ++i) change = std::max(change, std::fabs(w[i] - v[i]));
        v.swap(w);
        bool done = std::fabs(nm - mu) <= 1e-15 * nm && change < 1e-13;
        mu = nm;
        if (done) break;
    }
    if (mu == 0.0) {
        u.assign(L, 0.0);
        u[0] = 1.0;
        return 0.0;
    }
    const double lam_abs = std::sqrt(mu);
    matvec(L, A, v, t);
    std::vector<double> vp(L), vm(L);
    for (int i = 0; i < L; ++i) {
        vp[i] = 0.5 * (lam_abs * v[i] + t[i]);
        vm[i] = 0.5 * (lam_abs * v[i] - t[i]);
    }
    double np_ = normalise(vp), nm_ = normalise(vm);
    u = (np_ >= nm_) ? vp : vm;
    double rho = (np_ >= nm_) ? lam_abs : -lam_abs;
    for (int it = 0; it < 3; ++it) {
        std::vector<double> x;
        if (!solve_shifted(L, A, rho * (1.0 + 1e-14), u, x)) break;
        normalise(x);
        // keep a consistent sign
        double dot = 0.0;
        for (int i = 0; i < L; ++i) dot += x[i] * u[i];
        if (dot < 0)
            for (double& q : x) q = -q;
        u.swap(x);
        matvec(L, A, u, t);
        double r = 0.0;
        for (int i = 0; i < L; ++i) r += u[i] * t[i];
        rho = r;
    }
    return rho;
}

double cf_correct_real(const std::vector<double>& a, int K, std::vector<double>& p) {
    const int M = (int)a.size() - 1;
    p.assign(K + 1, 0.0);
    // Trim trailing zeros / negligible tail so the Hankel matrix is not padded.
    int top = M;
    while (top > K && a[top] == 0.0) --top;
    const int L = top - K;
    if (L <= 0) {
        for (int j = 0; j <= K && j <= M; ++j) p[j] = a[j];
        return 0.0;
    }
    std::vector<double> Hk((size_t)L * L, 0.0);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            int idx = K + 1 + i + j;
            Hk[(size_t)i * L + j] = (idx <= top) ? a[idx] : 0.0;
        }
    std::vector<double> u;
    const double lambda = dominant_eigenpair(L, Hk, u);
    // Laurent coefficients b_j of the error function (Eq. iter), j from top down to -K.
    const int off = K;
    std::vector<double> b((size_t)top + K + 2, 0.0);
    for (int j = K + 1; j <= top; ++j) b[j + off] = a[j];
    double peak = 0.0;
    for (int j = K + 1; j <= top; ++j) peak = std::max(peak, std::fabs(a[j]));
    int quiet = 0;
    for (int j = K; j >= -K; --j) {
        double s = 0.0;
        for (int k = 1; k < L; ++k) {
            int q = j + k;
            if (q > top) break;
            s += u[k] * b[q + off];
        }
        double v = -s / u[0];
        b[j + off] = v;
        // early exit once the series has decayed far below the error level
        if (std::fabs(v) < 1e-30 * std::max(peak, std::fabs(lambda))) {
            if (++quiet >= L) break;
        } else {
            quiet = 0;
        }
    }
    p[0] = a[0] - b[0 + off];
    for (int j = 1; j <= K; ++j) p[j] = a[j] - b[j + off] - b[-j + off];
    return lambda;
}

// ---------------------------------------------------------------------------
// Remez exchange (Sec. II.C, first method): the best uniform approximation of degree
// <= K to f(x) = cos(a x) (odd = false) or sin(a x) (odd = true) on [-1, 1]. By
// symmetry the best approximation of an even (odd) function is even (odd), so the
// exchange runs in that subspace, spanned by phi_j = T_{2j} (T_{2j+1}), j = 0..J, on
// [0, 1], where it satisfies the Haar condition (for the odd space on (0, 1]: x = 0
// is a common zero of f and p). Each round solves p(x_i) + (-1)^i E = f(x_i) on a
// reference of J + 2 increasing points (dense elimination with partial pivoting) and
// moves the reference to the extrema of f - p, one per run of constant sign (found on
// a Chebyshev-spaced grid, refined by golden section). Stops when max |f - p| is
// within a factor 1 + 1e-7 of |E| (by de la Vallee Poussin's bound the minimax error
// lies between the two, so p is minimax to that factor; tighter is below the rounding
// of f - p at the largest degrees).
// Returns max |f - p| and the Chebyshev coefficients p_0..p_K; -1 on failure.
namespace {

// Gaussian elimination with partial pivoting (A is m x m, row-major); false if singular.
bool solve_dense(int m, std::vector<long double>& A, std::vector<long double>& b) {
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabsl(A[(size_t)r * m + c]) > fabsl(A[(size_t)piv * m + c])) piv = r;
        if (A[(size_t)piv * m + c] == 0.0L) return false;
        if (piv != c) {
            for (int k = 0; k < m; ++k) std::swap(A[(size_t)c * m + k], A[(size_t)piv * m + k]);
            std::swap(b[c], b[piv]);
        }
        const long double d = A[(size_t)c * m + c];
        for (int r = c + 1; r < m; ++r) {
            const long double f = A[(size_t)r * m + c] / d;
            if (f == 0.0L) continue;
            for (int k = c; k < m; ++k) A[(size_t)r * m + k] -= f * A[(size_t)c * m + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = m - 1; c >= 0; --c) {
        long double acc = b[c];
        for (int k = c + 1; k < m; ++k) acc -= A[(size_t)c * m + k] * b[k];
        b[c] = acc / A[(size_t)c * m + c];
    }
    return true;
}

}  // namespace

double remez_real(bool odd, double a_in, int K, std::vector<double>& p) {
    const long double a = a_in, pi = 3.141592653589793238462643383279502884L;
    auto f = [&](long double t) { return odd ? sinl(a * t) : cosl(a * t); };
    const int par = odd ? 1 : 0;
    const int J = odd ? (K - 1) / 2 : K / 2;  // highest index j with 2j + par <= K
    p.assign(K + 1, 0.0);
    // phi_j(x) = T_{2j+par}(x) for j = 0..J at one point, by the three-term recurrence
    auto basis = [&](long double x, std::vector<long double>& out) {
        long double t0 = 1.0L, t1 = x;
        int deg = 0;
        for (int j = 0; j <= J; ++j) {
            const int want = 2 * j + par;
            while (deg < want) {
                const long double t2 = 2.0L * x * t1 - t0;
                t0 = t1;
                t1 = t2;
                ++deg;
            }
            out[j] = t0;
        }
    };
    const int G = 8 * (J + 2) + 64;
    std::vector<long double> tg(G + 1);
    for (int g = 0; g <= G; ++g) tg[g] = cosl(pi * (G - g) / (2.0L * G));  // 0 .. 1, increasing
    if (J < 0) {  // no odd term allowed (K = 0): p = 0
        long double m0 = 0.0L;
        for (int g = 0; g <= G; ++g) m0 = std::max(m0, fabsl(f(tg[g])));
        return (double)m0;
    }
    const int m = J + 2;
    std::vector<long double> x(m), c(J + 1, 0.0L), phi(J + 1);
    // initial reference: extrema of T_{2J+2+par} in [0, 1] (those > 0 for odd f)
    for (int i = 0; i < m; ++i) x[i] = cosl(pi * (m - 1 - i) / (2.0L * m - 2.0L + 2.0L * par));
    auto P = [&](long double t) {
        basis(t, phi);
        long double acc = 0.0L;
        for (int j = 0; j <= J; ++j) acc += c[j] * phi[j];
        return acc;
    };
    long double emax = 0.0L;
    for (int it = 0; it < 60; ++it) {
        std::vector<long double> A((size_t)m * m), b(m);
        for (int i = 0; i < m; ++i) {
            basis(x[i], phi);
            for (int j = 0; j <= J; ++j) A[(size_t)i * m + j] = phi[j];
            A[(size_t)i * m + J + 1] = (i & 1) ? -1.0L : 1.0L;
            b[i] = f(x[i]);
        }
        if (!solve_dense(m, A, b)) return -1.0;
        for (int j = 0; j <= J; ++j) c[j] = b[j];
        const long double E = b[J + 1];
        auto err = [&](long double t) { return f(t) - P(t); };
        std::vector<long double> eg(G + 1);
        long double gmax = 0.0L;
        for (int g = 0; g <= G; ++g) {
            eg[g] = err(tg[g]);
            gmax = std::max(gmax, fabsl(eg[g]));
        }
        if (gmax <= 1e-17L) {  // f is (up to rounding) in the space
            emax = gmax;
            break;
        }
        // extrema, one per run of constant sign (the odd error vanishes at x = 0: skip it)
        std::vector<long double> ex, ev;
        int g = odd ? 1 : 0;
        while (g <= G) {
            const bool pos = eg[g] >= 0.0L;
            int best = g, h = g;
            while (h <= G && ((eg[h] >= 0.0L) == pos)) {
                if (fabsl(eg[h]) > fabsl(eg[best])) best = h;
                ++h;
            }
            long double lo = tg[std::max(best - 1, g)], hi = tg[std::min(best + 1, h - 1)];
            long double xb = tg[best], eb = eg[best];
            if (hi > lo) {
                const long double gr = 0.6180339887498948482L;
                long double c1 = hi - gr * (hi - lo), c2 = lo + gr * (hi - lo);
                long double f1 = fabsl(err(c1)), f2 = fabsl(err(c2));
                for (int r = 0; r < 24; ++r) {  // the error is flat at its extremum
                    if (f1 > f2) {
                        hi = c2;
                        c2 = c1;
                        f2 = f1;
                        c1 = hi - gr * (hi - lo);
                        f1 = fabsl(err(c1));
                    } else {
                        lo = c1;
                        c1 = c2;
                        f1 = f2;
                        c2 = lo + gr * (hi - lo);
                        f2 = fabsl(err(c2));
                    }
                }
                const long double xc = 0.5L * (lo + hi), ec = err(xc);
                if (fabsl(ec) > fabsl(eb) && ((ec >= 0.0L) == pos)) {
                    xb = xc;
                    eb = ec;
                }
            }
            ex.push_back(xb);
            ev.push_back(eb);
            g = h;
        }
        if ((int)ex.size() < m) return -1.0;
        size_t lo_i = 0, hi_i = ex.size();  // keep m alternating extrema: drop the smaller end
        while (hi_i - lo_i > (size_t)m) {
            if (fabsl(ev[lo_i]) < fabsl(ev[hi_i - 1])) ++lo_i;
            else --hi_i;
        }
        emax = 0.0L;
        for (size_t i = 0; i < ev.size(); ++i) emax = std::max(emax, fabsl(ev[i]));
        for (int i = 0; i < m; ++i) x[i] = ex[lo_i + i];
        if (emax - fabsl(E) <= 1e-7L * emax) break;
    }
    for (int j = 0; j <= J; ++j) p[2 * j + par] = (double)c[j];
    return (double)emax;
}

// ---------------------------------------------------------------------------
int make_coefficients(double a, std::complex<double> phase, double tol, int method, int max_K,
                      std::vector<std::complex<double>>& c, double* err_bound) {
    const int T = table_length(a);
    std::vector<double> jm;
    bessel_jn(a, T, jm);
    std::vector<double> mag(T + 1);
    for (int m = 0; m <= T; ++m) mag[m] = (m == 0 ? 1.0 : 2.0) * std::fabs(jm[m]);
    // suffix sums from the small end: tail(k) = sum_{m>k} |c_m|
    std::vector<double> tail(T + 2, 0.0);
    for (int m = T; m >= 0; --m) tail[m] = tail[m + 1] + mag[m];
    int K = 0;
    while (K < T && tail[K + 1] > tol) ++K;
    double err = tail[K + 1];
    if (method == 0) {
        if (K > max_K) return -1;
        c.resize(K + 1);
        std::complex<double> rot(1.0, 0.0);
        for (int m = 0; m <= K; ++m) {
            c[m] = (m == 0 ? 1.0 : 2.0) * jm[m] * rot * phase;
            rot *= std::complex<double>(0.0, -1.0);
        }
        if (err_bound) *err_bound = err;
        return K;
    }
    // CF: cos(a x) and sin(a x) separately, then p = p_cos - i p_sin.
    std::vector<double> ac(T + 1, 0.0), as(T + 1, 0.0);
    for (int m = 0; m <= T; ++m) {
        double v = (m == 0 ? 1.0 : 2.0) * jm[m] * (((m >> 1) & 1) ? -1.0 : 1.0);
        if (m & 1) as[m] = v; else ac[m] = v;
    }
    if (method == 2) {
        // Remez: the degree comes from the CF estimate of the minimax error (cheap);
        // the exchange then runs at that degree, and one degree more while its
        // combined error hypot(E_cos, E_sin) exceeds tol (the Chebyshev degree always
        // suffices: the minimax error is below the series' truncation error).
        std::vector<double> qc, qs;
        const int Kcheb = K;
        while (K > 0) {
            const double lc2 = cf_correct_real(ac, K - 1, qc), ls2 = cf_correct_real(as, K - 1, qs);
            if (!(std::hypot(lc2, ls2) <= tol)) break;
            --K;
        }
        std::vector<double> pc, ps;
        for (;; ++K) {
            const double ec = remez_real(false, a, K, pc), es = remez_real(true, a, K, ps);
            if (ec < 0 || es < 0) return -1;
            err = std::hypot(ec, es);
            if (err <= tol || K >= Kcheb) break;
        }
        if (K > max_K) return -1;
        c.resize(K + 1);
        for (int m = 0; m <= K; ++m) c[m] = std::complex<double>(pc[m], -ps[m]) * phase;
        if (err_bound) *err_bound = err;
        return K;
    }
    std::vector<double> pc, ps, qc, qs;
    double lc = cf_correct_real(ac, K, pc), ls = cf_correct_real(as, K, ps);
    err = std::hypot(lc, ls);
    while (K > 0) {
        double lc2 = cf_correct_real(ac, K - 1, qc), ls2 = cf_correct_real(as, K - 1, qs);
        double e2 = std::hypot(lc2, ls2);
        if (!(e2 <= tol)) break;
        --K;
        pc.swap(qc);
        ps.swap(qs);
        err = e2;
    }
    if (K > max_K) return -1;
    c.resize(K + 1);
    for (int m = 0; m <= K; ++m) c[m] = std::complex<double>(pc[m], -ps[m]) * phase;
    if (err_bound) *err_bound = err;
    return K;
}

// Monomial -> Chebyshev basis (Sec. II.B, the two bases of the series): with
// P_m = x^m = sum_k p_{m,k} T_k, the next power follows from x T_0 = T_1 and
// x T_k = (T_{k+1} + T_{k-1}) / 2; c = sum_m a_m P_m. Long double, O(K^2).
void monomial_to_chebyshev(int K, const std::complex<double>* a, std::complex<double>* c) {
    std::vector<long double> P(K + 2, 0.0L), Q(K + 2, 0.0L);
    std::vector<long double> cr(K + 1, 0.0L), ci(K + 1, 0.0L);
    P[0] = 1.0L;  // x^0 = T_0
    for (int m = 0; m <= K; ++m) {
        const long double ar = a[m].real(), ai = a[m].imag();
        for (int k = 0; k <= m; ++k) {
            cr[k] += ar * P[k];
            ci[k] += ai * P[k];
        }
        if (m == K) break;
        std::fill(Q.begin(), Q.end(), 0.0L);
        Q[1] += P[0];
        for (int k = 1; k <= m; ++k) {
            Q[k + 1] += 0.5L * P[k];
            Q[k - 1] += 0.5L * P[k];
        }
        P.swap(Q);
    }
    for (int k = 0; k <= K; ++k) c[k] = std::complex<double>((double)cr[k], (double)ci[k]);
}

}  // namespace cheb
