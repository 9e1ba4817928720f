// Reverse-mode gradients of exp(-itH) psi and of annealing schedules.
//
// Forward (Algorithm 2, Eq. recursion): b_{K+1} = 0, b_K = c_K psi,
//   b_k = 2 Ht b_{k+1} - b_{k+2} + c_k psi (k = K-1..1),  y = Ht b_1 - b_2 + c_0 psi.
// For a real loss L with ybar = dL/dy (the convention of torch autograd for complex
// tensors: dL = Re<ybar, dy>), reversing those assignments gives
//   bbar_0 = ybar, bbar_1 = Ht bbar_0, bbar_k = 2 Ht bbar_{k-1} - bbar_{k-2}  (so
//   bbar_k = T_k(Ht) ybar), psibar = sum_k conj(c_k) bbar_k = p(Ht)^H ybar, and
//   dL = Re sum_{k=0}^{K-1} w_k <bbar_k, dHt b_{k+1}>,  w_0 = 1, w_k = 2.
// With Ht = D + g sum_j X_j, D = (E - c)/r, g = gamma/r, and the spectral interval
// (c, r) held fixed (the exact exp(-itH) does not depend on it):
//   dL/dD(z)  = G(z) = Re sum_k w_k conj(bbar_k(z)) b_{k+1}(z),
//   dL/dgamma = (1/r) Re sum_k w_k <bbar_k, (sum_j X_j) b_{k+1}>,
//   dL/dh_i   = (1/r) sum_z G(z) s_i(z),  dL/dJ_ij = (1/r) sum_z G(z) s_i(z) s_j(z),
//   dL/dt     = Im <ybar, H y>            (from dy/dt = -i H y).
// The b_k are needed in increasing k while the forward produces them decreasing;
// they are regenerated upward, b_{k+2} = 2 Ht b_{k+1} - b_k + c_k psi, from (b_1, b_2),
// and reset every C steps from anchor pairs saved by a forward recomputation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "fused.cuh"
#include "kernels.cuh"
#include "pipeline.h"

namespace cheb {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ int64_t sgn_sel(uint64_t bit, int64_t v) { return bit ? -v : v; }

__device__ __forceinline__ int64_t energy_fx(int M, const int64_t* __restrict__ tiles, const int64_t* __restrict__ elow,
                                             uint64_t z) {
    const uint64_t T = z >> M;
    const uint64_t x = z & ((1ull << M) - 1);
    const int64_t* row = tiles + T * (M + 1);
    int64_t e = __ldg(row + M) + __ldg(elow + x);
    for (int i = 0; i < M; ++i) e += sgn_sel((x >> i) & 1, __ldg(row + i));
    return e;
}

constexpr int kAdjThreads = 256;

// Block-level FP64 sum into slot[blockIdx.x] (accumulated, fixed order).
__device__ __forceinline__ void block_accumulate(double v, double* slot) {
    __shared__ double red[kAdjThreads];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) slot[blockIdx.x] += red[0];
}

struct AdjArgs {
    int n, M, Q;
    const int64_t* tiles;
    const int64_t* elow;
    double g;            // gamma / r
    double inv_r;        // 1 / r (G is accumulated already divided by r)
    // adjoint chain
    const void* bb1;     // bbar_{k-1}
    void* bb2;           // in: bbar_{k-2}; out: bbar_k
    double alpha, beta;  // bbar_k = alpha * Ht bbar_{k-1} - beta * bbar_{k-2}
    void* psibar;        // += conj(c_k) bbar_k
    double cc_re, cc_im; // conj(c_k)
    // forward regeneration
    const void* f1;      // b_{k+1}
    void* f0;            // in: b_k; out: b_{k+2} (when regen)
    const void* psi;
    double ck_re, ck_im; // c_k
    int regen;           // produce b_{k+2}
    int pair;            // accumulate the k-th gradient terms (k <= K-1)
    double w;            // w_k
    double* G;           // FP64 per element
    double* dg_slots;    // per-block FP64 accumulators of Re<bbar_k, A b_{k+1}>
};

template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_step(AdjArgs a) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << a.n;
    const C* bb1 = (const C*)a.bb1;
    C* bb2 = (C*)a.bb2;
    const C* f1 = (const C*)a.f1;
    C* f0 = (C*)a.f0;
    const C* psi = (const C*)a.psi;
    C* pb = (C*)a.psibar;
    const double sc = ldexp(1.0, -a.Q);
    double dg = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const double D = __ll2double_rn(energy_fx(a.M, a.tiles, a.elow, (uint64_t)z)) * sc;
        // flip sums of bbar_{k-1} and b_{k+1}
        double sax = 0, say = 0, sbx = 0, sby = 0;
        for (int j = 0; j < a.n; ++j) {
            const int64_t zp = z ^ ((int64_t)1 << j);
            const C u = bb1[zp];
            const C v = f1[zp];
            sax += u.x;
            say += u.y;
            sbx += v.x;
            sby += v.y;
        }
        const C u = bb1[z];
        const C v = f1[z];
        double ox = 0.0, oy = 0.0;
        if (a.beta != 0.0) {  // the first step has no bbar_{k-2}; its slot holds stale data
            const C old = bb2[z];
            ox = old.x;
            oy = old.y;
        }
        // bbar_k
        double nx = a.alpha * (D * u.x + a.g * sax) - a.beta * ox;
        double ny = a.alpha * (D * u.y + a.g * say) - a.beta * oy;
        C nb;
        nb.x = (R)nx;
        nb.y = (R)ny;
        bb2[z] = nb;
        nx = nb.x;
        ny = nb.y;
        // psibar += conj(c_k) bbar_k
        C p = pb[z];
        p.x = (R)(p.x + a.cc_re * nx - a.cc_im * ny);
        p.y = (R)(p.y + a.cc_re * ny + a.cc_im * nx);
        pb[z] = p;
        if (a.pair) {
            // Re(conj(bbar_k) b_{k+1}) and Re(conj(bbar_k) (A b_{k+1}))
            a.G[z] += a.w * a.inv_r * (nx * v.x + ny * v.y);
            dg += a.w * (nx * sbx + ny * sby);
        }
        if (a.regen) {
            const C w0 = f0[z];
            const C ps = psi[z];
            C nf;
            nf.x = (R)(2.0 * (D * v.x + a.g * sbx) - w0.x + a.ck_re * ps.x - a.ck_im * ps.y);
            nf.y = (R)(2.0 * (D * v.y + a.g * sby) - w0.y + a.ck_re * ps.y + a.ck_im * ps.x);
            f0[z] = nf;
        }
    }
    if (a.pair) block_accumulate(dg, a.dg_slots);
}

// k = 0 terms: psibar = conj(c_0) ybar, G += (1/r) Re(conj(ybar) b_1),
// dg += Re(conj(ybar) A b_1).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_init(AdjArgs a) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << a.n;
    const C* yb = (const C*)a.bb1;
    const C* b1 = (const C*)a.f1;
    C* pb = (C*)a.psibar;
    double dg = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        double sbx = 0, sby = 0;
        for (int j = 0; j < a.n; ++j) {
            const C v = b1[z ^ ((int64_t)1 << j)];
            sbx += v.x;
            sby += v.y;
        }
        const C y = yb[z];
        const C v = b1[z];
        C p;
        p.x = (R)(a.cc_re * y.x - a.cc_im * y.y);
        p.y = (R)(a.cc_re * y.y + a.cc_im * y.x);
        pb[z] = p;
        a.G[z] += a.inv_r * ((double)y.x * v.x + (double)y.y * v.y);
        dg += (double)y.x * sbx + (double)y.y * sby;
    }
    block_accumulate(dg, a.dg_slots);
}

// Im <ybar, H y> with H = diag(E) + gamma sum_j X_j, E = c + r D.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_dt(int n, int M, int Q, const int64_t* tiles, const int64_t* elow,
                                                    double c, double r, double gamma, const void* ybar_v,
                                                    const void* y_v, double* slots) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << n;
    const C* yb = (const C*)ybar_v;
    const C* y = (const C*)y_v;
    const double sc = ldexp(1.0, -Q);
    double acc = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const double E = c + r * (__ll2double_rn(energy_fx(M, tiles, elow, (uint64_t)z)) * sc);
        double sx = 0, sy = 0;
        for (int j = 0; j < n; ++j) {
            const C v = y[z ^ ((int64_t)1 << j)];
            sx += v.x;
            sy += v.y;
        }
        const C v = y[z];
        const double hx = E * v.x + gamma * sx, hy = E * v.y + gamma * sy;
        const C u = yb[z];
        acc += (double)u.x * hy - (double)u.y * hx;  // Im(conj(u) * h)
    }
    block_accumulate(acc, slots);
}

// Loss L = <psi|H_P|psi>: grad = 2 E psi; G += |psi|^2 (weight 1); value in slots.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_energy_grad(int n, int M, int Q, const int64_t* tiles,
                                                             const int64_t* elow, double c, double r,
                                                             const void* psi_v, void* grad_v, double* G,
                                                             double* slots) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << n;
    const C* psi = (const C*)psi_v;
    C* gr = (C*)grad_v;
    const double sc = ldexp(1.0, -Q);
    double acc = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const double E = c + r * (__ll2double_rn(energy_fx(M, tiles, elow, (uint64_t)z)) * sc);
        const C v = psi[z];
        const double p2 = (double)v.x * v.x + (double)v.y * v.y;
        C o;
        o.x = (R)(2.0 * E * v.x);
        o.y = (R)(2.0 * E * v.y);
        gr[z] = o;
        G[z] += p2;
        acc += E * p2;
    }
    block_accumulate(acc, slots);
}

// dh_i = sum_z G(z) s_i(z) (blocks 0..n-1), dJ_ij = sum_z G s_i s_j (one block per
// pair i < j); deterministic FP64 sums.
__global__ void __launch_bounds__(kAdjThreads) k_grad_reduce(int n, const double* __restrict__ G, double* out) {
    const int64_t N = (int64_t)1 << n;
    int b = blockIdx.x, i = 0, j = -1;
    if (b < n) {
        i = b;
    } else {
        b -= n;
        for (i = 0; i < n; ++i) {
            const int cnt = n - 1 - i;
            if (b < cnt) {
                j = i + 1 + b;
                break;
            }
            b -= cnt;
        }
    }
    double acc = 0.0;
    for (int64_t z = threadIdx.x; z < N; z += blockDim.x) {
        double v = G[z];
        if ((z >> i) & 1) v = -v;
        if (j >= 0 && ((z >> j) & 1)) v = -v;
        acc += v;
    }
    __shared__ double red[kAdjThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__global__ void k_sum_slots(const double* slots, int nb, double* out) {
    __shared__ double red[256];
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += slots[b];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

unsigned grid_n(int64_t N) {
    int64_t b = (N + kAdjThreads - 1) / kAdjThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kRedBlocks));
}

// Workspace of the adjoint: the forward layout, then 4 state vectors (bbar pair,
// psibar, scratch), G (FP64 per element), anchors, gradient outputs.
struct AdjLayout {
    Layout fwd;
    size_t bb0, bb1, pbar, tmp, G, slots, outs, anchors;
    size_t per_anchor;
    size_t total_fixed;
};

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

AdjLayout adj_layout(int n, int prec) {
    AdjLayout A;
    A.fwd = make_layout(n, prec);
    const size_t vb = ((size_t)1 << n) * A.fwd.cbytes;
    size_t off = a256(A.fwd.total);
    A.bb0 = off;
    off = a256(off + vb);
    A.bb1 = off;
    off = a256(off + vb);
    A.pbar = off;
    off = a256(off + vb);
    A.tmp = off;
    off = a256(off + vb);
    A.G = off;
    off = a256(off + ((size_t)1 << n) * sizeof(double));
    A.slots = off;
    off = a256(off + 4 * (size_t)kRedBlocks * sizeof(double));
    A.outs = off;
    off = a256(off + ((size_t)n * n + n + 8) * sizeof(double));
    A.anchors = off;
    A.per_anchor = 2 * a256(vb);
    A.total_fixed = off;
    return A;
}

template <typename R>
cudaError_t launch_adj_step(const AdjArgs& a, cudaStream_t s) {
    note_launch(kKindReduce);
    k_adj_step<R><<<grid_n((int64_t)1 << a.n), kAdjThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" size_t cheb_adjoint_workspace_bytes(int n, cheb_precision_t precision, int anchors) {
    if (n < 1 || n > kMaxQubits || anchors < 1) return 0;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return 0;
    AdjLayout A = adj_layout(n, precision);
    return A.total_fixed + (size_t)anchors * A.per_anchor;
}

// Gradient of a loss on the output of a schedule (S = 1: a single exp(-itH) psi).
extern "C" cheb_status_t cheb_anneal_adjoint(int n, const double* h, const double* J, int S, const double* gamma_s,
                                             const double* t_s, const void* boundaries, const void* psi_T,
                                             void* grad, cheb_precision_t precision, double tol,
                                             cheb_method_t method, double* grad_gamma, double* grad_t,
                                             double* grad_h, double* grad_J, void* workspace, size_t ws_bytes,
                                             void* stream) {
    if (n < 1 || n > kMaxQubits || S < 1 || !h || !J || !gamma_s || !t_s || !boundaries || !psi_T || !grad)
        return CHEB_ERR_INVALID_ARG;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(h, n) || !finite_all(J, (size_t)n * n) || !finite_all(gamma_s, S) || !finite_all(t_s, S))
        return CHEB_ERR_INVALID_ARG;
    if (!(tol > 0) || !std::isfinite(tol)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF) return CHEB_ERR_INVALID_ARG;
    if (((uintptr_t)boundaries | (uintptr_t)psi_T | (uintptr_t)grad) & 15) return CHEB_ERR_INVALID_ARG;
    AdjLayout A = adj_layout(n, precision);
    if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < A.total_fixed + A.per_anchor) return CHEB_ERR_WORKSPACE;
    const int max_anchors = (int)std::min<size_t>((ws_bytes - A.total_fixed) / A.per_anchor, 1 << 20);
    unsigned char* ws = (unsigned char*)workspace;
    cudaStream_t s0 = (cudaStream_t)stream;
    Ctx C{n, precision, A.fwd, ws, s0};
    const int64_t N = (int64_t)1 << n;
    const size_t vb = (size_t)N * A.fwd.cbytes;
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
    CUDA_TRY(cudaMemsetAsync(ws + A.G, 0, (size_t)N * sizeof(double), s0));
    double emin = 0, emax = 0;
    cheb_status_t st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    const double c = 0.5 * (emax + emin);
    const double tol_s = tol / S;
    double* slots = (double*)(ws + A.slots);
    double* outs = (double*)(ws + A.outs);
    unsigned char* B0 = ws + A.fwd.b0;
    unsigned char* B1 = ws + A.fwd.b1;
    unsigned char* BB[2] = {ws + A.bb0, ws + A.bb1};
    unsigned char* pbar = ws + A.pbar;
    std::vector<double> gg(S), gt(S);
    const int Mt = A.fwd.M;
    for (int s = S - 1; s >= 0; --s) {
        double r = 0.5 * (emax - emin) + std::fabs(gamma_s[s]) * n;
        if (!(r > 0)) r = 1.0;
        const double g = gamma_s[s] / r;
        FixedOp F = make_fixed(n, h, J, c, r, precision == CHEB_FP32 ? kMaxQF32 : 62);
        if (F.Q < 24) return CHEB_ERR_UNSUPPORTED;
        st = upload_tables(C, F);
        if (st != CHEB_OK) return st;
        std::vector<std::complex<double>> coef;
        int K = -1, slices = 1;
        double err = 0.0;
        st = slice_coefficients(t_s[s], c, r, tol_s, method, 0, coef, &K, &slices, &err);
        if (st != CHEB_OK) return st;
        if (slices != 1) return CHEB_ERR_UNSUPPORTED;
        const void* psi_s = (const unsigned char*)boundaries + (size_t)s * vb;
        const void* y_s = (s == S - 1) ? psi_T : (const unsigned char*)boundaries + (size_t)(s + 1) * vb;
        // dt_s = Im <ybar, H_s y_s>
        {
            CUDA_TRY(cudaMemsetAsync(slots, 0, kRedBlocks * sizeof(double), s0));
            const unsigned gb = grid_n(N);
            note_launch(kKindReduce);
            if (precision == CHEB_FP32)
                k_dt<float><<<gb, kAdjThreads, 0, s0>>>(n, Mt, F.Q, C.tiles(), C.elow(), c, r, gamma_s[s], grad, y_s, slots);
            else
                k_dt<double><<<gb, kAdjThreads, 0, s0>>>(n, Mt, F.Q, C.tiles(), C.elow(), c, r, gamma_s[s], grad, y_s, slots);
            k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, outs + 0);
            CUDA_TRY(cudaMemcpyAsync(&gt[s], outs + 0, sizeof(double), cudaMemcpyDeviceToHost, s0));
        }
        if (K == 0) {
            // y = c_0 psi: psibar = conj(c_0) ybar, no operator dependence
            launch_scale(precision, N, grad, grad, coef[0].real(), -coef[0].imag(), s0);
            gg[s] = 0.0;
            continue;
        }
        // forward recomputation from psi_s down to (b_1, b_2), saving anchor pairs
        const int C_gap = std::max(1, (K - 1 + max_anchors - 1) / max_anchors);
        std::vector<int> anchor_k;  // anchors store (b_k, b_{k+1}) for k = 1 + m*C_gap < K
        for (int k = 1; k < K; k += C_gap) anchor_k.push_back(k);
        if ((int)anchor_k.size() > max_anchors) return CHEB_ERR_WORKSPACE;
        unsigned char* Bv[2] = {B0, B1};
        launch_scale(precision, N, psi_s, Bv[1], coef[K].real(), coef[K].imag(), s0);  // b_K
        int cur = 1;
        FusedPlan plan;
        const bool fused = fused_supported(n, precision) && n > (precision == CHEB_FP32 ? kSmallMaxF32 : kSmallMaxF64);
        if (fused) plan = fused_plan(n, precision);
        for (int k = K - 1; k >= 1; --k) {
            StepArgs a;
            a.n = n;
            a.M = Mt;
            a.Q = F.Q;
            a.tiles = C.tiles();
            a.elow = C.elow();
            a.jq = (const int64_t*)(ws + A.fwd.jq);
            a.b1 = Bv[cur];
            a.b2 = Bv[cur ^ 1];
            a.psi = psi_s;
            a.out = Bv[cur ^ 1];
            a.ck_re = coef[k].real();
            a.ck_im = coef[k].imag();
            a.scale = 2.0;
            a.sgn = (k == K - 1) ? 0.0 : -1.0;
            a.g = g;
            if (fused) {
                if (launch_step_fused(plan, a, nullptr, C.flags(), s0) != cudaSuccess) return CHEB_ERR_CUDA;
            } else {
                launch_step_plain(precision, a, s0);
            }
            cur ^= 1;  // Bv[cur] = b_k, Bv[cur ^ 1] = b_{k+1}
            for (size_t m = 0; m < anchor_k.size(); ++m)
                if (anchor_k[m] == k) {
                    unsigned char* dst = ws + A.anchors + m * A.per_anchor;
                    CUDA_TRY(cudaMemcpyAsync(dst, Bv[cur], vb, cudaMemcpyDeviceToDevice, s0));
                    if (k + 1 < K)
                        CUDA_TRY(cudaMemcpyAsync(dst + A.per_anchor / 2, Bv[cur ^ 1], vb, cudaMemcpyDeviceToDevice, s0));
                    else
                        launch_scale(precision, N, psi_s, dst + A.per_anchor / 2, coef[K].real(), coef[K].imag(), s0);
                }
        }
        // now Bv[cur] = b_1 and Bv[cur ^ 1] = b_2 (or b_K = b_1 and b_2 = 0 when K == 1)
        unsigned char* f_k = Bv[cur];       // b_k   (k = 1)
        unsigned char* f_k1 = Bv[cur ^ 1];  // b_{k+1}
        if (K == 1) CUDA_TRY(cudaMemsetAsync(f_k1, 0, vb, s0));
        // k = 0 terms
        CUDA_TRY(cudaMemsetAsync(slots, 0, kRedBlocks * sizeof(double), s0));
        AdjArgs x{};
        x.n = n;
        x.M = Mt;
        x.Q = F.Q;
        x.tiles = C.tiles();
        x.elow = C.elow();
        x.g = g;
        x.inv_r = 1.0 / r;
        x.G = (double*)(ws + A.G);
        x.dg_slots = slots;
        x.psi = psi_s;
        x.psibar = pbar;
        {
            AdjArgs y0 = x;
            y0.bb1 = grad;
            y0.f1 = f_k;
            y0.cc_re = coef[0].real();
            y0.cc_im = -coef[0].imag();
            note_launch(kKindReduce);
            if (precision == CHEB_FP32)
                k_adj_init<float><<<grid_n(N), kAdjThreads, 0, s0>>>(y0);
            else
                k_adj_init<double><<<grid_n(N), kAdjThreads, 0, s0>>>(y0);
        }
        // bbar_{-1} is unused (beta = 0 at k = 1): BB[1] receives bbar_1
        const void* bbm1 = grad;                 // bbar_{k-1}
        unsigned char* bbm2 = BB[1];             // bbar_{k-2} slot, overwritten by bbar_k
        unsigned char* spare = BB[0];
        for (int k = 1; k <= K; ++k) {
            // reset the regenerated pair at anchors
            for (size_t m = 0; m < anchor_k.size(); ++m)
                if (anchor_k[m] == k && k > 1) {
                    const unsigned char* src = ws + A.anchors + m * A.per_anchor;
                    CUDA_TRY(cudaMemcpyAsync(f_k, src, vb, cudaMemcpyDeviceToDevice, s0));
                    CUDA_TRY(cudaMemcpyAsync(f_k1, src + A.per_anchor / 2, vb, cudaMemcpyDeviceToDevice, s0));
                }
            AdjArgs y = x;
            y.bb1 = bbm1;
            y.bb2 = bbm2;
            y.alpha = (k == 1) ? 1.0 : 2.0;
            y.beta = (k == 1) ? 0.0 : 1.0;
            y.cc_re = coef[k].real();
            y.cc_im = -coef[k].imag();
            y.f1 = f_k1;
            y.f0 = f_k;
            y.ck_re = coef[k].real();
            y.ck_im = coef[k].imag();
            y.pair = (k <= K - 1) ? 1 : 0;
            y.regen = (k + 2 <= K) ? 1 : 0;
            y.w = 2.0;
            cudaError_t e = precision == CHEB_FP32 ? launch_adj_step<float>(y, s0) : launch_adj_step<double>(y, s0);
            if (e != cudaSuccess) return CHEB_ERR_CUDA;
            // rotate: bbar_k now in bbm2; next step reads it as bbar_{k-1}
            const void* new_b1 = bbm2;
            unsigned char* new_b2 = (k == 1) ? spare : (unsigned char*)bbm1;  // bbar_{k-1} becomes bbar_{k-2}
            if (k == 1) {
                // bbar_0 = ybar lives in the caller's buffer; copy it into the spare slot
                CUDA_TRY(cudaMemcpyAsync(spare, grad, vb, cudaMemcpyDeviceToDevice, s0));
            }
            bbm1 = new_b1;
            bbm2 = new_b2;
            // forward pair advances: (b_{k+1}, b_{k+2}) now in (f_k1, f_k)
            std::swap(f_k, f_k1);
        }
        k_sum_slots<<<1, 256, 0, s0>>>(slots, grid_n(N), outs + 1);
        double dgv = 0.0;
        CUDA_TRY(cudaMemcpyAsync(&dgv, outs + 1, sizeof(double), cudaMemcpyDeviceToHost, s0));
        // psibar becomes ybar of the previous segment
        CUDA_TRY(cudaMemcpyAsync(grad, pbar, vb, cudaMemcpyDeviceToDevice, s0));
        CUDA_TRY(cudaStreamSynchronize(s0));
        gg[s] = dgv / r;
    }
    // dh, dJ from G (already divided by r per segment)
    const int nblk = n + n * (n - 1) / 2;
    note_launch(kKindReduce);
    k_grad_reduce<<<nblk, kAdjThreads, 0, s0>>>(n, (const double*)(ws + A.G), outs);
    std::vector<double> red(nblk);
    CUDA_TRY(cudaMemcpyAsync(red.data(), outs, nblk * sizeof(double), cudaMemcpyDeviceToHost, s0));
    st = read_flags(C);
    if (st != CHEB_OK) return st;
    if (grad_gamma)
        for (int s = 0; s < S; ++s) grad_gamma[s] = gg[s];
    if (grad_t)
        for (int s = 0; s < S; ++s) grad_t[s] = gt[s];
    if (grad_h)
        for (int i = 0; i < n; ++i) grad_h[i] = red[i];
    if (grad_J) {
        for (size_t q = 0; q < (size_t)n * n; ++q) grad_J[q] = 0.0;
        int b = n;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) grad_J[(size_t)i * n + j] = red[b++];
    }
    return CHEB_OK;
}

// Loss L = <psi|H_P|psi>: value, dL/dpsi (torch convention: 2 H_P psi), dL/dh, dL/dJ.
extern "C" cheb_status_t cheb_energy_grad(int n, const double* h, const double* J, const void* psi, void* grad_psi,
                                          cheb_precision_t precision, double* energy, double* grad_h,
                                          double* grad_J, void* workspace, size_t ws_bytes, void* stream) {
    cheb_status_t st = check_common(n, h, J, precision, workspace, ws_bytes);
    if (st != CHEB_OK) return st;
    if (!psi || !grad_psi || (((uintptr_t)psi | (uintptr_t)grad_psi) & 15)) return CHEB_ERR_INVALID_ARG;
    AdjLayout A = adj_layout(n, precision);
    if (ws_bytes < A.total_fixed) return CHEB_ERR_WORKSPACE;
    unsigned char* ws = (unsigned char*)workspace;
    cudaStream_t s0 = (cudaStream_t)stream;
    Ctx C{n, precision, A.fwd, ws, s0};
    const int64_t N = (int64_t)1 << n;
    FixedOp F = make_fixed(n, h, J, 0.0, 1.0);
    st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    double* G = (double*)(ws + A.G);
    double* slots = (double*)(ws + A.slots);
    double* outs = (double*)(ws + A.outs);
    CUDA_TRY(cudaMemsetAsync(G, 0, (size_t)N * sizeof(double), s0));
    CUDA_TRY(cudaMemsetAsync(slots, 0, kRedBlocks * sizeof(double), s0));
    const unsigned gb = grid_n(N);
    note_launch(kKindReduce);
    if (precision == CHEB_FP32)
        k_energy_grad<float><<<gb, kAdjThreads, 0, s0>>>(n, A.fwd.M, F.Q, C.tiles(), C.elow(), 0.0, 1.0, psi, grad_psi, G, slots);
    else
        k_energy_grad<double><<<gb, kAdjThreads, 0, s0>>>(n, A.fwd.M, F.Q, C.tiles(), C.elow(), 0.0, 1.0, psi, grad_psi, G, slots);
    k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, outs + n * n + n);
    const int nblk = n + n * (n - 1) / 2;
    k_grad_reduce<<<nblk, kAdjThreads, 0, s0>>>(n, G, outs);
    std::vector<double> red(nblk + 1);
    CUDA_TRY(cudaMemcpyAsync(red.data(), outs, nblk * sizeof(double), cudaMemcpyDeviceToHost, s0));
    CUDA_TRY(cudaMemcpyAsync(&red[nblk], outs + n * n + n, sizeof(double), cudaMemcpyDeviceToHost, s0));
    CUDA_TRY(cudaStreamSynchronize(s0));
    CUDA_TRY(cudaGetLastError());
    if (energy) *energy = red[nblk];
    if (grad_h)
        for (int i = 0; i < n; ++i) grad_h[i] = red[i];
    if (grad_J) {
        for (size_t q = 0; q < (size_t)n * n; ++q) grad_J[q] = 0.0;
        int b = n;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) grad_J[(size_t)i * n + j] = red[b++];
    }
    return CHEB_OK;
}
