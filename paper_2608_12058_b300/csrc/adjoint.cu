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
//   dL/dgamma = (1/r) Re sum_k w_k <bbar_k, (sum_j X_j) b_{k+1}>
//             = (1/gamma) Re sum_k w_k <bbar_k, (Ht - D) b_{k+1}>,
//   dL/dh_i   = (1/r) sum_z G(z) s_i(z),  dL/dJ_ij = (1/r) sum_z G(z) s_i(z) s_j(z),
//   dL/dt     = Im <ybar, H y>            (from dy/dt = -i H y).
// Ht b_{k+1} needs no matvec: the recurrence itself gives
//   Ht b_{k+1} = (b_{k+2} + b_k - c_k psi)/2 (k >= 1),  Ht b_1 = y + b_2 - c_0 psi.
// The b_k are needed in increasing k while the forward produces them decreasing;
// they are regenerated upward, b_{k+2} = 2 Ht b_{k+1} - b_k + c_k psi, from (b_1, b_2),
// and reset every C steps from anchor pairs saved by a forward recomputation. Both
// recurrences run on the same step kernels as the forward pass.
//
// Round-off gauge: <bbar_s, y_s> = <ybar_T, y_T> holds exactly for every segment s
// (it is <P^H a, b> = <a, P b>). In FP32 the adjoint chain and the stored forward
// states drift in relative phase; that drift is measured from the invariant and
// removed by rotating ybar at the start of each segment (and the returned psibar).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>
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

// Block-level FP64 sum of v, added into slot[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_accumulate(double v, double* slot) {
    __shared__ double red[kAdjThreads];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) slot[blockIdx.x] += red[0];
    __syncthreads();
}

// Elementwise work of up to kAccBatch consecutive adjoint steps k = k0 .. k0+m-1
// (every constant that would scale all elements alike - the gauge phase, 1/r - is
// applied in FP64 per segment):
//   psibar (+)= conj(c_k) bbar_k                      (mode 1 add, 2 set)
//   Gs     += w_k Re(conj(bbar_k) b_{k+1})            (pair: w_k != 0, i.e. k < K)
//   hsum   += Re(conj(bbar_k) x_k),  x_k = b_k + b_{k+2} - c_k psi - w_k D b_{k+1}
// with b_0 := y (the segment's output) and b_{K+1} := 0. Since
// Ht b_{k+1} = hs (b_k + b_{k+2} - c_k psi) with w_k hs = 1 (hs = 1/2, and 1 at
// k = 0), x_k = w_k (Ht - D) b_{k+1} = w_k g sum_j X_j b_{k+1}: the cancellation
// between Ht and D happens per element, where its rounding is of the size of the
// rounding of b_{k+2} itself, and the sums over z have none. c_k is used as the step
// kernels hold it. Batching reads each b_j, psi, psibar and Gs once per batch.
constexpr int kAccBatch = 4;
struct AccArgs {
    int n, m, mode, M, Q;
    const int64_t* tiles;
    const int64_t* elow;
    const void* bbar[kAccBatch];    // bbar_{k0+i}
    const void* fb[kAccBatch + 2];  // b_{k0+j}; nullptr = the zero vector
    const void* psi;
    void* psibar;
    void* Gs;
    double* slots;
    double cc_re[kAccBatch], cc_im[kAccBatch];  // conj(c_{k0+i})
    double w[kAccBatch];                         // w_k, 0 when k = K (no pair)
};

// One block per tile of 2^M amplitudes (z = T 2^M + x): the tile's energy partial
// sums over the low 5 and the next 6 bits of x go to shared memory once, so that
// e(z) = A(T) + Wlo[x & 31] + Whi[x >> 5] + elow(x) costs three adds.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_adj_acc(AccArgs a) {
    using C = typename Cx<R>::T;
    __shared__ int64_t Wlo[32], Whi[64];
    const int M = a.M;
    const int64_t tsize = (int64_t)1 << M;
    const int64_t ntiles = (int64_t)1 << (a.n - M);
    const C* psi = (const C*)a.psi;
    C* pb = (C*)a.psibar;
    R* Gs = (R*)a.Gs;
    bool any_pair = false;
#pragma unroll
    for (int i = 0; i < kAccBatch; ++i) any_pair |= (i < a.m) && a.w[i] != 0.0;
    // D = e 2^-Q from the fixed-point energy e (from its two 32-bit halves)
    const R s_hi = (R)ldexp(1.0, 32 - a.Q), s_lo = (R)ldexp(1.0, -a.Q);
    const int t = threadIdx.x;
    R hsum = 0;  // a few elements per thread: no cancellation in these sums
    for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
        const int64_t* row = a.tiles + T * (M + 1);
        if (any_pair) {
            __syncthreads();  // the previous tile's tables are no longer read
            if (t < 96) {
                const int lo = t < 32 ? 0 : 5, hi = t < 32 ? 5 : 11;
                const int x = t < 32 ? t : (t - 32) << 5;
                int64_t v = 0;
                for (int i = lo; i < hi && i < M; ++i) v += sgn_sel((x >> i) & 1, __ldg(row + i));
                if (t < 32) Wlo[t] = v;
                else Whi[t - 32] = v;
            }
            __syncthreads();
        }
        const int64_t Abase = any_pair ? __ldg(row + M) : 0;
        for (int64_t x = t; x < tsize; x += blockDim.x) {
            const int64_t z = T * tsize + x;
            C f[kAccBatch + 2];
#pragma unroll
            for (int j = 0; j < kAccBatch + 2; ++j) {
                if (j < a.m + 2 && a.fb[j]) {
                    f[j] = ((const C*)a.fb[j])[z];
                } else {
                    f[j].x = 0;
                    f[j].y = 0;
                }
            }
            C p;
            if (a.mode == 1) {
                p = pb[z];
            } else {
                p.x = 0;
                p.y = 0;
            }
            const C ps = psi[z];
            R D = 0;
            if (any_pair) {
                const int64_t e = Abase + Wlo[x & 31] + Whi[(x >> 5) & 63] + __ldg(a.elow + x);
                D = (R)(int)(e >> 32) * s_hi + (R)(uint32_t)(e & 0xffffffffll) * s_lo;
            }
            R g = 0, hs = 0;
#pragma unroll
            for (int i = 0; i < kAccBatch; ++i) {
                if (i >= a.m) break;
                const C u = ((const C*)a.bbar[i])[z];
                const R cr = (R)a.cc_re[i], ci = (R)a.cc_im[i];
                p.x += cr * u.x - ci * u.y;
                p.y += cr * u.y + ci * u.x;
                if (a.w[i] != 0.0) {
                    const R w = (R)a.w[i];
                    const C v = f[i + 1];
                    g += w * (u.x * v.x + u.y * v.y);
                    // c_k = conj(cc): c_k psi = (cr x + ci y, cr y - ci x)
                    const R wD = w * D;
                    const R xr = (f[i].x + f[i + 2].x) - (cr * ps.x + ci * ps.y) - wD * v.x;
                    const R xi = (f[i].y + f[i + 2].y) - (cr * ps.y - ci * ps.x) - wD * v.y;
                    hs += u.x * xr + u.y * xi;
                }
            }
            pb[z] = p;
            if (any_pair) {
                Gs[z] += g;
                hsum += hs;
            }
        }
    }
    if (any_pair) block_accumulate((double)hsum, a.slots);
}

// FP32 variant of k_adj_acc: each thread takes two neighbouring amplitudes per
// iteration (16-byte loads), which doubles the bytes in flight per load and halves
// the load instructions; the arithmetic is the same.
__global__ void __launch_bounds__(kAdjThreads) k_adj_acc_f32x2(AccArgs a) {
    __shared__ int64_t Wlo[32], Whi[64];
    const int M = a.M;
    const int64_t tsize = (int64_t)1 << M;
    const int64_t ntiles = (int64_t)1 << (a.n - M);
    const float4* psi = (const float4*)a.psi;
    float4* pb = (float4*)a.psibar;
    float2* Gs = (float2*)a.Gs;
    bool any_pair = false;
#pragma unroll
    for (int i = 0; i < kAccBatch; ++i) any_pair |= (i < a.m) && a.w[i] != 0.0;
    const float s_hi = (float)ldexp(1.0, 32 - a.Q), s_lo = (float)ldexp(1.0, -a.Q);
    const int t = threadIdx.x;
    float hsum = 0.f;
    for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
        const int64_t* row = a.tiles + T * (M + 1);
        if (any_pair) {
            __syncthreads();
            if (t < 96) {
                const int lo = t < 32 ? 0 : 5, hi = t < 32 ? 5 : 11;
                const int x = t < 32 ? t : (t - 32) << 5;
                int64_t v = 0;
                for (int i = lo; i < hi && i < M; ++i) v += sgn_sel((x >> i) & 1, __ldg(row + i));
                if (t < 32) Wlo[t] = v;
                else Whi[t - 32] = v;
            }
            __syncthreads();
        }
        const int64_t Abase = any_pair ? __ldg(row + M) : 0;
        for (int64_t x = 2 * t; x < tsize; x += 2 * blockDim.x) {
            const int64_t z2 = (T * tsize + x) >> 1;  // float4 index of amplitudes z, z + 1
            float4 f[kAccBatch + 2];
#pragma unroll
            for (int j = 0; j < kAccBatch + 2; ++j)
                f[j] = (j < a.m + 2 && a.fb[j]) ? ((const float4*)a.fb[j])[z2] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 u[kAccBatch];
#pragma unroll
            for (int i = 0; i < kAccBatch; ++i)
                u[i] = (i < a.m) ? ((const float4*)a.bbar[i])[z2] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 p = a.mode == 1 ? pb[z2] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 ps = psi[z2];
            float2 gz = any_pair ? Gs[z2] : make_float2(0.f, 0.f);
            float D0 = 0.f, D1 = 0.f;
            if (any_pair) {
                const int64_t e0 = Abase + Wlo[x & 31] + Whi[(x >> 5) & 63] + __ldg(a.elow + x);
                const int64_t e1 = Abase + Wlo[(x + 1) & 31] + Whi[((x + 1) >> 5) & 63] + __ldg(a.elow + x + 1);
                D0 = (float)(int)(e0 >> 32) * s_hi + (float)(uint32_t)(e0 & 0xffffffffll) * s_lo;
                D1 = (float)(int)(e1 >> 32) * s_hi + (float)(uint32_t)(e1 & 0xffffffffll) * s_lo;
            }
#pragma unroll
            for (int i = 0; i < kAccBatch; ++i) {
                if (i >= a.m) break;
                const float cr = (float)a.cc_re[i], ci = (float)a.cc_im[i];
                const float4 uu = u[i];
                p.x += cr * uu.x - ci * uu.y;
                p.y += cr * uu.y + ci * uu.x;
                p.z += cr * uu.z - ci * uu.w;
                p.w += cr * uu.w + ci * uu.z;
                if (a.w[i] != 0.0) {
                    const float w = (float)a.w[i];
                    const float4 v = f[i + 1], f0 = f[i], f2 = f[i + 2];
                    gz.x += w * (uu.x * v.x + uu.y * v.y);
                    gz.y += w * (uu.z * v.z + uu.w * v.w);
                    // c_k = conj(cc): c_k psi = (cr x + ci y, cr y - ci x)
                    const float wD0 = w * D0, wD1 = w * D1;
                    const float xr0 = (f0.x + f2.x) - (cr * ps.x + ci * ps.y) - wD0 * v.x;
                    const float xi0 = (f0.y + f2.y) - (cr * ps.y - ci * ps.x) - wD0 * v.y;
                    const float xr1 = (f0.z + f2.z) - (cr * ps.z + ci * ps.w) - wD1 * v.z;
                    const float xi1 = (f0.w + f2.w) - (cr * ps.w - ci * ps.z) - wD1 * v.w;
                    hsum += (uu.x * xr0 + uu.y * xi0) + (uu.z * xr1 + uu.w * xi1);
                }
            }
            pb[z2] = p;
            if (any_pair) Gs[z2] = gz;
        }
    }
    if (any_pair) block_accumulate((double)hsum, a.slots);
}

unsigned grid_tiles(int n, int M) {
    const int64_t nt = (int64_t)1 << (n - M);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(nt, kRedBlocks));
}

// End of a segment: G(z) += fac Gs(z) (FP64; fac = b_s / r_s) and, when the unscaled
// energy tables are given, slots += sum_z Gs(z) E(z) (for dL/db_s of general segments).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_fold(int n, const R* __restrict__ Gs, double fac, double* G,
                                                      int M, int Q0, const int64_t* tiles0, const int64_t* elow0,
                                                      double* slots) {
    const int64_t N = (int64_t)1 << n;
    const double sc = ldexp(1.0, -Q0);
    double acc = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const double g = (double)Gs[z];
        G[z] += g * fac;
        if (tiles0) acc += g * (__ll2double_rn(energy_fx(M, tiles0, elow0, (uint64_t)z)) * sc);
    }
    if (tiles0) block_accumulate(acc, slots);
}

// Fallback for gamma = 0, where (Ht - D)/gamma is not available: the flip sums of
// b_{k+1} are formed explicitly; slots += w Re(conj(bbar_k) sum_j X_j b_{k+1}).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_dg_flip(int n, const void* bbar_v, const void* f1_v, double w,
                                                        double* slots) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << n;
    const C* bb = (const C*)bbar_v;
    const C* f1 = (const C*)f1_v;
    double dg = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        double sx = 0, sy = 0;
        for (int j = 0; j < n; ++j) {
            const C v = f1[z ^ ((int64_t)1 << j)];
            sx += v.x;
            sy += v.y;
        }
        const C u = bb[z];
        dg += w * ((double)u.x * sx + (double)u.y * sy);
    }
    block_accumulate(dg, slots);
}

// <ybar, H y> and <ybar, y> (complex), H = diag(E) + gamma sum_j X_j, E = c + r D:
// slots[0..3] x kRedBlocks = Re, Im of each. One block per tile of 2^M amplitudes:
// the tile of y is staged in shared memory for the flip partners of the low M bits
// (the others are read from global memory), E comes from the tile's shared energy
// partial sums, the flip sums are formed in the vector precision and the products
// and sums in FP64.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_dt(int n, int M, int Q, const int64_t* tiles, const int64_t* elow,
                                                    double c, double r, double gamma, const void* ybar_v,
                                                    const void* y_v, double* slots) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char dt_smem[];
    C* ty = (C*)dt_smem;  // 2^M
    __shared__ int64_t Wlo[32], Whi[64];
    const int64_t tsize = (int64_t)1 << M;
    const int64_t ntiles = (int64_t)1 << (n - M);
    const C* yb = (const C*)ybar_v;
    const C* y = (const C*)y_v;
    const double sc = ldexp(1.0, -Q);
    const int t = threadIdx.x;
    double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
    for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
        const int64_t* row = tiles + T * (M + 1);
        __syncthreads();
        if (t < 96) {
            const int lo = t < 32 ? 0 : 5, hi = t < 32 ? 5 : 11;
            const int x = t < 32 ? t : (t - 32) << 5;
            int64_t v = 0;
            for (int i = lo; i < hi && i < M; ++i) v += sgn_sel((x >> i) & 1, __ldg(row + i));
            if (t < 32) Wlo[t] = v;
            else Whi[t - 32] = v;
        }
        for (int64_t x = t; x < tsize; x += blockDim.x) ty[x] = y[T * tsize + x];
        __syncthreads();
        const int64_t A = __ldg(row + M);
        for (int64_t x = t; x < tsize; x += blockDim.x) {
            const int64_t z = T * tsize + x;
            const int64_t e = A + Wlo[x & 31] + Whi[(x >> 5) & 63] + __ldg(elow + x);
            const double E = c + r * (__ll2double_rn(e) * sc);
            R sx = 0, sy = 0;
            for (int j = 0; j < M; ++j) {
                const C v = ty[x ^ ((int64_t)1 << j)];
                sx += v.x;
                sy += v.y;
            }
            for (int j = M; j < n; ++j) {
                const C v = y[z ^ ((int64_t)1 << j)];
                sx += v.x;
                sy += v.y;
            }
            const C v = ty[x];
            const double hx = E * v.x + gamma * (double)sx, hy = E * v.y + gamma * (double)sy;
            const C u = yb[z];
            ar += (double)u.x * hx + (double)u.y * hy;
            ai += (double)u.x * hy - (double)u.y * hx;
            br += (double)u.x * v.x + (double)u.y * v.y;
            bi += (double)u.x * v.y - (double)u.y * v.x;
        }
    }
    block_accumulate(ar, slots);
    block_accumulate(ai, slots + kRedBlocks);
    block_accumulate(br, slots + 2 * kRedBlocks);
    block_accumulate(bi, slots + 3 * kRedBlocks);
}

// <a, b> (complex) into slots[0..1] x kRedBlocks.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_dot(int n, const void* a_v, const void* b_v, double* slots) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << n;
    const C* a = (const C*)a_v;
    const C* b = (const C*)b_v;
    double re = 0.0, im = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const C u = a[z], v = b[z];
        re += (double)u.x * v.x + (double)u.y * v.y;
        im += (double)u.x * v.y - (double)u.y * v.x;
    }
    block_accumulate(re, slots);
    block_accumulate(im, slots + kRedBlocks);
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

// dh_i = sum_z G(z) s_i(z), dJ_ij = sum_z G(z) s_i(z) s_j(z) (i < j), written as
// out[i] and out[n + pair(i, j)] (pairs in row order). One pass over G: with
// z = T 2^M + x, each tile's Walsh coefficients W_T[w] = sum_x G(T, x) prod_{i in w} s_i(x)
// come from a fast Walsh-Hadamard transform of the tile in shared memory, and
//   sum_z G s_i      = sum_T W_T[1<<i]            (i < M),   sum_T W_T[0] s_i(T)        (i >= M)
//   sum_z G s_i s_j  = sum_T W_T[(1<<i)|(1<<j)]   (i,j < M), sum_T W_T[1<<i] s_j(T)     (i < M <= j),
//                      sum_T W_T[0] s_i(T) s_j(T) (M <= i, j),
// with s_i(T) the spin of bit i - M of T. Per-block partial sums, then a fixed-order
// sum over blocks (deterministic).
constexpr int kMaxMoments = kMaxQubits + kMaxQubits * (kMaxQubits - 1) / 2;
constexpr int kMomentsPerThread = (kMaxMoments + kAdjThreads - 1) / kAdjThreads;

__device__ __forceinline__ void moment_pair(int n, int o, int& i, int& j) {
    if (o < n) {
        i = o;
        j = -1;
        return;
    }
    o -= n;
    for (i = 0; i < n; ++i) {
        const int cnt = n - 1 - i;
        if (o < cnt) {
            j = i + 1 + o;
            return;
        }
        o -= cnt;
    }
}

__global__ void __launch_bounds__(kAdjThreads) k_moments(int n, int M, const double* __restrict__ G, double* partial) {
    extern __shared__ double W[];  // 2^M
    const int nout = n + n * (n - 1) / 2;
    const int64_t tsize = (int64_t)1 << M;
    const int64_t ntiles = (int64_t)1 << (n - M);
    double acc[kMomentsPerThread];
    int oi[kMomentsPerThread], oj[kMomentsPerThread];
    for (int q = 0; q < kMomentsPerThread; ++q) {
        acc[q] = 0.0;
        const int o = threadIdx.x + q * kAdjThreads;
        oi[q] = -1;
        oj[q] = -1;
        if (o < nout) moment_pair(n, o, oi[q], oj[q]);
    }
    for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
        __syncthreads();  // the previous tile's coefficients are no longer read
        for (int64_t x = threadIdx.x; x < tsize; x += blockDim.x) W[x] = G[T * tsize + x];
        __syncthreads();
        for (int b = 0; b < M; ++b) {
            for (int64_t pr = threadIdx.x; pr < tsize / 2; pr += blockDim.x) {
                const int64_t lo = ((pr >> b) << (b + 1)) | (pr & ((1 << b) - 1));
                const int64_t hi = lo | (1 << b);
                const double u = W[lo], v = W[hi];
                W[lo] = u + v;
                W[hi] = u - v;
            }
            __syncthreads();
        }
        for (int q = 0; q < kMomentsPerThread; ++q) {
            const int i = oi[q], j = oj[q];
            if (i < 0) continue;
            auto spin = [&](int k) { return ((T >> (k - M)) & 1) ? -1.0 : 1.0; };
            double v;
            if (j < 0) {
                v = i < M ? W[1 << i] : W[0] * spin(i);
            } else if (j < M) {
                v = W[(1 << i) | (1 << j)];
            } else if (i < M) {
                v = W[1 << i] * spin(j);
            } else {
                v = W[0] * spin(i) * spin(j);
            }
            acc[q] += v;
        }
    }
    for (int q = 0; q < kMomentsPerThread; ++q) {
        const int o = threadIdx.x + q * kAdjThreads;
        if (o < nout) partial[(size_t)blockIdx.x * nout + o] = acc[q];
    }
}

__global__ void k_moments_final(int nb, int nout, const double* __restrict__ partial, double* out) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += partial[(size_t)b * nout + o];
        out[o] = a;
    }
}

// Launch both stages on the stream; out receives n + n(n-1)/2 doubles.
cudaError_t launch_moments(int n, const double* G, double* partial, double* out, cudaStream_t s) {
    const int M = n < kTileBits ? n : kTileBits;
    const int nout = n + n * (n - 1) / 2;
    const int64_t ntiles = (int64_t)1 << (n - M);
    const unsigned nb = (unsigned)std::min<int64_t>(ntiles, kRedBlocks);
    note_launch(kKindReduce);
    k_moments<<<nb, kAdjThreads, ((size_t)1 << M) * sizeof(double), s>>>(n, M, G, partial);
    k_moments_final<<<(nout + 127) / 128, 128, 0, s>>>((int)nb, nout, partial, out);
    return cudaGetLastError();
}

__global__ void k_sum_slots(const double* slots, int nb, int count, double* out) {
    __shared__ double red[256];
    for (int q = 0; q < count; ++q) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += slots[q * kRedBlocks + b];
        red[threadIdx.x] = a;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = red[0];
        __syncthreads();
    }
}

// Phase gauge on the device. rec holds <ybar, H y_s> (re, im) and <ybar, y_s>
// (re, im) of this segment; bt holds <ybar_T, y_T> (copied from the first segment
// processed). Writes rot = e^{-i th} with th = arg(bt) - arg(<ybar, y_s>), and
// rec[4] = dL/dt_s = Im(e^{i th} <ybar, H y_s>).
__global__ void k_gauge(double* rec, double* bt, int first, double* rot) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (first) {
        bt[0] = rec[2];
        bt[1] = rec[3];
    }
    double th = 0.0;
    if (hypot(rec[2], rec[3]) > 1e-300 && hypot(bt[0], bt[1]) > 1e-300)
        th = atan2(bt[1], bt[0]) - atan2(rec[3], rec[2]);
    const double c = cos(th), s = sin(th);
    rot[0] = c;
    rot[1] = -s;
    rec[4] = s * rec[0] + c * rec[1];
}

// rot = e^{-i th0}, th0 = arg(bt) - arg(b0) (1 when either is ~0).
__global__ void k_gauge_final(const double* b0, const double* bt, double* rot) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double th = 0.0;
    if (hypot(b0[0], b0[1]) > 1e-300 && hypot(bt[0], bt[1]) > 1e-300) th = atan2(bt[1], bt[0]) - atan2(b0[1], b0[0]);
    rot[0] = cos(th);
    rot[1] = -sin(th);
}

// v *= rot[0] + i rot[1] (rot on the device).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_rotate(int64_t N, void* v_, const double* rot) {
    using C = typename Cx<R>::T;
    C* v = (C*)v_;
    const R cr = (R)rot[0], ci = (R)rot[1];
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const C x = v[z];
        C o;
        o.x = cr * x.x - ci * x.y;
        o.y = cr * x.y + ci * x.x;
        v[z] = o;
    }
}

unsigned grid_n(int64_t N) {
    int64_t b = (N + kAdjThreads - 1) / kAdjThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kRedBlocks));
}

// Workspace of the adjoint: the forward layout (whose two Clenshaw vectors start the
// ring of adjoint vectors), four more ring vectors, G (FP64 per element), Gs (8 bytes
// per element), reduction slots, gradient outputs, then a pool of state vectors that
// holds either every b_k of a segment or a ring of 6 plus anchor pairs.
constexpr int kRing = kAccBatch + 2;
// per-segment results stay on the device and are read back every kRecBatch segments:
// record = <ybar,Hy> (2), <ybar,y> (2), dL/dt, hsum, flip sum, unused
constexpr int kRecBatch = 64;
constexpr int kRecLen = 8;
constexpr int kOutGauge = 8;  // bt (2), rot (2), <psibar_0, psi_0> (2)
struct AdjLayout {
    Layout fwd;
    size_t ring[kRing];
    size_t G, Gs, slots, outs, jq0, tiles0, elow0, moments, pool;
    size_t vstride;
    size_t total_fixed;
};

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

AdjLayout adj_layout(int n, int prec) {
    AdjLayout A;
    A.fwd = make_layout(n, prec);
    const size_t vb = ((size_t)1 << n) * A.fwd.cbytes;
    A.vstride = a256(vb);
    size_t off = a256(A.fwd.total);
    A.ring[0] = A.fwd.b0;
    A.ring[1] = A.fwd.b1;
    for (int i = 2; i < kRing; ++i) {
        A.ring[i] = off;
        off += A.vstride;
    }
    A.G = off;
    off = a256(off + ((size_t)1 << n) * sizeof(double));
    A.Gs = off;
    off = a256(off + ((size_t)1 << n) * 8);  // float-float (FP32) or double (FP64)
    A.slots = off;
    off = a256(off + 4 * (size_t)kRedBlocks * sizeof(double));
    A.outs = off;
    off = a256(off + ((size_t)n * n + n + 16 + kOutGauge + kRecBatch * kRecLen) * sizeof(double));
    A.jq0 = off;  // unscaled fixed-point couplings and their energy tables (general segments)
    off = a256(off + ((size_t)n * n + n + 1) * sizeof(int64_t));
    A.tiles0 = off;
    off = a256(off + ((size_t)1 << (n - A.fwd.M)) * (A.fwd.M + 1) * sizeof(int64_t));
    A.elow0 = off;
    off = a256(off + ((size_t)1 << A.fwd.M) * sizeof(int64_t));
    A.moments = off;  // per-block partial sums of the dh, dJ moments
    off = a256(off + (size_t)kRedBlocks * ((size_t)n + (size_t)n * (n - 1) / 2) * sizeof(double));
    A.pool = off;
    A.total_fixed = off;
    return A;
}

// One Clenshaw-form step out = scale (D b1 + g sum_j X_j b1) + sgn b2 + ck psi on the
// fastest kernel available for (n, precision).
struct StepRunner {
    bool fused = false;
    FusedPlan plan;
    int prec = 0;
    int* flags = nullptr;
    void* scratch = nullptr;  // the fused kernels' scratch vectors of the forward layout
    cudaError_t run(const StepArgs& a, cudaStream_t s) const {
        if (fused) return launch_step_fused(plan, a, scratch, flags, s);
        launch_step_plain(prec, a, s);
        return cudaGetLastError();
    }
};

StepRunner make_runner(const Ctx& C, const AdjLayout& A, int n, int precision) {
    StepRunner R;
    R.prec = precision;
    R.flags = C.flags();
    R.scratch = C.ws + A.fwd.coef + (size_t)(kMaxK + 1) * 2 * sizeof(double);
    R.fused = fused_supported(n, precision) && n > (precision == CHEB_FP32 ? kSmallMaxF32 : kSmallMaxF64);
    if (R.fused) R.plan = fused_plan(n, precision);
    return R;
}

// One segment's operator and series: H_s = b_s H_P + gamma_s sum_j X_j on the frozen
// interval (b_s c, r_s), its fixed-point tables (uploaded) and coefficients.
struct Segment {
    double bsc = 1.0, c = 0.0, r = 1.0, g = 0.0;
    FixedOp F;
    std::vector<std::complex<double>> coef;
    int K = -1;
};

cheb_status_t segment_setup(const Ctx& C, int n, const double* h, const double* J, const double* b_s,
                            const double* gamma_s, const double* t_s, int s, double emin, double emax, double tol_s,
                            cheb_method_t method, Segment& G) {
    G.bsc = b_s ? b_s[s] : 1.0;
    G.c = G.bsc * 0.5 * (emax + emin);
    G.r = std::fabs(G.bsc) * 0.5 * (emax - emin) + std::fabs(gamma_s[s]) * n;
    if (!(G.r > 0)) G.r = 1.0;
    G.g = gamma_s[s] / G.r;
    std::vector<double> hb(n), Jb((size_t)n * n);
    for (int i = 0; i < n; ++i) hb[i] = G.bsc * h[i];
    for (size_t q = 0; q < (size_t)n * n; ++q) Jb[q] = G.bsc * J[q];
    G.F = make_fixed(n, hb.data(), Jb.data(), G.c, G.r, C.prec == CHEB_FP32 ? kMaxQF32 : 62);
    if (G.F.Q < 24) return CHEB_ERR_UNSUPPORTED;
    cheb_status_t st = upload_tables(C, G.F);
    if (st != CHEB_OK) return st;
    int slices = 1;
    double err = 0.0;
    st = slice_coefficients(t_s[s], G.c, G.r, tol_s, method, 0, G.coef, &G.K, &slices, &err);
    if (st != CHEB_OK) return st;
    return slices == 1 ? CHEB_OK : CHEB_ERR_UNSUPPORTED;
}

StepArgs segment_base(const Ctx& C, const AdjLayout& A, const Segment& G) {
    StepArgs b{};
    b.n = C.n;
    b.M = A.fwd.M;
    b.Q = G.F.Q;
    b.tiles = C.tiles();
    b.elow = C.elow();
    b.jq = (const int64_t*)(C.ws + A.fwd.jq);
    b.g = G.g;
    return b;
}

// Where the b_k of a segment of degree K live: all of them in the pool (store), or a
// ring of kRing regenerated upward from anchor pairs (b_a, b_{a+1}) every `gap` steps.
struct SegPool {
    unsigned char* pool = nullptr;
    size_t vstride = 0;
    int K = 0;
    bool store = true;
    int n_anch = 0, gap = 0;
    SegPool(unsigned char* p, size_t vs, int K_, int64_t nvec) : pool(p), vstride(vs), K(K_) {
        store = nvec >= K;
        if (!store) {
            n_anch = (int)std::min<int64_t>(std::max<int64_t>(0, (nvec - kRing) / 2), 1 << 16);
            gap = std::max(1, (K - 1 + n_anch) / (n_anch + 1));
        }
    }
    static bool fits(int K, int64_t nvec) { return nvec >= K || nvec >= kRing + 2; }
    unsigned char* bvec(int j) const {  // b_j, 1 <= j <= K
        return store ? pool + (size_t)(j - 1) * vstride : pool + (size_t)(j % kRing) * vstride;
    }
    int anchor_slot(int a) const {  // anchor pair index for b_a, or -1
        if (store || a < 1 + gap || (a - 1) % gap != 0 || a > K - 2) return -1;
        const int m = (a - 1) / gap - 1;
        return m < n_anch ? m : -1;
    }
    unsigned char* anchor_ptr(int m, int which) const { return pool + (size_t)(kRing + 2 * m + which) * vstride; }
};

// The segment's forward Clenshaw vectors b_K .. b_1 from its start state psi_s into
// the pool (Algorithm 2's recurrence on the step kernels), saving the anchor pairs.
// Afterwards b_1 .. b_min(K, kRing) (every b_k when storing) are in their slots.
cheb_status_t forward_fill(const SegPool& P, const StepRunner& runner, const StepArgs& base,
                           const std::vector<std::complex<double>>& coef, const void* psi_s, int prec, int64_t N,
                           size_t vb, cudaStream_t s0) {
    const int K = P.K;
    launch_scale(prec, N, psi_s, P.bvec(K), coef[K].real(), coef[K].imag(), s0);
    for (int j = K - 1; j >= 1; --j) {
        StepArgs a = base;
        a.b1 = P.bvec(j + 1);
        a.b2 = (j + 2 <= K) ? P.bvec(j + 2) : P.bvec(j);  // not read when sgn = 0
        a.psi = psi_s;
        a.out = P.bvec(j);
        a.ck_re = coef[j].real();
        a.ck_im = coef[j].imag();
        a.scale = 2.0;
        a.sgn = (j + 2 <= K) ? -1.0 : 0.0;
        if (runner.run(a, s0) != cudaSuccess) return CHEB_ERR_CUDA;
        const int m = P.anchor_slot(j);
        if (m >= 0) {
            CUDA_TRY(cudaMemcpyAsync(P.anchor_ptr(m, 0), P.bvec(j), vb, cudaMemcpyDeviceToDevice, s0));
            CUDA_TRY(cudaMemcpyAsync(P.anchor_ptr(m, 1), P.bvec(j + 1), vb, cudaMemcpyDeviceToDevice, s0));
        }
    }
    return CHEB_OK;
}

// Checkpoints left by cheb_anneal(_general)_checkpointed: the last segment's pool is
// filled, so the next adjoint call on the same workspace with the same arguments
// skips that segment's forward recomputation. Any adjoint call on the workspace
// consumes the record (the pool is overwritten by the adjoint).
struct Checkpoint {
    const void* ws = nullptr;
    size_t ws_bytes = 0;
    int n = 0, S = 0, prec = 0, method = 0;
    double tol = 0.0;
    uint64_t hash = 0;
    const void* psi_T = nullptr;
    const void* boundaries = nullptr;
    bool operator==(const Checkpoint& o) const {
        return ws == o.ws && ws_bytes == o.ws_bytes && n == o.n && S == o.S && prec == o.prec &&
               method == o.method && tol == o.tol && hash == o.hash && psi_T == o.psi_T &&
               boundaries == o.boundaries;
    }
};

std::mutex g_ck_mu;
std::vector<Checkpoint> g_ck;

// FNV-1a over the schedule and couplings (b_s absent hashes as a marker).
uint64_t schedule_hash(int n, const double* h, const double* J, int S, const double* b_s, const double* a_s,
                       const double* t_s) {
    uint64_t x = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t bytes) {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < bytes; ++i) x = (x ^ c[i]) * 1099511628211ull;
    };
    mix(h, sizeof(double) * n);
    mix(J, sizeof(double) * n * n);
    mix(a_s, sizeof(double) * S);
    mix(t_s, sizeof(double) * S);
    const int has_b = b_s ? 1 : 0;
    mix(&has_b, sizeof(has_b));
    if (b_s) mix(b_s, sizeof(double) * S);
    return x;
}

void checkpoint_put(const Checkpoint& k) {
    std::lock_guard<std::mutex> lk(g_ck_mu);
    g_ck.erase(std::remove_if(g_ck.begin(), g_ck.end(), [&](const Checkpoint& c) { return c.ws == k.ws; }),
               g_ck.end());
    g_ck.push_back(k);
}

// Removes the workspace's record; true when it matches k.
bool checkpoint_take(const Checkpoint& k) {
    std::lock_guard<std::mutex> lk(g_ck_mu);
    bool hit = false;
    for (auto it = g_ck.begin(); it != g_ck.end();) {
        if (it->ws == k.ws) {
            hit = hit || (*it == k);
            it = g_ck.erase(it);
        } else {
            ++it;
        }
    }
    return hit;
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" size_t cheb_adjoint_workspace_bytes(int n, cheb_precision_t precision, int store_vectors) {
    if (n < 1 || n > kMaxQubits || store_vectors < 0) return 0;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return 0;
    AdjLayout A = adj_layout(n, precision);
    return A.total_fixed + (size_t)store_vectors * A.vstride;
}

namespace {

// Gradient of a loss on the output of a schedule of segments H_s = b_s H_P + gamma_s
// sum_j X_j (b_s = 1 when b_s is null; S = 1: a single exp(-itH) psi). With the centre
// b_s c and radius r_s = |b_s| (Emax - Emin)/2 + |gamma_s| n frozen, D_s = (b_s E - b_s c)/r_s,
// so dL/db_s = sum_z G_s(z) E(z) / r_s and dh, dJ collect b_s / r_s times the moments of G_s.
cheb_status_t adjoint_impl(int n, const double* h, const double* J, int S, const double* b_s,
                           const double* gamma_s, const double* t_s, const void* boundaries, const void* psi_T,
                           void* grad, cheb_precision_t precision, double tol, cheb_method_t method,
                           double* grad_gamma, double* grad_b, double* grad_t, double* grad_h, double* grad_J,
                           void* workspace, size_t ws_bytes, void* stream) {
    if (n < 1 || n > kMaxQubits || S < 1 || !h || !J || !gamma_s || !t_s || !boundaries || !psi_T || !grad)
        return CHEB_ERR_INVALID_ARG;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(h, n) || !finite_all(J, (size_t)n * n) || !finite_all(gamma_s, S) || !finite_all(t_s, S) ||
        (b_s && !finite_all(b_s, S)))
        return CHEB_ERR_INVALID_ARG;
    if (!(tol > 0) || !std::isfinite(tol)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    if (((uintptr_t)boundaries | (uintptr_t)psi_T | (uintptr_t)grad) & 15) return CHEB_ERR_INVALID_ARG;
    AdjLayout A = adj_layout(n, precision);
    if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < A.total_fixed) return CHEB_ERR_WORKSPACE;
    const int64_t nvec = (int64_t)std::min<size_t>((ws_bytes - A.total_fixed) / A.vstride, 1 << 20);
    unsigned char* ws = (unsigned char*)workspace;
    cudaStream_t s0 = (cudaStream_t)stream;
    Ctx C{n, precision, A.fwd, ws, s0};
    const int64_t N = (int64_t)1 << n;
    const size_t vb = (size_t)N * A.fwd.cbytes;
    const unsigned gb = grid_n(N);
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
    CUDA_TRY(cudaMemsetAsync(ws + A.G, 0, (size_t)N * sizeof(double), s0));
    double emin = 0, emax = 0;
    cheb_status_t st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    const double tol_s = tol / S;
    // unscaled energy tables for dL/db_s (general segments only)
    int Q0 = 0;
    if (b_s && grad_b) {
        FixedOp F0 = make_fixed(n, h, J, 0.0, 1.0);
        Q0 = F0.Q;
        CUDA_TRY(cudaMemcpyAsync(ws + A.jq0, F0.jq.data(), F0.jq.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                 s0));
        launch_tables(n, A.fwd.M, (const int64_t*)(ws + A.jq0), (int64_t*)(ws + A.tiles0), (int64_t*)(ws + A.elow0),
                      s0);
        CUDA_TRY(cudaGetLastError());
    }
    std::vector<double> gb_out(S, 0.0);
    double* slots = (double*)(ws + A.slots);
    double* outs = (double*)(ws + A.outs);
    unsigned char* pool = ws + A.pool;
    unsigned char* Gs = ws + A.Gs;
    auto ring = [&](int k) { return ws + A.ring[k % kRing]; };  // bbar_k
    std::vector<double> gg(S), gt(S);
    const int Mt = A.fwd.M;
    const StepRunner runner = make_runner(C, A, n, precision);
    // the last segment's pool may already hold its forward vectors
    Checkpoint key;
    key.ws = workspace;
    key.ws_bytes = ws_bytes;
    key.n = n;
    key.S = S;
    key.prec = precision;
    key.method = method;
    key.tol = tol;
    key.hash = schedule_hash(n, h, J, S, b_s, gamma_s, t_s);
    key.psi_T = psi_T;
    key.boundaries = boundaries;
    const bool have_ckpt = checkpoint_take(key);
    double* gauge = outs + (size_t)n * n + n + 16;
    double* bt = gauge;       // <ybar_T, y_T>
    double* rot = gauge + 2;  // e^{-i th} of the current segment
    double* b0 = gauge + 4;   // <psibar_0, psi_0>
    double* recs = gauge + kOutGauge;
    std::vector<double> seg_r(S, 1.0);
    std::vector<int> seg_K(S, 0);
    for (int s = S - 1; s >= 0; --s) {
        Segment G;
        st = segment_setup(C, n, h, J, b_s, gamma_s, t_s, s, emin, emax, tol_s, method, G);
        if (st != CHEB_OK) return st;
        const double bsc = G.bsc, c = G.c, r = G.r;
        const FixedOp& F = G.F;
        const std::vector<std::complex<double>>& coef = G.coef;
        const int K = G.K;
        const void* psi_s = (const unsigned char*)boundaries + (size_t)s * vb;
        const void* y_s = (s == S - 1) ? psi_T : (const unsigned char*)boundaries + (size_t)(s + 1) * vb;
        // <ybar, H y_s> and the gauge invariant <ybar, y_s> into this segment's record;
        // the gauge rotation of ybar happens on the device (no host round trip)
        const int q = (S - 1 - s) % kRecBatch;
        double* rec = recs + (size_t)q * kRecLen;
        seg_r[s] = r;
        seg_K[s] = K;
        {
            CUDA_TRY(cudaMemsetAsync(slots, 0, 4 * kRedBlocks * sizeof(double), s0));
            note_launch(kKindReduce);
            const size_t dsm = ((size_t)1 << Mt) * A.fwd.cbytes;
            if (precision == CHEB_FP32)
                k_dt<float><<<grid_tiles(n, Mt), kAdjThreads, dsm, s0>>>(n, Mt, F.Q, C.tiles(), C.elow(), c, r,
                                                                        gamma_s[s], grad, y_s, slots);
            else
                k_dt<double><<<grid_tiles(n, Mt), kAdjThreads, dsm, s0>>>(n, Mt, F.Q, C.tiles(), C.elow(), c, r,
                                                                         gamma_s[s], grad, y_s, slots);
            k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, 4, rec);
            k_gauge<<<1, 32, 0, s0>>>(rec, bt, s == S - 1 ? 1 : 0, rot);
            // Re(e^{i th} conj(u) x) = Re(conj(e^{-i th} u) x): the gauge moves into ybar
            if (precision == CHEB_FP32) k_rotate<float><<<gb, kAdjThreads, 0, s0>>>(N, grad, rot);
            else k_rotate<double><<<gb, kAdjThreads, 0, s0>>>(N, grad, rot);
            CUDA_TRY(cudaMemsetAsync(rec + 5, 0, 3 * sizeof(double), s0));
        }
        auto flush = [&]() -> cheb_status_t {  // read back the records of segments s .. s + q
            std::vector<double> h((size_t)(q + 1) * kRecLen);
            CUDA_TRY(cudaMemcpyAsync(h.data(), recs, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s0));
            CUDA_TRY(cudaStreamSynchronize(s0));
            for (int i = 0; i <= q; ++i) {
                const int sg = S - 1 - ((S - 1 - s) - q + i);
                const double* v = h.data() + (size_t)i * kRecLen;
                gt[sg] = v[4];
                // hsum = sum_k w_k Re <bbar_k, (Ht - D) b_{k+1}> = gamma dL/dgamma
                if (seg_K[sg] == 0) gg[sg] = 0.0;
                else if (gamma_s[sg] == 0.0) gg[sg] = v[6] / seg_r[sg];
                else gg[sg] = v[5] / gamma_s[sg];
                gb_out[sg] = seg_K[sg] == 0 ? 0.0 : v[7] / seg_r[sg];
            }
            return CHEB_OK;
        };
        if (K == 0) {
            // y = c_0 psi: psibar = conj(c_0) ybar, no operator dependence
            launch_scale(precision, N, grad, grad, coef[0].real(), -coef[0].imag(), s0);
            if (q == kRecBatch - 1 || s == 0) {
                st = flush();
                if (st != CHEB_OK) return st;
            }
            continue;
        }
        if (!SegPool::fits(K, nvec)) return CHEB_ERR_WORKSPACE;
        const SegPool P(pool, A.vstride, K, nvec);
        const bool store = P.store;
        auto bvec = [&](int j) { return P.bvec(j); };
        const StepArgs base = segment_base(C, A, G);
        // forward recomputation from psi_s down to b_1 (already done by a checkpointed
        // forward for the last segment)
        if (!(have_ckpt && s == S - 1)) {
            st = forward_fill(P, runner, base, coef, psi_s, precision, N, vb, s0);
            if (st != CHEB_OK) return st;
        }
        int have = store ? K : std::min(K, kRing);  // b_1 .. b_have are current
        // b_0 := y; bbar_0 = ybar moves into the ring and grad accumulates psibar
        CUDA_TRY(cudaMemcpyAsync(ring(0), grad, vb, cudaMemcpyDeviceToDevice, s0));
        CUDA_TRY(cudaMemsetAsync(slots, 0, 4 * kRedBlocks * sizeof(double), s0));
        CUDA_TRY(cudaMemsetAsync(Gs, 0, (size_t)N * 8, s0));
        const bool use_flip = gamma_s[s] == 0.0;
        auto bk = [&](int j) -> const void* {  // b_j for 0 <= j <= K + 1
            if (j == 0) return y_s;
            if (j > K) return nullptr;
            return bvec(j);
        };
        for (int k0 = 0; k0 <= K; k0 += kAccBatch) {
            const int k1 = std::min(k0 + kAccBatch - 1, K);
            // bbar_k = alpha Ht bbar_{k-1} - beta bbar_{k-2}: Clenshaw-form steps with c = 0
            for (int k = std::max(k0, 1); k <= k1; ++k) {
                StepArgs a = base;
                a.b1 = ring(k - 1);
                a.b2 = (k >= 2) ? ring(k - 2) : ring(k);  // not read when sgn = 0
                a.psi = ring(k - 1);                      // multiplied by c = 0
                a.out = ring(k);
                a.ck_re = 0.0;
                a.ck_im = 0.0;
                a.scale = (k == 1) ? 1.0 : 2.0;
                a.sgn = (k == 1) ? 0.0 : -1.0;
                if (runner.run(a, s0) != cudaSuccess) return CHEB_ERR_CUDA;
            }
            // b_j up to k1 + 2: b_j = 2 Ht b_{j-1} - b_{j-2} + c_{j-2} psi, resetting
            // (b_{j-2}, b_{j-1}) from an anchor where there is one
            const int need = std::min(k1 + 2, K);
            for (int j = have + 1; j <= need; ++j) {
                const int m = P.anchor_slot(j - 2);
                if (m >= 0) {
                    CUDA_TRY(cudaMemcpyAsync(bvec(j - 2), P.anchor_ptr(m, 0), vb, cudaMemcpyDeviceToDevice, s0));
                    CUDA_TRY(cudaMemcpyAsync(bvec(j - 1), P.anchor_ptr(m, 1), vb, cudaMemcpyDeviceToDevice, s0));
                }
                StepArgs a = base;
                a.b1 = bvec(j - 1);
                a.b2 = bvec(j - 2);
                a.psi = psi_s;
                a.out = bvec(j);
                a.ck_re = coef[j - 2].real();
                a.ck_im = coef[j - 2].imag();
                a.scale = 2.0;
                a.sgn = -1.0;
                if (runner.run(a, s0) != cudaSuccess) return CHEB_ERR_CUDA;
            }
            have = std::max(have, need);
            AccArgs x{};
            x.n = n;
            x.m = k1 - k0 + 1;
            x.mode = (k0 == 0) ? 2 : 1;
            x.M = Mt;
            x.Q = F.Q;
            x.tiles = C.tiles();
            x.elow = C.elow();
            x.psi = psi_s;
            x.psibar = grad;
            x.Gs = Gs;
            x.slots = slots;
            for (int i = 0; i < x.m; ++i) {
                const int k = k0 + i;
                x.bbar[i] = ring(k);
                x.cc_re[i] = coef[k].real();
                x.cc_im[i] = -coef[k].imag();
                x.w[i] = (k <= K - 1) ? (k == 0 ? 1.0 : 2.0) : 0.0;
            }
            for (int j = 0; j < x.m + 2; ++j) x.fb[j] = bk(k0 + j);
            note_launch(kKindReduce);
            const int pi = prof_begin(kKindReduce, s0);
            if (precision == CHEB_FP32) k_adj_acc_f32x2<<<grid_tiles(n, Mt), kAdjThreads, 0, s0>>>(x);
            else k_adj_acc<double><<<grid_tiles(n, Mt), kAdjThreads, 0, s0>>>(x);
            prof_end(pi, s0);
            CUDA_TRY(cudaGetLastError());
            if (use_flip) {
                for (int i = 0; i < x.m; ++i) {
                    if (x.w[i] == 0.0) continue;
                    note_launch(kKindReduce);
                    double* sl = slots + kRedBlocks;
                    if (precision == CHEB_FP32)
                        k_dg_flip<float><<<gb, kAdjThreads, 0, s0>>>(n, x.bbar[i], x.fb[i + 1], x.w[i], sl);
                    else
                        k_dg_flip<double><<<gb, kAdjThreads, 0, s0>>>(n, x.bbar[i], x.fb[i + 1], x.w[i], sl);
                }
            }
        }
        // slots: [0] hsum, [1] flip sums (gamma = 0), [2] sum_z Gs E (general) -> record [5..7]
        note_launch(kKindReduce);
        const int64_t* t0p = (b_s && grad_b) ? (const int64_t*)(ws + A.tiles0) : nullptr;
        const int64_t* e0p = (const int64_t*)(ws + A.elow0);
        if (precision == CHEB_FP32)
            k_fold<float><<<gb, kAdjThreads, 0, s0>>>(n, (const float*)Gs, bsc / r, (double*)(ws + A.G), Mt, Q0, t0p,
                                                      e0p, slots + 2 * kRedBlocks);
        else
            k_fold<double><<<gb, kAdjThreads, 0, s0>>>(n, (const double*)Gs, bsc / r, (double*)(ws + A.G), Mt, Q0,
                                                       t0p, e0p, slots + 2 * kRedBlocks);
        k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, 3, rec + 5);
        if (q == kRecBatch - 1 || s == 0) {
            st = flush();
            if (st != CHEB_OK) return st;
        }
    }
    // the returned psibar carries the accumulated relative phase drift; remove it
    {
        CUDA_TRY(cudaMemsetAsync(slots, 0, 2 * kRedBlocks * sizeof(double), s0));
        note_launch(kKindReduce);
        if (precision == CHEB_FP32)
            k_dot<float><<<gb, kAdjThreads, 0, s0>>>(n, grad, boundaries, slots);
        else
            k_dot<double><<<gb, kAdjThreads, 0, s0>>>(n, grad, boundaries, slots);
        k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, 2, b0);
        k_gauge_final<<<1, 32, 0, s0>>>(b0, bt, rot);
        if (precision == CHEB_FP32) k_rotate<float><<<gb, kAdjThreads, 0, s0>>>(N, grad, rot);
        else k_rotate<double><<<gb, kAdjThreads, 0, s0>>>(N, grad, rot);
    }
    // dh, dJ from G (already divided by r per segment)
    const int nblk = n + n * (n - 1) / 2;
    CUDA_TRY(launch_moments(n, (const double*)(ws + A.G), (double*)(ws + A.moments), outs, s0));
    std::vector<double> red(nblk);
    CUDA_TRY(cudaMemcpyAsync(red.data(), outs, nblk * sizeof(double), cudaMemcpyDeviceToHost, s0));
    st = read_flags(C);
    if (st != CHEB_OK) return st;
    if (grad_gamma)
        for (int s = 0; s < S; ++s) grad_gamma[s] = gg[s];
    if (grad_b)
        for (int s = 0; s < S; ++s) grad_b[s] = gb_out[s];
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

}  // namespace

extern "C" cheb_status_t cheb_anneal_adjoint(int n, const double* h, const double* J, int S, const double* gamma_s,
                                             const double* t_s, const void* boundaries, const void* psi_T,
                                             void* grad, cheb_precision_t precision, double tol,
                                             cheb_method_t method, double* grad_gamma, double* grad_t,
                                             double* grad_h, double* grad_J, void* workspace, size_t ws_bytes,
                                             void* stream) {
    return adjoint_impl(n, h, J, S, nullptr, gamma_s, t_s, boundaries, psi_T, grad, precision, tol, method,
                        grad_gamma, nullptr, grad_t, grad_h, grad_J, workspace, ws_bytes, stream);
}

extern "C" cheb_status_t cheb_anneal_general_adjoint(int n, const double* h, const double* J, int S,
                                                     const double* a_s, const double* b_s, const double* t_s,
                                                     const void* boundaries, const void* psi_T, void* grad,
                                                     cheb_precision_t precision, double tol, cheb_method_t method,
                                                     double* grad_a, double* grad_b, double* grad_t,
                                                     double* grad_h, double* grad_J, void* workspace,
                                                     size_t ws_bytes, void* stream) {
    if (!b_s) return CHEB_ERR_INVALID_ARG;
    return adjoint_impl(n, h, J, S, b_s, a_s, t_s, boundaries, psi_T, grad, precision, tol, method, grad_a, grad_b,
                        grad_t, grad_h, grad_J, workspace, ws_bytes, stream);
}

namespace {

// Forward run of a schedule for a later adjoint call: segments 0..S-2 as in
// cheb_anneal_general, then the last segment on the adjoint's own step runner with its
// Clenshaw vectors placed in the adjoint workspace's pool (every b_k, or the ring and
// anchor pairs), and y = Ht b_1 - b_2 + c_0 psi_s (Algorithm 2's final step) into psi.
cheb_status_t checkpointed_impl(int n, const double* h, const double* J, int S, const double* b_s,
                                const double* gamma_s, const double* t_s, void* psi, cheb_precision_t precision,
                                double tol, cheb_method_t method, void* boundaries, void* workspace, size_t ws_bytes,
                                void* stream) {
    if (n < 1 || n > kMaxQubits || S < 1 || !h || !J || !gamma_s || !t_s || !psi || !boundaries)
        return CHEB_ERR_INVALID_ARG;
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (!finite_all(h, n) || !finite_all(J, (size_t)n * n) || !finite_all(gamma_s, S) || !finite_all(t_s, S) ||
        (b_s && !finite_all(b_s, S)))
        return CHEB_ERR_INVALID_ARG;
    if (!(tol > 0) || !std::isfinite(tol)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    if (((uintptr_t)boundaries | (uintptr_t)psi) & 15) return CHEB_ERR_INVALID_ARG;
    AdjLayout A = adj_layout(n, precision);
    if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < A.total_fixed) return CHEB_ERR_WORKSPACE;
    const int64_t nvec = (int64_t)std::min<size_t>((ws_bytes - A.total_fixed) / A.vstride, 1 << 20);
    // the workspace's pool is about to change: no earlier checkpoint of it stays valid
    Checkpoint key;
    key.ws = workspace;
    checkpoint_take(key);
    unsigned char* ws = (unsigned char*)workspace;
    cudaStream_t s0 = (cudaStream_t)stream;
    Ctx C{n, precision, A.fwd, ws, s0};
    const int64_t N = (int64_t)1 << n;
    const size_t vb = (size_t)N * A.fwd.cbytes;
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
    double emin = 0, emax = 0;
    cheb_status_t st = bounds_impl(C, h, J, &emin, &emax);
    if (st != CHEB_OK) return st;
    // the last segment's degree and time slicing, checked before psi changes
    {
        Segment G0;
        st = segment_setup(C, n, h, J, b_s, gamma_s, t_s, S - 1, emin, emax, tol / S, method, G0);
        if (st != CHEB_OK) return st;
        if (G0.K > 0 && !SegPool::fits(G0.K, nvec)) return CHEB_ERR_WORKSPACE;
    }
    if (S > 1) {
        // the adjoint workspace starts with a forward workspace
        st = anneal_run(n, h, J, S, b_s, gamma_s, t_s, psi, precision, tol, method, boundaries, workspace, ws_bytes,
                        stream, nullptr, S - 1);
        if (st != CHEB_OK) return st;
        CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
    }
    Segment G;
    st = segment_setup(C, n, h, J, b_s, gamma_s, t_s, S - 1, emin, emax, tol / S, method, G);
    if (st != CHEB_OK) return st;
    unsigned char* psi_s = (unsigned char*)boundaries + (size_t)(S - 1) * vb;
    CUDA_TRY(cudaMemcpyAsync(psi_s, psi, vb, cudaMemcpyDeviceToDevice, s0));
    const int K = G.K;
    if (K == 0) {
        launch_scale(precision, N, psi_s, psi, G.coef[0].real(), G.coef[0].imag(), s0);
    } else {
        const SegPool P(ws + A.pool, A.vstride, K, nvec);
        const StepRunner runner = make_runner(C, A, n, precision);
        const StepArgs base = segment_base(C, A, G);
        st = forward_fill(P, runner, base, G.coef, psi_s, precision, N, vb, s0);
        if (st != CHEB_OK) return st;
        StepArgs a = base;
        a.b1 = P.bvec(1);
        a.b2 = K >= 2 ? P.bvec(2) : P.bvec(1);  // not read when sgn = 0
        a.psi = psi_s;
        a.out = psi;
        a.ck_re = G.coef[0].real();
        a.ck_im = G.coef[0].imag();
        a.scale = 1.0;
        a.sgn = K >= 2 ? -1.0 : 0.0;
        if (runner.run(a, s0) != cudaSuccess) return CHEB_ERR_CUDA;
    }
    CUDA_TRY(cudaGetLastError());
    st = read_flags(C);
    if (st != CHEB_OK) return st;
    key.ws_bytes = ws_bytes;
    key.n = n;
    key.S = S;
    key.prec = precision;
    key.method = method;
    key.tol = tol;
    key.hash = schedule_hash(n, h, J, S, b_s, gamma_s, t_s);
    key.psi_T = psi;
    key.boundaries = boundaries;
    checkpoint_put(key);
    return CHEB_OK;
}

}  // namespace

extern "C" cheb_status_t cheb_anneal_checkpointed(int n, const double* h, const double* J, int S,
                                                  const double* gamma_s, const double* t_s, void* psi,
                                                  cheb_precision_t precision, double tol, cheb_method_t method,
                                                  void* boundaries, void* workspace, size_t ws_bytes, void* stream) {
    return checkpointed_impl(n, h, J, S, nullptr, gamma_s, t_s, psi, precision, tol, method, boundaries, workspace,
                             ws_bytes, stream);
}

extern "C" cheb_status_t cheb_anneal_general_checkpointed(int n, const double* h, const double* J, int S,
                                                          const double* a_s, const double* b_s, const double* t_s,
                                                          void* psi, cheb_precision_t precision, double tol,
                                                          cheb_method_t method, void* boundaries, void* workspace,
                                                          size_t ws_bytes, void* stream) {
    if (!b_s) return CHEB_ERR_INVALID_ARG;
    return checkpointed_impl(n, h, J, S, b_s, a_s, t_s, psi, precision, tol, method, boundaries, workspace,
                             ws_bytes, stream);
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
    k_sum_slots<<<1, 256, 0, s0>>>(slots, gb, 1, outs + n * n + n);
    const int nblk = n + n * (n - 1) / 2;
    CUDA_TRY(launch_moments(n, G, (double*)(ws + A.moments), outs, s0));
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
