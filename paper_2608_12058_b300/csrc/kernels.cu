// Device kernels of the single-pass path: energy tables, spectral bounds, the
// plain one-pass Clenshaw step (FP32 and FP64), the whole-run shared-memory
// kernel for small n, and the FP64 norm / energy reductions.
//
// Energies are exact sums of fixed-point integers. With the basis index split
// as z = (T, x), T = z >> M (tile) and x = z & (2^M - 1):
//   E(z) - c = A(T) + sum_{i<M} s_i(x) f_i(T) + elow(x),
//   f_i(T) = sum_{j>=M} J_ij s_j(T),
//   A(T)   = sum_{M<=i<j} J_ij s_i s_j + sum_{i>=M} h_i s_i - c,
//   elow(x)= sum_{i<j<M} J_ij s_i s_j + sum_{i<M} h_i s_i,
// which is the Ising diagonal of Sec. I regrouped by bit position and generated
// on the device from the couplings (Sec. III.A) instead of being stored.
#include <cuda_runtime.h>
#include <cstdint>

#include "cheb_internal.h"
#include "kernels.cuh"
#include "kernels_dev.cuh"

namespace cheb {


// ---------------------------------------------------------------------------
__global__ void k_tables(int n, int M, const int64_t* __restrict__ jq, int64_t* __restrict__ tiles,
                         int64_t* __restrict__ elow) {
    const int64_t ntiles = (int64_t)1 << (n - M);
    const int64_t nlow = (int64_t)1 << M;
    const int64_t* J = jq;
    const int64_t* h = jq + (size_t)n * n;
    const int64_t c = jq[(size_t)n * n + n];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ntiles + nlow;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (idx < ntiles) {
            const uint64_t zh = (uint64_t)idx << M;
            int64_t* row = tiles + idx * (M + 1);
            for (int i = 0; i < M; ++i) {
                int64_t f = 0;
                for (int j = M; j < n; ++j) f += sgn_sel((zh >> j) & 1, J[(size_t)i * n + j]);
                row[i] = f;
            }
            int64_t A = -c;
            for (int i = M; i < n; ++i) {
                int64_t hi = h[i];
                for (int j = i + 1; j < n; ++j) hi += sgn_sel((zh >> j) & 1, J[(size_t)i * n + j]);
                A += sgn_sel((zh >> i) & 1, hi);
            }
            row[M] = A;
        } else {
            const uint64_t x = (uint64_t)(idx - ntiles);
            int64_t e = 0;
            for (int i = 0; i < M; ++i) {
                int64_t hi = h[i];
                for (int j = i + 1; j < M; ++j) hi += sgn_sel((x >> j) & 1, J[(size_t)i * n + j]);
                e += sgn_sel((x >> i) & 1, hi);
            }
            elow[x] = e;
        }
    }
}

void launch_tables(int n, int M, const int64_t* jq, int64_t* tiles, int64_t* elow, cudaStream_t s) {
    int64_t total = ((int64_t)1 << (n - M)) + ((int64_t)1 << M);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4 * 148 * 8) blocks = 4 * 148 * 8;
    note_launch(kKindTables);
    k_tables<<<(unsigned)blocks, 256, 0, s>>>(n, M, jq, tiles, elow);
}

// ---------------------------------------------------------------------------
// Spectral bounds (Sec. II.A): exact min / max of the fixed-point energies.
__global__ void __launch_bounds__(256) k_minmax(int n, int M, const int64_t* __restrict__ tiles,
                                                const int64_t* __restrict__ elow,
                                                int64_t* __restrict__ part) {
    __shared__ int64_t f[kTileBits + 1];
    __shared__ int64_t rmin[256], rmax[256];
    const int64_t ntiles = (int64_t)1 << (n - M);
    const int nlow = 1 << M;
    int64_t mn = INT64_MAX, mx = INT64_MIN;
    for (int64_t T = blockIdx.x; T < ntiles; T += gridDim.x) {
        __syncthreads();
        if (threadIdx.x <= M) f[threadIdx.x] = tiles[T * (M + 1) + threadIdx.x];
        __syncthreads();
        const int64_t A = f[M];
        for (int x = threadIdx.x; x < nlow; x += blockDim.x) {
            int64_t e = A + elow[x];
            for (int i = 0; i < M; ++i) e += sgn_sel((x >> i) & 1, f[i]);
            mn = e < mn ? e : mn;
            mx = e > mx ? e : mx;
        }
    }
    rmin[threadIdx.x] = mn;
    rmax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rmin[threadIdx.x] = min(rmin[threadIdx.x], rmin[threadIdx.x + w]);
            rmax[threadIdx.x] = max(rmax[threadIdx.x], rmax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rmin[0];
        part[kRedBlocks + blockIdx.x] = rmax[0];
    }
}

__global__ void k_minmax_final(const int64_t* __restrict__ part, int nb, int64_t* __restrict__ out) {
    __shared__ int64_t rmin[256], rmax[256];
    int64_t mn = INT64_MAX, mx = INT64_MIN;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        mn = min(mn, part[b]);
        mx = max(mx, part[kRedBlocks + b]);
    }
    rmin[threadIdx.x] = mn;
    rmax[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rmin[threadIdx.x] = min(rmin[threadIdx.x], rmin[threadIdx.x + w]);
            rmax[threadIdx.x] = max(rmax[threadIdx.x], rmax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = rmin[0];
        out[1] = rmax[0];
    }
}

void launch_minmax(int n, int M, const int64_t* tiles, const int64_t* elow, int64_t* part,
                   int64_t* out2, cudaStream_t s) {
    int64_t ntiles = (int64_t)1 << (n - M);
    int nb = (int)(ntiles < kRedBlocks ? ntiles : kRedBlocks);
    note_launch(kKindMinmax);
    k_minmax<<<nb, 256, 0, s>>>(n, M, tiles, elow, part);
    note_launch(kKindMinmax);
    k_minmax_final<<<1, 256, 0, s>>>(part, nb, out2);
}

template <typename R>
__global__ void k_scale(int64_t N, const typename Cx<R>::T* __restrict__ src,
                        typename Cx<R>::T* dst, R cr, R ci) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N;
         z += (int64_t)gridDim.x * blockDim.x) {
        auto v = src[z];
        typename Cx<R>::T o;
        o.x = cr * v.x - ci * v.y;
        o.y = cr * v.y + ci * v.x;
        dst[z] = o;
    }
}

static unsigned grid_for(int64_t N, int threads, int64_t cap = (int64_t)148 * 64) {
    int64_t b = (N + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

void launch_scale(int prec, int64_t N, const void* src, void* dst, double cr, double ci, cudaStream_t s) {
    note_launch(kKindScale);
    if (prec == 0)
        k_scale<float><<<grid_for(N, 256), 256, 0, s>>>(N, (const float2*)src, (float2*)dst, (float)cr, (float)ci);
    else
        k_scale<double><<<grid_for(N, 256), 256, 0, s>>>(N, (const double2*)src, (double2*)dst, cr, ci);
}

// Plain one-pass step: every flip partner read straight from global memory.
template <typename R>
__global__ void __launch_bounds__(256) k_step_plain(StepArgs a, R ghi, R glo) {
    using C = typename Cx<R>::T;
    const int64_t N = (int64_t)1 << a.n;
    const C* __restrict__ b1 = (const C*)a.b1;
    const C* b2 = (const C*)a.b2;
    const C* psi = (const C*)a.psi;
    C* out = (C*)a.out;
    const R ckr = (R)a.ck_re, cki = (R)a.ck_im, sc = (R)a.scale, sg = (R)a.sgn;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N;
         z += (int64_t)gridDim.x * blockDim.x) {
        R sx = 0, sy = 0;
        for (int j = 0; j < a.n; ++j) {
            C p = b1[z ^ ((int64_t)1 << j)];
            sx += p.x;
            sy += p.y;
        }
        const C v = b1[z];
        const int64_t e = energy_fixed(a.M, a.tiles, a.elow, (uint64_t)z);
        R hx, hy;
        if constexpr (sizeof(R) == 4) {
            float dhi, dlo;
            fixed_to_ff(e, a.Q, dhi, dlo);
            hx = fmaf(dhi, v.x, dlo * v.x) + fmaf(ghi, sx, glo * sx);
            hy = fmaf(dhi, v.y, dlo * v.y) + fmaf(ghi, sy, glo * sy);
        } else {
            const double d = __ll2double_rn(e) * ldexp(1.0, -a.Q);
            hx = d * v.x + ghi * sx;
            hy = d * v.y + ghi * sy;
        }
        R ox = sc * hx, oy = sc * hy;
        if (a.sgn != 0.0) {
            const C w = b2[z];
            ox += sg * w.x;
            oy += sg * w.y;
        }
        const C p = psi[z];
        ox += ckr * p.x - cki * p.y;
        oy += ckr * p.y + cki * p.x;
        C o;
        o.x = ox;
        o.y = oy;
        out[z] = o;
    }
}

void launch_step_plain(int prec, const StepArgs& a, cudaStream_t s) {
    const int64_t N = (int64_t)1 << a.n;
    const unsigned grid = grid_for(N, 256, (int64_t)1 << 30);
    if (prec == 0) {
        float ghi = (float)a.g;
        float glo = (float)(a.g - (double)ghi);
        note_launch(kKindStepPlain);
        const int pi = prof_begin(kKindStepPlain, s);
        k_step_plain<float><<<grid, 256, 0, s>>>(a, ghi, glo);
        prof_end(pi, s);
    } else {
        note_launch(kKindStepPlain);
        const int pi = prof_begin(kKindStepPlain, s);
        k_step_plain<double><<<grid, 256, 0, s>>>(a, a.g, 0.0);
        prof_end(pi, s);
    }
}

// ---------------------------------------------------------------------------
// Small n: one CTA runs the whole recurrence with psi, b1, b2 in shared memory.
// Each thread owns the same elements for all steps and keeps their Dt in registers.
template <typename R, int PER>
__global__ void __launch_bounds__(1024) k_small(int n, int K, const double2* __restrict__ coef, int Q,
                                                const int64_t* __restrict__ tiles,
                                                const int64_t* __restrict__ elow, double g,
                                                typename Cx<R>::T* psi_g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    small_run<R, PER>(n, K, coef, Q, tiles, elow, g, psi_g, smem_raw);
}

// Many independent small instances, one CTA each (the batching of Sec. III.A with
// every instance keeping its own polynomial).
template <typename R, int PER>
__global__ void __launch_bounds__(1024) k_small_batched(const SmallDesc* __restrict__ d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmallDesc x = d[blockIdx.x];
    if (x.K <= 0) return;
    small_run<R, PER>(x.n, x.K, (const double2*)x.coef, x.Q, x.tiles, x.elow, x.g, (typename Cx<R>::T*)x.psi,
                      smem_raw);
}

cudaError_t launch_small_batched(int prec, int count, int max_n, const SmallDesc* descs, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int N = 1 << max_n;
    const int threads = N < 1024 ? (N < 32 ? 32 : N) : 1024;
    const size_t smem = 3 * (size_t)N * (prec == 0 ? 8 : 16);
    if (prec == 0) {
        auto kern = k_small_batched<float, 8>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        note_launch(kKindSmall);
        kern<<<count, threads, smem, s>>>(descs);
    } else {
        auto kern = k_small_batched<double, 4>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        note_launch(kKindSmall);
        kern<<<count, threads, smem, s>>>(descs);
    }
    return cudaGetLastError();
}

cudaError_t launch_small(int prec, int n, int K, const double* coef_dev, int Q, const int64_t* tiles,
                         const int64_t* elow, double g, void* psi, cudaStream_t s) {
    const int N = 1 << n;
    const int threads = N < 1024 ? (N < 32 ? 32 : N) : 1024;
    const size_t cb = prec == 0 ? 8 : 16;
    const size_t smem = 3 * (size_t)N * cb;
    if (prec == 0) {
        auto kern = k_small<float, 8>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        note_launch(kKindSmall);
        kern<<<1, threads, smem, s>>>(n, K, (const double2*)coef_dev, Q, tiles, elow, g, (float2*)psi);
    } else {
        auto kern = k_small<double, 4>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        note_launch(kKindSmall);
        kern<<<1, threads, smem, s>>>(n, K, (const double2*)coef_dev, Q, tiles, elow, g, (double2*)psi);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||y||^2 and <y|H_P|y> = sum_z (c + r Dt(z)) |y(z)|^2 in FP64, two-stage and
// deterministic (fixed block partition, fixed tree order).
template <typename R>
__global__ void __launch_bounds__(256) k_norm_energy(int n, int M, int Q, const int64_t* __restrict__ tiles,
                                                     const int64_t* __restrict__ elow, double c, double r,
                                                     const typename Cx<R>::T* __restrict__ y,
                                                     double* __restrict__ part) {
    __shared__ double sn[256], se[256];
    const int64_t N = (int64_t)1 << n;
    const double sc = ldexp(1.0, -Q);
    double an = 0.0, ae = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N;
         z += (int64_t)gridDim.x * blockDim.x) {
        const auto v = y[z];
        const double p2 = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        const double E = c + r * (__ll2double_rn(energy_fixed(M, tiles, elow, (uint64_t)z)) * sc);
        an += p2;
        ae += E * p2;
    }
    sn[threadIdx.x] = an;
    se[threadIdx.x] = ae;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sn[threadIdx.x] += sn[threadIdx.x + w];
            se[threadIdx.x] += se[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sn[0];
        part[kRedBlocks + blockIdx.x] = se[0];
    }
}

__global__ void k_sum2_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sn[256], se[256];
    double an = 0.0, ae = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        an += part[b];
        ae += part[kRedBlocks + b];
    }
    sn[threadIdx.x] = an;
    se[threadIdx.x] = ae;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sn[threadIdx.x] += sn[threadIdx.x + w];
            se[threadIdx.x] += se[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sn[0];
        out[1] = se[0];
    }
}

// ---------------------------------------------------------------------------
// Norms for the evaluation-error bound of Sec. II.B.3: out[0] += ||b||^2 and, when
// want_c, out_c[0] += ||c psi - b||^2, accumulated in FP64 (block tree, then one
// atomic add per block: the order of the block sums is not fixed, which only moves
// the last bits of a bound).
template <typename R>
__global__ void __launch_bounds__(256) k_step_norms(int64_t N, const typename Cx<R>::T* __restrict__ b,
                                                    const typename Cx<R>::T* __restrict__ psi, double cr,
                                                    double ci, int want_c, double* out_b, double* out_c) {
    __shared__ double sb[256], sc[256];
    double ab = 0.0, ac = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N;
         z += (int64_t)gridDim.x * blockDim.x) {
        const auto v = b[z];
        const double vx = (double)v.x, vy = (double)v.y;
        ab += vx * vx + vy * vy;
        if (want_c) {
            const auto p = psi[z];
            const double px = (double)p.x, py = (double)p.y;
            const double dx = cr * px - ci * py - vx, dy = cr * py + ci * px - vy;
            ac += dx * dx + dy * dy;
        }
    }
    sb[threadIdx.x] = ab;
    sc[threadIdx.x] = ac;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sb[threadIdx.x] += sb[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out_b, sb[0]);
        if (want_c) atomicAdd(out_c, sc[0]);
    }
}

// The same for float-float vectors (float4: re_hi, im_hi, re_lo, im_lo).
__global__ void __launch_bounds__(256) k_step_norms_ff(int64_t N, const float4* __restrict__ b,
                                                       const float4* __restrict__ psi, double cr, double ci,
                                                       int want_c, double* out_b, double* out_c) {
    __shared__ double sb[256], sc[256];
    double ab = 0.0, ac = 0.0;
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N;
         z += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = b[z];
        const double vx = (double)v.x + (double)v.z, vy = (double)v.y + (double)v.w;
        ab += vx * vx + vy * vy;
        if (want_c) {
            const float4 p = psi[z];
            const double px = (double)p.x + (double)p.z, py = (double)p.y + (double)p.w;
            const double dx = cr * px - ci * py - vx, dy = cr * py + ci * px - vy;
            ac += dx * dx + dy * dy;
        }
    }
    sb[threadIdx.x] = ab;
    sc[threadIdx.x] = ac;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sb[threadIdx.x] += sb[threadIdx.x + w];
            sc[threadIdx.x] += sc[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out_b, sb[0]);
        if (want_c) atomicAdd(out_c, sc[0]);
    }
}

void launch_step_norms(int prec, int64_t N, const void* b, const void* psi, double cr, double ci, int want_c,
                       double* out_b, double* out_c, cudaStream_t s) {
    const unsigned nb = grid_for(N, 256, kRedBlocks);
    note_launch(kKindReduce);
    if (prec == kFormatFF)
        k_step_norms_ff<<<nb, 256, 0, s>>>(N, (const float4*)b, (const float4*)psi, cr, ci, want_c, out_b, out_c);
    else if (prec == 0)
        k_step_norms<float><<<nb, 256, 0, s>>>(N, (const float2*)b, (const float2*)psi, cr, ci, want_c, out_b,
                                               out_c);
    else
        k_step_norms<double><<<nb, 256, 0, s>>>(N, (const double2*)b, (const double2*)psi, cr, ci, want_c, out_b,
                                                out_c);
}

void launch_norm_energy(int prec, int n, int M, int Q, const int64_t* tiles, const int64_t* elow,
                        double c, double r, const void* psi, double* part, double* out2, cudaStream_t s) {
    const int64_t N = (int64_t)1 << n;
    const int nb = (int)grid_for(N, 256, kRedBlocks);
    note_launch(kKindReduce);
    if (prec == 0)
        k_norm_energy<float><<<nb, 256, 0, s>>>(n, M, Q, tiles, elow, c, r, (const float2*)psi, part);
    else
        k_norm_energy<double><<<nb, 256, 0, s>>>(n, M, Q, tiles, elow, c, r, (const double2*)psi, part);
    note_launch(kKindReduce);
    k_sum2_final<<<1, 256, 0, s>>>(part, nb, out2);
}

}  // namespace cheb
