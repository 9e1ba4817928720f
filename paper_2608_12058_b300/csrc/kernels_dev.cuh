// Device helpers shared by the kernels of the single-pass paths (kernels.cu) and the
// persistent batch kernel (batch_team.cu): complex element types, the fixed-point
// Ising diagonal of the energy tables, and the whole-run shared-memory Clenshaw loop.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "cheb_internal.h"

namespace cheb {

__device__ __forceinline__ int64_t sgn_sel(uint64_t bit, int64_t v) { return bit ? -v : v; }

// ---------------------------------------------------------------------------
// Complex element types.
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// ---------------------------------------------------------------------------
// Dt(z) from the fixed-point tables.
__device__ __forceinline__ int64_t energy_fixed(int M, const int64_t* __restrict__ tiles,
                                                const int64_t* __restrict__ elow, uint64_t z) {
    const uint64_t T = z >> M;
    const uint64_t x = z & ((1ull << M) - 1);
    const int64_t* row = tiles + T * (M + 1);
    int64_t e = __ldg(row + M) + __ldg(elow + x);
    for (int i = 0; i < M; ++i) e += sgn_sel((x >> i) & 1, __ldg(row + i));
    return e;
}

// int64 at scale 2^-Q (Q <= 56, |value| <= 1) -> float-float: the high 32-bit word
// is exact in a float, the low word carries the next 24 bits.
__device__ __forceinline__ void fixed_to_ff(int64_t e, int Q, float& hi, float& lo) {
    const int eh = (int)(e >> 32);
    const unsigned el = (unsigned)(e & 0xffffffffll);
    hi = __int2float_rn(eh) * __int_as_float((127 + 32 - Q) << 23);
    lo = __uint2float_rn(el) * __int_as_float((127 - Q) << 23);
}

template <typename R, int PER>
__device__ __forceinline__ void small_run(int n, int K, const double2* __restrict__ coef, int Q,
                                          const int64_t* __restrict__ tiles, const int64_t* __restrict__ elow,
                                          double g, typename Cx<R>::T* psi_g, unsigned char* smem_raw) {
    using C = typename Cx<R>::T;
    const int N = 1 << n;
    C* sp = (C*)smem_raw;
    C* s1 = sp + N;
    C* s2 = s1 + N;
    const int M = n < kTileBits ? n : kTileBits;  // same split as the workspace tables
    R dhi[PER], dlo[PER];
    const double2 cK = coef[K];
    for (int q = 0; q < PER; ++q) {
        const int z = threadIdx.x + q * blockDim.x;
        if (z < N) {
            const int64_t e = energy_fixed(M, tiles, elow, (uint64_t)z);
            if constexpr (sizeof(R) == 4) {
                float h_, l_;
                fixed_to_ff(e, Q, h_, l_);
                dhi[q] = h_;
                dlo[q] = l_;
            } else {
                dhi[q] = __ll2double_rn(e) * ldexp(1.0, -Q);
                dlo[q] = 0;
            }
            const C p = psi_g[z];
            sp[z] = p;
            C b;
            b.x = (R)cK.x * p.x - (R)cK.y * p.y;
            b.y = (R)cK.x * p.y + (R)cK.y * p.x;
            s1[z] = b;
            C zero;
            zero.x = 0;
            zero.y = 0;
            s2[z] = zero;
        }
    }
    R ghi, glo;
    if constexpr (sizeof(R) == 4) {
        ghi = (float)g;
        glo = (float)(g - (double)ghi);
    } else {
        ghi = g;
        glo = 0;
    }
    __syncthreads();
    C* b1 = s1;
    C* b2 = s2;
    for (int k = K - 1; k >= 0; --k) {
        const double2 ck = coef[k];
        const R sc = (k == 0) ? R(1) : R(2);
        for (int q = 0; q < PER; ++q) {
            const int z = threadIdx.x + q * blockDim.x;
            if (z < N) {
                R sx = 0, sy = 0;
                for (int j = 0; j < n; ++j) {
                    const C p = b1[z ^ (1 << j)];
                    sx += p.x;
                    sy += p.y;
                }
                const C v = b1[z];
                R hx, hy;
                if constexpr (sizeof(R) == 4) {
                    hx = fmaf(dhi[q], v.x, dlo[q] * v.x) + fmaf(ghi, sx, glo * sx);
                    hy = fmaf(dhi[q], v.y, dlo[q] * v.y) + fmaf(ghi, sy, glo * sy);
                } else {
                    hx = dhi[q] * v.x + ghi * sx;
                    hy = dhi[q] * v.y + ghi * sy;
                }
                const C w = b2[z];
                const C p = sp[z];
                C o;
                o.x = sc * hx - w.x + (R)ck.x * p.x - (R)ck.y * p.y;
                o.y = sc * hy - w.y + (R)ck.x * p.y + (R)ck.y * p.x;
                if (k == 0) psi_g[z] = o;
                else b2[z] = o;
            }
        }
        __syncthreads();
        C* t = b1;
        b1 = b2;
        b2 = t;
    }
}

}  // namespace cheb
