// Whole Clenshaw runs (Algorithm 2) of mid-size instances on one thread-block
// cluster each, with psi, b_{k+1} and b_{k+2} held in the cluster's distributed
// shared memory for all K steps: one launch per group of instances instead of one
// or two launches per step.
//
// The 2^n amplitudes are split into 2^(n - SB) slices of 2^SB (SB = 13 for FP32,
// 12 for FP64: 3 x 2^SB amplitudes = 192 KB per CTA); CTA q of the cluster owns the
// slice z = q 2^SB + x. The flip partners of bits j < SB are in the CTA's own shared
// memory, those of bits j >= SB at the same offset x in CTA q xor 2^(j - SB). The
// recurrence overwrites b_{k+2} in place (Sec. II.D), and one cluster barrier per
// step orders every CTA's writes of b_k before any read of it as the next b_{k+1}
// and every read of b_{k+1} before it is overwritten. The last barrier also keeps
// each CTA's shared memory alive until no other CTA reads it.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "cheb_internal.h"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace cheb {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ int64_t sgn_sel(uint64_t bit, int64_t v) { return bit ? -v : v; }

__device__ __forceinline__ int64_t energy_of(int M, const int64_t* __restrict__ tiles,
                                             const int64_t* __restrict__ elow, uint64_t z) {
    const uint64_t T = z >> M;
    const uint64_t x = z & ((1ull << M) - 1);
    const int64_t* row = tiles + T * (M + 1);
    int64_t e = __ldg(row + M) + __ldg(elow + x);
    for (int i = 0; i < M; ++i) e += sgn_sel((x >> i) & 1, __ldg(row + i));
    return e;
}

constexpr int kClusterThreads = 1024;
constexpr int kMaxRemoteBits = 4;  // clusters of up to 16 CTAs

template <typename R, int SB>
__global__ void __launch_bounds__(kClusterThreads, 1) k_cluster_run(const SmallDesc* __restrict__ descs) {
    using C = typename Cx<R>::T;
    constexpr int kSlice = 1 << SB;
    constexpr int PER = kSlice / kClusterThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned csize = cl.num_blocks();
    const unsigned rank = cl.block_rank();
    const SmallDesc x = descs[blockIdx.x / csize];
    C* sp = (C*)smem_raw;
    C* s1 = sp + kSlice;
    C* s2 = s1 + kSlice;
    const int n = x.n;
    const int M = n < kTileBits ? n : kTileBits;
    int nrem = n - SB;
    if (nrem < 0) nrem = 0;
    if (nrem > kMaxRemoteBits) nrem = kMaxRemoteBits;  // the host never launches this
    const int64_t base = (int64_t)rank << SB;
    C* gpsi = (C*)x.psi;
    const double2 cK = ((const double2*)x.coef)[x.K];
    R dhi[PER], dlo[PER];
    const double sc = ldexp(1.0, -x.Q);
    for (int q = 0; q < PER; ++q) {
        const int xl = threadIdx.x + q * kClusterThreads;
        const int64_t e = energy_of(M, x.tiles, x.elow, (uint64_t)(base + xl));
        if constexpr (sizeof(R) == 4) {
            // float-float D = hi + lo from the two 32-bit halves of the fixed-point value
            // (|e| < 2^56, so the high half is exact in a float and lo is good to 2^-48)
            dhi[q] = (float)(int)(e >> 32) * (float)ldexp(1.0, 32 - x.Q);
            dlo[q] = (float)(uint32_t)(e & 0xffffffffll) * (float)sc;
        } else {
            dhi[q] = __ll2double_rn(e) * sc;
            dlo[q] = 0;
        }
        const C p = gpsi[base + xl];
        sp[xl] = p;
        C b;
        b.x = (R)cK.x * p.x - (R)cK.y * p.y;
        b.y = (R)cK.x * p.y + (R)cK.y * p.x;
        s1[xl] = b;
        s2[xl].x = 0;
        s2[xl].y = 0;
    }
    R ghi, glo;
    if constexpr (sizeof(R) == 4) {
        ghi = (float)x.g;
        glo = (float)(x.g - (double)ghi);
    } else {
        ghi = x.g;
        glo = 0;
    }
    C* r1[kMaxRemoteBits];
    C* r2[kMaxRemoteBits];
    for (int j = 0; j < kMaxRemoteBits; ++j) {
        const unsigned peer = j < nrem ? (rank ^ (1u << j)) : rank;
        r1[j] = cl.map_shared_rank(s1, peer);
        r2[j] = cl.map_shared_rank(s2, peer);
    }
    cl.sync();
    bool flip = false;
    for (int k = x.K - 1; k >= 0; --k) {
        C* b1 = flip ? s2 : s1;
        C* b2 = flip ? s1 : s2;
        C* const* rb = flip ? r2 : r1;
        const double2 ck = ((const double2*)x.coef)[k];
        const R scale = (k == 0) ? R(1) : R(2);
        for (int q = 0; q < PER; ++q) {
            const int xl = threadIdx.x + q * kClusterThreads;
            R sx = 0, sy = 0;
#pragma unroll
            for (int j = 0; j < SB; ++j) {
                const C p = b1[xl ^ (1 << j)];
                sx += p.x;
                sy += p.y;
            }
            for (int j = 0; j < nrem; ++j) {
                const C p = rb[j][xl];
                sx += p.x;
                sy += p.y;
            }
            const C v = b1[xl];
            R hx, hy;
            if constexpr (sizeof(R) == 4) {
                hx = fmaf(dhi[q], v.x, dlo[q] * v.x) + fmaf(ghi, sx, glo * sx);
                hy = fmaf(dhi[q], v.y, dlo[q] * v.y) + fmaf(ghi, sy, glo * sy);
            } else {
                hx = dhi[q] * v.x + ghi * sx;
                hy = dhi[q] * v.y + ghi * sy;
            }
            const C w = b2[xl];
            const C p = sp[xl];
            C o;
            o.x = scale * hx - w.x + (R)ck.x * p.x - (R)ck.y * p.y;
            o.y = scale * hy - w.y + (R)ck.x * p.y + (R)ck.y * p.x;
            if (k == 0) gpsi[base + xl] = o;
            else b2[xl] = o;
        }
        cl.sync();
        flip = !flip;
    }
}

template <typename R, int SB>
cudaError_t launch_cluster_t(int n, int count, const SmallDesc* descs, cudaStream_t s) {
    auto kern = k_cluster_run<R, SB>;
    const unsigned csize = 1u << (n - SB);
    const size_t smem = 3 * ((size_t)1 << SB) * sizeof(typename Cx<R>::T);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize * (unsigned)count, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, (void*)kern, &cfg);
    if (e != cudaSuccess) return e;
    if (active < 1) return cudaErrorNotSupported;
    note_launch(kKindSmall);
    e = cudaLaunchKernelEx(&cfg, kern, descs);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

int cluster_slice_bits(int prec) { return prec == 0 ? 13 : 12; }

cudaError_t launch_cluster_batched(int prec, int n, int count, const SmallDesc* descs, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int sb = cluster_slice_bits(prec);
    if (n <= sb || n - sb > kMaxRemoteBits) return cudaErrorInvalidValue;
    return prec == 0 ? launch_cluster_t<float, 13>(n, count, descs, s) : launch_cluster_t<double, 12>(n, count, descs, s);
}

}  // namespace cheb
