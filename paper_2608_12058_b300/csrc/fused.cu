// Fused FP32 Clenshaw step for n >= 12: the matrix-free hypercube matvec of
// Sec. II.D fused with the recurrence b_k = 2 Ht b_{k+1} - b_{k+2} + c_k psi
// (Eq. recursion), split over at most two passes over memory.
//
//  * High pass (only when h > 0): bits [n-h, n). A tile is 2^h rows of 16
//    consecutive amplitudes (128 B) whose top h bits run over all values; each
//    thread loads its own rows (coalesced 128-bit loads, prefetched one tile
//    ahead), exchanges them through shared memory and forms the flip sum over
//    the h bits. It writes q = scale*g*S_high + sgn*b_{k+2} into the slot of
//    b_{k+2}.
//  * Low pass: bits [0, 12) from a 32 KB contiguous tile of b_{k+1}, with psi and
//    the slot tile beside it, all three staged in shared memory by 1-D TMA bulk
//    copies in a two-stage mbarrier pipeline; bits [12, 12 + l) from the partner
//    tiles through L2 (persistent CTAs walk the tiles in order, so partners 2^j
//    tiles away are in flight or were just used). It recomputes the Ising
//    diagonal from the fixed-point tables (float-float hi + lo, exact to ~2^-48)
//    and writes out = scale*(Dt.*b1 + g*S_low) + slot_coeff*slot + c_k*psi.
//
// Thread layout of the low pass (1024 threads, 4 amplitudes each): a thread's
// float4 p holds amplitudes {2t + 2048p, 2t + 2048p + 1}: bit 0 lies inside the
// float4, bits 1..10 are the thread index (partners read from shared memory;
// 8 consecutive threads read 8 consecutive 16-byte words, free of bank
// conflicts), bit 11 selects one of the thread's 2 float4 registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "cheb_internal.h"
#include "fused.cuh"

namespace cheb {

namespace {

constexpr int kLowBits = kTileBits;                // 12
constexpr int kLowThreads = 1024;
constexpr int kTile = 1 << kLowBits;               // amplitudes per low tile
constexpr int kTileF4 = kTile / 2;                 // float4 per tile
constexpr int kPerThread = kTileF4 / kLowThreads;  // float4 per thread (4)
constexpr uint32_t kTileBytes = kTile * 8;         // 32 KB
constexpr int kMaxL2Bits = 10;
constexpr int kPrefetchDefault = 0;                // tiles per CTA prefetched into L2 ahead (0 = off)
constexpr long long kWaitCycles = 4000000000LL;    // ~2 s at 2 GHz
static_assert(kPerThread == 2, "layout assumes 2 float4 per thread");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Fire-and-forget bulk prefetch of global memory into L2 (no shared memory used).
__device__ __forceinline__ void l2_prefetch_bulk(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void l2_prefetch_line(const void* src) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(src));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after kWaitCycles and reports it through the flags word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flags) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(flags, kFlagTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ int64_t sel(uint32_t bit, int64_t v) { return bit ? -v : v; }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

// Two complex numbers (a float4) accumulated with packed FP32x2 adds.
struct Acc {
    float2 a, b;
    __device__ __forceinline__ void zero() { a = b = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float4 v) {
        a = __fadd2_rn(a, lo2(v));
        b = __fadd2_rn(b, hi2(v));
    }
};

// o = scale*(d*v + g*s) + cs*q + ck*ps for one complex amplitude, float-float
// d = dh + dl and g = gh + gl.
__device__ __forceinline__ float2 combine(float dh, float dl, float2 v, float2 gh, float2 gl, float2 s,
                                          float2 scale, float2 cs, float2 q, float2 ckr, float2 cki_s,
                                          float2 ps) {
    float2 h = __ffma2_rn(dup(dh), v, __fmul2_rn(dup(dl), v));
    h = __fadd2_rn(h, __ffma2_rn(gh, s, __fmul2_rn(gl, s)));
    float2 o = __ffma2_rn(scale, h, __fmul2_rn(cs, q));
    o = __ffma2_rn(ckr, ps, o);
    o = __ffma2_rn(cki_s, make_float2(ps.y, ps.x), o);  // cki_s = (-cki, cki)
    return o;
}

struct LowArgs {
    const float4* b1;
    const float4* slot;
    const float4* psi;
    float4* out;
    const int64_t* tiles;  // (kLowBits + 1) int64 per tile
    const int64_t* jq;     // J symmetric n*n, h[n], c
    int* flags;
    int n;
    int l;
    int Q;
    int prefetch;          // tiles per CTA prefetched into L2 ahead of use
    int64_t ntiles;
    float ck_re, ck_im, scale, slot_coeff, ghi, glo;
};

// Per-tile energy scalars shared by the CTA: W[x] = A(T) + sum_{i=1..5} s_i f_i(T)
// for the 5 lane bits x, W[32 + y] = sum_{i=6..10} s_i f_i(T) for the 5 warp bits y,
// then f_11 + f_0 and f_11 - f_0.
constexpr int kWEntries = 66;

// Shared memory: 2 stages x {b1, psi, slot} tiles, 2 x kWEntries energy scalars,
// then 2 mbarriers.
constexpr size_t kWOff = 6 * (size_t)kTileBytes;
constexpr size_t kBarOff = kWOff + 2 * kWEntries * sizeof(int64_t);
constexpr size_t kLowSmem = kBarOff + 64;

__device__ __forceinline__ void tile_scalars(const int64_t* __restrict__ row, int t, int64_t* w) {
    if (t < 32) {
        int64_t e = __ldg(row + kLowBits);
#pragma unroll
        for (int i = 1; i <= 5; ++i) e += sel((t >> (i - 1)) & 1, __ldg(row + i));
        w[t] = e;
    } else if (t < 64) {
        int64_t e = 0;
#pragma unroll
        for (int i = 6; i <= 10; ++i) e += sel(((t - 32) >> (i - 6)) & 1, __ldg(row + i));
        w[t] = e;
    } else if (t == 64) {
        w[64] = __ldg(row + 11) + __ldg(row + 0);
    } else if (t == 65) {
        w[65] = __ldg(row + 11) - __ldg(row + 0);
    }
}

__global__ void __launch_bounds__(kLowThreads, 1) k_low(const LowArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    int64_t* wsc = (int64_t*)(smem + kWOff);
    uint64_t* bar = (uint64_t*)(smem + kBarOff);
    const int t = threadIdx.x;
    const int n = a.n;
    const bool need_slot = a.slot_coeff != 0.f;
    const uint32_t stage_bytes = (need_slot ? 3u : 2u) * kTileBytes;

    // Thread constants of the energy split: K[p][w] collects every term of E that
    // involves only bits 0..11 of z (bits 1..10 = thread index, bit 0 = w, bit 11 = p).
    int64_t K00, K01, K10, K11;
    {
        const int64_t* J = a.jq;
        const int64_t* hq = a.jq + (size_t)n * n;
        int64_t e_tau = 0, phi0 = hq[0], phi11 = hq[11];
        for (int i = 1; i <= 10; ++i) {
            const uint32_t bi = (t >> (i - 1)) & 1;
            int64_t hi = hq[i];
            for (int j = i + 1; j <= 10; ++j) hi += sel((t >> (j - 1)) & 1, J[i * n + j]);
            e_tau += sel(bi, hi);
            phi0 += sel(bi, J[0 * n + i]);
            phi11 += sel(bi, J[11 * n + i]);
        }
        const int64_t j0b = J[0 * n + 11];
        K00 = e_tau + phi0 + phi11 + j0b;
        K01 = e_tau - phi0 + phi11 - j0b;
        K10 = e_tau + phi0 - phi11 - j0b;
        K11 = e_tau - phi0 - phi11 + j0b;
    }
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    int64_t T = blockIdx.x;
    if (T < a.ntiles) tile_scalars(a.tiles + T * (kLowBits + 1), t, wsc);
    __syncthreads();

    auto issue = [&](int stage, int64_t Tt) {
        float4* dst = (float4*)(smem + (size_t)stage * 3 * kTileBytes);
        mbar_expect_tx(&bar[stage], stage_bytes);
        tma_load_1d(dst, a.b1 + Tt * kTileF4, kTileBytes, &bar[stage]);
        tma_load_1d(dst + kTileF4, a.psi + Tt * kTileF4, kTileBytes, &bar[stage]);
        if (need_slot) tma_load_1d(dst + 2 * kTileF4, a.slot + Tt * kTileF4, kTileBytes, &bar[stage]);
    };

    const float2 ckr = dup(a.ck_re), cki_s = make_float2(-a.ck_im, a.ck_im);
    const float2 gh = dup(a.ghi), gl = dup(a.glo), sc = dup(a.scale), cs = dup(a.slot_coeff);
    const int scale_hi = (127 + 32 - a.Q) << 23, scale_lo = (127 - a.Q) << 23;
    if (t == 0 && T < a.ntiles) issue(0, T);
    for (int it = 0; T < a.ntiles; ++it, T += gridDim.x) {
        const int b = it & 1;
        const float4* sb1 = (const float4*)(smem + (size_t)b * 3 * kTileBytes);
        const float4* spsi = sb1 + kTileF4;
        const float4* sslot = sb1 + 2 * kTileF4;
        const int64_t* w = wsc + b * kWEntries;
        const int64_t Tn = T + gridDim.x;
        // Tiles several iterations ahead go to L2 now, so that the stage loads issued
        // one iteration ahead find them there: DRAM stays busy with far more bytes in
        // flight than the two shared-memory stages could hold.
        const int64_t Tp = T + (int64_t)a.prefetch * gridDim.x;
        if (a.prefetch > 0 && t == 32 && Tp < a.ntiles) {
            l2_prefetch_bulk(a.b1 + Tp * kTileF4, kTileBytes);
            l2_prefetch_bulk(a.psi + Tp * kTileF4, kTileBytes);
            if (need_slot) l2_prefetch_bulk(a.slot + Tp * kTileF4, kTileBytes);
        }
        if (Tn < a.ntiles) {
            if (t == 0) {
                fence_proxy_async();
                issue(b ^ 1, Tn);
            }
            tile_scalars(a.tiles + Tn * (kLowBits + 1), t, wsc + (b ^ 1) * kWEntries);
        }
        // flips of bits 12 .. 12+l-1 from the partner tiles through L2
        float2 S0a = make_float2(0.f, 0.f), S0b = S0a, S1a = S0a, S1b = S0a;
        int j = 0;
        for (; j + 1 < a.l; j += 2) {
            const float4* q0 = a.b1 + (T ^ ((int64_t)1 << j)) * kTileF4 + t;
            const float4* q1 = a.b1 + (T ^ ((int64_t)1 << (j + 1))) * kTileF4 + t;
            const float4 x00 = __ldg(q0), x01 = __ldg(q0 + kLowThreads);
            const float4 x10 = __ldg(q1), x11 = __ldg(q1 + kLowThreads);
            S0a = __fadd2_rn(S0a, __fadd2_rn(lo2(x00), lo2(x10)));
            S0b = __fadd2_rn(S0b, __fadd2_rn(hi2(x00), hi2(x10)));
            S1a = __fadd2_rn(S1a, __fadd2_rn(lo2(x01), lo2(x11)));
            S1b = __fadd2_rn(S1b, __fadd2_rn(hi2(x01), hi2(x11)));
        }
        if (j < a.l) {
            const float4* q0 = a.b1 + (T ^ ((int64_t)1 << j)) * kTileF4 + t;
            const float4 x00 = __ldg(q0), x01 = __ldg(q0 + kLowThreads);
            S0a = __fadd2_rn(S0a, lo2(x00));
            S0b = __fadd2_rn(S0b, hi2(x00));
            S1a = __fadd2_rn(S1a, lo2(x01));
            S1b = __fadd2_rn(S1b, hi2(x01));
        }
        const bool ok = mbar_wait(&bar[b], (it >> 1) & 1, a.flags);
        if (__syncthreads_or(!ok)) {
            // give up on this launch; let the copies already issued for the next tile land first
            if (Tn < a.ntiles) mbar_wait(&bar[b ^ 1], ((it + 1) >> 1) & 1, a.flags);
            break;
        }
        const float4 v0 = sb1[t], v1 = sb1[t + kLowThreads];
        // bit 0 (other half of the float4) and bit 11 (the other register)
        S0a = __fadd2_rn(S0a, __fadd2_rn(hi2(v0), lo2(v1)));
        S0b = __fadd2_rn(S0b, __fadd2_rn(lo2(v0), hi2(v1)));
        S1a = __fadd2_rn(S1a, __fadd2_rn(hi2(v1), lo2(v0)));
        S1b = __fadd2_rn(S1b, __fadd2_rn(lo2(v1), hi2(v0)));
        // bits 1..10: the partner thread's float4s in shared memory, summed in pairs
#pragma unroll
        for (int jj = 0; jj < 10; jj += 2) {
            const int pa = t ^ (1 << jj), pb = t ^ (2 << jj);
            const float4 y0 = sb1[pa], y1 = sb1[pa + kLowThreads];
            const float4 z0 = sb1[pb], z1 = sb1[pb + kLowThreads];
            S0a = __fadd2_rn(S0a, __fadd2_rn(lo2(y0), lo2(z0)));
            S0b = __fadd2_rn(S0b, __fadd2_rn(hi2(y0), hi2(z0)));
            S1a = __fadd2_rn(S1a, __fadd2_rn(lo2(y1), lo2(z1)));
            S1b = __fadd2_rn(S1b, __fadd2_rn(hi2(y1), hi2(z1)));
        }
        // energies: e(p, w) = W[t & 31] + W[32 + (t >> 5)] +- (f11 +- f0) + K[p][w]
        const int64_t base = w[t & 31] + w[32 + (t >> 5)];
        const int64_t up = w[64], um = w[65];
        const int64_t e00 = base + up + K00, e01 = base + um + K01;
        const int64_t e10 = base - um + K10, e11 = base - up + K11;
        const float4 ps0 = spsi[t], ps1 = spsi[t + kLowThreads];
        const float4 q0 = need_slot ? sslot[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = need_slot ? sslot[t + kLowThreads] : make_float4(0.f, 0.f, 0.f, 0.f);
        auto dd = [&](int64_t e, float& hi, float& lo) {
            hi = __int2float_rn((int)(e >> 32)) * __int_as_float(scale_hi);
            lo = __uint2float_rn((unsigned)(e & 0xffffffffll)) * __int_as_float(scale_lo);
        };
        float dh, dl;
        dd(e00, dh, dl);
        const float2 o00 = combine(dh, dl, lo2(v0), gh, gl, S0a, sc, cs, lo2(q0), ckr, cki_s, lo2(ps0));
        dd(e01, dh, dl);
        const float2 o01 = combine(dh, dl, hi2(v0), gh, gl, S0b, sc, cs, hi2(q0), ckr, cki_s, hi2(ps0));
        dd(e10, dh, dl);
        const float2 o10 = combine(dh, dl, lo2(v1), gh, gl, S1a, sc, cs, lo2(q1), ckr, cki_s, lo2(ps1));
        dd(e11, dh, dl);
        const float2 o11 = combine(dh, dl, hi2(v1), gh, gl, S1b, sc, cs, hi2(q1), ckr, cki_s, hi2(ps1));
        a.out[T * kTileF4 + t] = make_float4(o00.x, o00.y, o01.x, o01.y);
        a.out[T * kTileF4 + t + kLowThreads] = make_float4(o10.x, o10.y, o11.x, o11.y);
        __syncthreads();  // everyone is done with this stage before it is refilled
    }
}

// ---------------------------------------------------------------------------
// High pass over the top H bits. Rows of 16 amplitudes (8 float4); row index
// rho in [0, 2^H) selects the top bits. Thread t: u = t & 7 (float4 within the
// row), rho low bits = t >> 3 (up to 7 bits), rho high bits = register index p.
template <int H>
struct HighCfg {
    static constexpr int kRowBitsT = H < 7 ? H : 7;          // row bits in the thread index
    static constexpr int kThreads = 8 << kRowBitsT;          // 64 .. 1024
    static constexpr int kP = 1 << (H - kRowBitsT);          // float4 registers per thread
    static constexpr int kRows = 1 << H;
};

struct HighArgs {
    const float4* b1;
    float4* slot;       // in: b_{k+2} (if sgn != 0); out: q
    int n;
    int prefetch;       // tiles per CTA prefetched into L2 ahead of use
    int64_t ntiles;     // 2^(n - H - 4)
    float scale_g;      // scale * (gamma / r), float-float hi part
    float scale_glo;    // lo part
    float sgn;
};

template <int H>
__global__ void __launch_bounds__(HighCfg<H>::kThreads, 1) k_high(const HighArgs a) {
    using Cfg = HighCfg<H>;
    extern __shared__ __align__(16) float4 tile[];  // kRows * 8 float4
    const int t = threadIdx.x;
    const int u = t & 7;
    const int rlo = t >> 3;
    const int64_t row_stride_f4 = (int64_t)1 << (a.n - H - 1);  // 2^(n-H) amplitudes
    const bool need_slot = a.sgn != 0.f;
    const float2 g_hi = dup(a.scale_g), g_lo = dup(a.scale_glo), sg = dup(a.sgn);
    float4 nxt[Cfg::kP];
    int64_t T = blockIdx.x;
    if (T < a.ntiles) {
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            const int rho = rlo | (p << Cfg::kRowBitsT);
            nxt[p] = __ldg(a.b1 + T * 8 + rho * row_stride_f4 + u);
        }
    }
    for (; T < a.ntiles; T += gridDim.x) {
        float4 w[Cfg::kP];
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            const int rho = rlo | (p << Cfg::kRowBitsT);
            tile[rho * 8 + u] = nxt[p];
            if (need_slot) w[p] = a.slot[T * 8 + rho * row_stride_f4 + u];
        }
        const int64_t Tn = T + gridDim.x;
        if (Tn < a.ntiles) {
#pragma unroll
            for (int p = 0; p < Cfg::kP; ++p) {
                const int rho = rlo | (p << Cfg::kRowBitsT);
                nxt[p] = __ldg(a.b1 + Tn * 8 + rho * row_stride_f4 + u);
            }
        }
        // rows of tiles further ahead go to L2 (one 128-byte line per row)
        const int64_t Tp = T + (int64_t)a.prefetch * gridDim.x;
        if (a.prefetch > 0 && u == 0 && Tp < a.ntiles) {
#pragma unroll
            for (int p = 0; p < Cfg::kP; ++p) {
                const int rho = rlo | (p << Cfg::kRowBitsT);
                l2_prefetch_line(a.b1 + Tp * 8 + rho * row_stride_f4);
                if (need_slot) l2_prefetch_line(a.slot + Tp * 8 + rho * row_stride_f4);
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            Acc S;
            S.zero();
#pragma unroll
            for (int b = 1; b < Cfg::kP; b <<= 1) {
                const int rho = rlo | ((p ^ b) << Cfg::kRowBitsT);
                S.add(tile[rho * 8 + u]);
            }
#pragma unroll
            for (int j = 0; j < Cfg::kRowBitsT; ++j) {
                const int rho = (rlo ^ (1 << j)) | (p << Cfg::kRowBitsT);
                S.add(tile[rho * 8 + u]);
            }
            const int rho = rlo | (p << Cfg::kRowBitsT);
            const int64_t idx = T * 8 + rho * row_stride_f4 + u;
            float2 q0 = __ffma2_rn(g_hi, S.a, __fmul2_rn(g_lo, S.a));
            float2 q1 = __ffma2_rn(g_hi, S.b, __fmul2_rn(g_lo, S.b));
            if (need_slot) {
                q0 = __ffma2_rn(sg, lo2(w[p]), q0);
                q1 = __ffma2_rn(sg, hi2(w[p]), q1);
            }
            a.slot[idx] = make_float4(q0.x, q0.y, q1.x, q1.y);
        }
        __syncthreads();  // tile reused by the next iteration
    }
}

int g_num_sms = 0;
std::mutex g_mu;

int num_sms() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

template <int H>
cudaError_t launch_high_t(const HighArgs& a, cudaStream_t s) {
    using Cfg = HighCfg<H>;
    const size_t smem = (size_t)Cfg::kRows * 8 * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_high<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_high<H>, Cfg::kThreads, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)num_sms() * per_sm);
    if (grid < 1) grid = 1;
    note_launch(kKindHigh);
    const int pi = prof_begin(kKindHigh, s);
    k_high<H><<<(unsigned)grid, Cfg::kThreads, smem, s>>>(a);
    prof_end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_high(int H, const HighArgs& a, cudaStream_t s) {
    switch (H) {
        case 3: return launch_high_t<3>(a, s);
        case 4: return launch_high_t<4>(a, s);
        case 5: return launch_high_t<5>(a, s);
        case 6: return launch_high_t<6>(a, s);
        case 7: return launch_high_t<7>(a, s);
        case 8: return launch_high_t<8>(a, s);
        case 9: return launch_high_t<9>(a, s);
    }
    return cudaErrorInvalidValue;
}

// Two passes cover at most 12 + 10 + 9 = 31 bits; larger n runs the plain kernel.
constexpr int kFusedMaxQubits = kLowBits + kMaxL2Bits + 9;

}  // namespace

size_t fused_scratch_bytes(int, int) { return 0; }

bool fused_supported(int n, int prec) { return prec == 0 && n >= kLowBits && n <= kFusedMaxQubits; }

// Caller-chosen splits (cheb_set_fused_split), per n; l < 0 means "default".
static int g_split_l[kMaxQubits + 1];
static int g_split_h[kMaxQubits + 1];
static bool g_split_init = false;

static void split_table_init() {
    if (!g_split_init) {
        for (int i = 0; i <= kMaxQubits; ++i) g_split_l[i] = g_split_h[i] = -1;
        g_split_init = true;
    }
}

bool fused_split_valid(int n, int l, int h) {
    return n >= kLowBits && n <= kFusedMaxQubits && l >= 0 && l <= kMaxL2Bits &&
           (h == 0 || (h >= 3 && h <= 9)) && kLowBits + l + h == n;
}

bool fused_set_split(int n, int l, int h) {
    std::lock_guard<std::mutex> lk(g_mu);
    split_table_init();
    if (n < kLowBits || n > kFusedMaxQubits) return false;
    if (l < 0) {
        g_split_l[n] = g_split_h[n] = -1;
        return true;
    }
    if (!fused_split_valid(n, l, h)) return false;
    g_split_l[n] = l;
    g_split_h[n] = h;
    return true;
}

// Split of the n bits: the low pass takes 12 + l, the high pass the top h.
// Default: one pass while 12 + l covers n with l <= 9 (n <= 21); beyond that a
// high pass over as many top bits as possible (h <= 9) and at least 3 L2 bits,
// the split that timed fastest at n = 24 and n = 30 on the B300.
FusedPlan fused_plan(int n, int prec) {
    FusedPlan p;
    p.n = n;
    p.prec = prec;
    p.M = kLowBits;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        split_table_init();
        if (n >= kLowBits && n <= kMaxQubits && g_split_l[n] >= 0) {
            p.l = g_split_l[n];
            p.h = g_split_h[n];
            return p;
        }
    }
    const int rest = n - kLowBits;
    if (rest <= 9) {
        p.l = rest;
        p.h = 0;
    } else {
        p.h = std::min(9, rest - 3);
        p.l = rest - p.h;
    }
    return p;
}

// L2 prefetch distance in tiles per CTA: CHEB_L2_PREFETCH_TILES (0..16), default 0
// (off: on the B300 it did not raise either pass's bandwidth).
static int prefetch_tiles() {
    static int v = -1;
    if (v < 0) {
        int d = kPrefetchDefault;
        if (const char* e = std::getenv("CHEB_L2_PREFETCH_TILES")) {
            const int x = std::atoi(e);
            if (x >= 0 && x <= 16) d = x;
        }
        v = d;
    }
    return v;
}

cudaError_t launch_step_fused(const FusedPlan& plan, const StepArgs& s, void*, int* flags, cudaStream_t st) {
    if (plan.prec != 0 || plan.n != s.n || !fused_split_valid(s.n, plan.l, plan.h) || s.M != kLowBits)
        return cudaErrorInvalidValue;
    const float ghi = (float)s.g;
    const float glo = (float)(s.g - (double)ghi);
    float slot_coeff = (float)s.sgn;
    if (plan.h > 0) {
        HighArgs ha;
        ha.b1 = (const float4*)s.b1;
        ha.slot = (float4*)s.b2;
        ha.n = s.n;
        ha.ntiles = (int64_t)1 << (s.n - plan.h - 4);
        ha.scale_g = (float)s.scale * ghi;
        ha.scale_glo = (float)s.scale * glo;
        ha.sgn = (float)s.sgn;
        ha.prefetch = prefetch_tiles();
        cudaError_t e = launch_high(plan.h, ha, st);
        if (e != cudaSuccess) return e;
        slot_coeff = 1.0f;  // the slot now holds q
    }
    LowArgs la;
    la.b1 = (const float4*)s.b1;
    la.slot = (const float4*)s.b2;
    la.psi = (const float4*)s.psi;
    la.out = (float4*)s.out;
    la.tiles = s.tiles;
    la.jq = s.jq;
    la.flags = flags;
    la.n = s.n;
    la.l = plan.l;
    la.Q = s.Q;
    la.ntiles = (int64_t)1 << (s.n - kLowBits);
    la.ck_re = (float)s.ck_re;
    la.ck_im = (float)s.ck_im;
    la.scale = (float)s.scale;
    la.slot_coeff = slot_coeff;
    la.ghi = ghi;
    la.glo = glo;
    la.prefetch = prefetch_tiles();
    cudaError_t e = cudaFuncSetAttribute(k_low, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLowSmem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(la.ntiles, num_sms());
    note_launch(kKindLow);
    const int pi = prof_begin(kKindLow, st);
    k_low<<<(unsigned)grid, kLowThreads, kLowSmem, st>>>(la);
    prof_end(pi, st);
    return cudaGetLastError();
}

}  // namespace cheb
