// Fused Clenshaw step for complex128 states with float-float arithmetic: the
// matrix-free hypercube matvec of Sec. II.D fused with the recurrence
// b_k = 2 Ht b_{k+1} - b_{k+2} + c_k psi (Eq. recursion), for the FP64 path.
//
// On this part FP64 instructions run at a small fraction of the FP32 rate, so a
// step written in FP64 is bound by the FP64 units long before memory (the plain
// FP64 kernel reaches ~6% of HBM bandwidth). Here every value is a float-float
// pair hi + lo (|lo| <= ulp(hi)/2, ~48 significant bits) handled on the FP32 units
// with error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum and the FMA
// product error), so the step stays memory-bound:
//   * Clenshaw vectors are stored as float4 (re_hi, im_hi, re_lo, im_lo): 16 bytes
//     per amplitude, the size of a complex128. psi is converted to that form in
//     place when a run starts; the final step writes y back as complex128.
//   * The bit-flip sum over the partners of a pass accumulates the hi parts with
//     TwoSum and every rounding error and lo part in a second float (Ogita, Rump and
//     Oishi's Sum2 order), which is as accurate as summing in doubled precision.
//   * The Ising diagonal is exact: its 62-bit fixed-point value is split into three
//     21-bit words, each exact in a float, and both leading products are formed
//     exactly. gamma / r is a normalised float triple (exact to ~2^-72). Coefficients
//     c_k are float-float pairs.
// A systematic error in the operator would grow with a = t r over the run (the
// FP32 path keeps its operator constants in float-float for the same reason);
// the rounding errors of the products and sums are of the order 2^-48 per step.
//
// The kernels have the structure of the FP32 fused passes with one amplitude per
// float4 instead of two: the low pass covers bits [0, 10) from a 16 KB shared-memory
// tile (1024 amplitudes) and bits [10, 10 + l) from L2 partner tiles; strided passes
// cover ranges of 6..9 bits with rows of 8 amplitudes (128 B), or 5..8 bits with rows
// of 16 amplitudes (256 B) where rows lie megabytes apart.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "cheb_internal.h"
#include "fused.cuh"
#include "fused_ff.cuh"
#include "mbar.cuh"
#include "pair.cuh"

namespace cheb {

namespace {

constexpr int kLowBitsFF = 10;
constexpr int kTF = 1 << kLowBitsFF;        // float4 (amplitudes) per tile
constexpr uint32_t kTB = kTF * 16;          // 16 KB
constexpr int kNS = 3;                      // pipeline stages of {b1, psi, slot}
constexpr int kNP = 4;                      // partner-tile ring depth
constexpr int kCons = 512;                  // consumer threads, two amplitudes each
constexpr int kThreads = kCons + 32;        // + one producer warp
constexpr int kMaxL = 6;
constexpr int kMaxStrided = 9;
constexpr int kW = 50;
static_assert(kTF == 2 * kCons, "two amplitudes per consumer thread");

constexpr size_t kRingOff = (size_t)kNS * 3 * kTB;
constexpr size_t kWOff = kRingOff + (size_t)kNP * kTB;
constexpr size_t kBarOff = kWOff + (size_t)kNS * kW * sizeof(int64_t);
constexpr size_t kAbortOff = kBarOff + (size_t)(2 * kNS + 2 * kNP) * sizeof(uint64_t);
constexpr size_t kLowSmem = kAbortOff + 16;

// ---------------------------------------------------------------------------
// Float-float arithmetic on (re, im) pairs with packed FP32x2 instructions.
struct FF2 {
    float2 h, l;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ng(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 ad(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sb(float2 a, float2 b) { return __fadd2_rn(a, ng(b)); }
__device__ __forceinline__ float2 mu(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fm(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dp(float x) { return make_float2(x, x); }

__device__ __forceinline__ FF2 ld(float4 v) { return {f2(v.x, v.y), f2(v.z, v.w)}; }
__device__ __forceinline__ float4 pk(FF2 a) { return make_float4(a.h.x, a.h.y, a.l.x, a.l.y); }

// s + e = a + b exactly (TwoSum: no assumption on the magnitudes).
__device__ __forceinline__ void two_sum(float2 a, float2 b, float2& s, float2& e) {
    s = ad(a, b);
    const float2 bb = sb(s, a);
    e = ad(sb(a, sb(s, bb)), sb(b, bb));
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Fast2Sum).
__device__ __forceinline__ FF2 renorm(float2 a, float2 b) {
    FF2 r;
    r.h = ad(a, b);
    r.l = sb(b, sb(r.h, a));
    return r;
}

__device__ __forceinline__ FF2 ff_add(FF2 a, FF2 b) {
    float2 s, e;
    two_sum(a.h, b.h, s, e);
    return renorm(s, ad(e, ad(a.l, b.l)));
}

// (ah + al) x: the leading product exactly (FMA error), the rest below 2^-48 relative.
__device__ __forceinline__ FF2 ff_mul2(float ah, float al, FF2 x) {
    const float2 p = mu(dp(ah), x.h);
    float2 e = fm(dp(ah), x.h, ng(p));
    e = fm(dp(ah), x.l, e);
    e = fm(dp(al), x.h, e);
    return renorm(p, e);
}

// (cr + i ci) (xr + i xi) with float-float cr, ci: re = cr xr - ci xi, im = cr xi + ci xr.
__device__ __forceinline__ FF2 ff_cmul(float crh, float crl, float cih, float cil, FF2 x) {
    const FF2 xs = {f2(-x.h.y, x.h.x), f2(-x.l.y, x.l.x)};  // i x
    return ff_add(ff_mul2(crh, crl, x), ff_mul2(cih, cil, xs));
}

// The fixed-point energy e * 2^-Q (|e| < 2^62) as three exact floats.
__device__ __forceinline__ void energy_words(int64_t e, int Q, float& d2, float& d1, float& d0) {
    const int w2 = (int)(e >> 42);
    const int w1 = (int)((e >> 21) & 0x1FFFFF);
    const int w0 = (int)(e & 0x1FFFFF);
    d2 = __int2float_rn(w2) * __int_as_float((127 + 42 - Q) << 23);
    d1 = __int2float_rn(w1) * __int_as_float((127 + 21 - Q) << 23);
    d0 = __int2float_rn(w0) * __int_as_float((127 - Q) << 23);
}

// Multi-term float-float accumulator (the summation order of Ogita, Rump and Oishi's
// Sum2): the high parts of the terms go through a TwoSum chain in s, every rounding
// error and every low part is added into c, and the value s + c is renormalised once.
struct FFAcc {
    float2 s, c;
    __device__ __forceinline__ void zero() { s = c = f2(0.f, 0.f); }
    __device__ __forceinline__ void start(float2 h, float2 l) {
        s = h;
        c = l;
    }
    __device__ __forceinline__ void add(float2 h, float2 l) {
        float2 e;
        two_sum(s, h, s, e);
        c = ad(c, ad(e, l));
    }
    __device__ __forceinline__ void add(float4 v) { add(f2(v.x, v.y), f2(v.z, v.w)); }
    __device__ __forceinline__ FF2 result() const { return renorm(s, c); }
};

// Adds a * x for a float-float scalar a = ah + al and an unnormalised pair x = xh + xl:
// the leading product exactly (FMA error) into the chain, the rest as low parts.
__device__ __forceinline__ void acc_mul2(FFAcc& A, float ah, float al, float2 xh, float2 xl) {
    const float2 p = mu(dp(ah), xh);
    float2 e = fm(dp(ah), xh, ng(p));
    e = fm(dp(ah), xl, e);
    e = fm(dp(al), xh, e);
    A.add(p, e);
}

// Adds (a2 + a1 + a0) x for a normalised float triple.
__device__ __forceinline__ void acc_mul3(FFAcc& A, float a2, float a1, float a0, float2 xh, float2 xl) {
    const float2 p = mu(dp(a2), xh);
    float2 e = fm(dp(a2), xh, ng(p));
    e = fm(dp(a2), xl, e);
    e = fm(dp(a1), xh, e);
    e = fm(dp(a1), xl, e);
    e = fm(dp(a0), xh, e);
    A.add(p, e);
}

// Starts the accumulator with D x for the exact diagonal value D = d2 + d1 + d0 (three
// 21-bit words, not normalised: both upper products are taken exactly).
__device__ __forceinline__ void acc_start_energy(FFAcc& A, float d2, float d1, float d0, float2 xh, float2 xl) {
    const float2 p2 = mu(dp(d2), xh);
    float2 e = fm(dp(d2), xh, ng(p2));
    const float2 p1 = mu(dp(d1), xh);
    const float2 e1 = fm(dp(d1), xh, ng(p1));
    e = ad(e, e1);
    e = fm(dp(d0), xh, e);
    e = fm(dp(__fadd_rn(d2, d1)), xl, e);
    A.start(p2, e);
    A.add(p1, f2(0.f, 0.f));
}

__device__ __forceinline__ int64_t sel(uint32_t bit, int64_t v) { return bit ? -v : v; }

// ---------------------------------------------------------------------------
// Low pass. Consumer thread t holds amplitudes t and t + 512 of a 1024-amplitude tile:
// bits 0..8 = t (partners read from shared memory), bit 9 = which of the two. Bit 10
// is the parity of the tile index (the energy tables are built for 2048-amplitude
// tiles, so two tiles of this pass share one table row).
struct LowFFArgs {
    const float4* b1;
    const float4* slot;
    const float4* psi;
    void* out;
    const int64_t* tiles;  // 12 int64 per 2048-amplitude tile: f_0..f_10, A
    const int64_t* jq;     // J symmetric n*n, h[n], c
    int* flags;
    int n;
    int l;
    int Q;
    int out_f64;           // write complex128 (the final step) instead of float-float
    int64_t ntiles;        // 2^(n - 10)
    float scale;           // 2 for inner steps, 1 for the final step
    float slot_coeff;      // -1, 0 or +1
    float g2, g1, g0;      // gamma / r as a normalised triple
    float crh, crl, cih, cil;  // c_k as float-float
};

__global__ void __launch_bounds__(kThreads, 1) k_low_ff(const LowFFArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full_s = (uint64_t*)(smem + kBarOff);
    uint64_t* empty_s = full_s + kNS;
    uint64_t* full_p = empty_s + kNS;
    uint64_t* empty_p = full_p + kNP;
    volatile int* abort = (volatile int*)(smem + kAbortOff);
    int64_t* wall = (int64_t*)(smem + kWOff);
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const bool need_slot = a.slot_coeff != 0.f;
    const bool need_psi = a.crh != 0.f || a.cih != 0.f;

    if (t == 0) {
        for (int i = 0; i < kNS; ++i) {
            mbar_init(&full_s[i], 1);
            mbar_init(&empty_s[i], kCons / 32);
        }
        for (int i = 0; i < kNP; ++i) {
            mbar_init(&full_p[i], 1);
            mbar_init(&empty_p[i], kCons / 32);
        }
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    pdl_trigger();

    if (warp == kCons / 32) {
        // ---------------- producer warp ----------------
        pdl_wait();  // the previous step kernel's output is read from here on
        const uint32_t stage_bytes = (1u + (need_psi ? 1u : 0u) + (need_slot ? 1u : 0u)) * kTB;
        int last_s[kNS], last_p[kNP];
        for (int i = 0; i < kNS; ++i) last_s[i] = -1;
        for (int i = 0; i < kNP; ++i) last_p[i] = -1;
        int it = 0;
        long long pj = 0;
        // Per-tile energy partial sums: W[x] = A + sum_{i=0..4} s_i f_i over the lane bits
        // x, W[32 + y] = sum_{i=5..8} s_i f_i over the warp bits y, W[48/49] = s_10 f_10 +- f_9.
        // Each lane needs at most 6 table entries; they are loaded one tile ahead.
        int64_t r0[6], r1[4];
        auto load_row = [&](int64_t T10, int64_t* x0, int64_t* x1) {
            const int64_t* row = a.tiles + (T10 >> 1) * 12;
            x0[0] = __ldg(row + 11);
#pragma unroll
            for (int i = 0; i <= 4; ++i) x0[1 + i] = __ldg(row + i);
            if (lane < 16) {
#pragma unroll
                for (int i = 5; i <= 8; ++i) x1[i - 5] = __ldg(row + i);
            } else {
                x1[0] = __ldg(row + 10);
                x1[1] = __ldg(row + 9);
            }
        };
        if ((int64_t)blockIdx.x < a.ntiles) load_row(blockIdx.x, r0, r1);
        for (int64_t T = blockIdx.x; T < a.ntiles; T += gridDim.x, ++it) {
            const int s = it % kNS, k = it / kNS;
            int64_t n0[6], n1[4];
            const int64_t Tn = T + gridDim.x;
            if (Tn < a.ntiles) load_row(Tn, n0, n1);
            int ok = 1;
            if (lane == 0 && k > 0) ok = mbar_wait(&empty_s[s], (k - 1) & 1, a.flags, abort);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            int64_t* W = wall + s * kW;
            {
                int64_t e = r0[0];
#pragma unroll
                for (int i = 0; i <= 4; ++i) e += sel((lane >> i) & 1, r0[1 + i]);
                W[lane] = e;
                if (lane < 16) {
                    int64_t f = 0;
#pragma unroll
                    for (int i = 5; i <= 8; ++i) f += sel((lane >> (i - 5)) & 1, r1[i - 5]);
                    W[32 + lane] = f;
                } else if (lane == 16) {
                    W[48] = sel((uint32_t)(T & 1), r1[0]) + r1[1];
                } else if (lane == 17) {
                    W[49] = sel((uint32_t)(T & 1), r1[0]) - r1[1];
                }
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) r0[i] = n0[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) r1[i] = n1[i];
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                unsigned char* d = smem + (size_t)s * 3 * kTB;
                mbar_expect_tx(&full_s[s], stage_bytes);
                tma_load_1d(d, a.b1 + T * kTF, kTB, &full_s[s]);
                if (need_psi) tma_load_1d(d + kTB, a.psi + T * kTF, kTB, &full_s[s]);
                if (need_slot) tma_load_1d(d + 2 * kTB, a.slot + T * kTF, kTB, &full_s[s]);
                last_s[s] = k;
                for (int j = 0; j < a.l; ++j, ++pj) {
                    const int q = (int)(pj % kNP);
                    const long long kq = pj / kNP;
                    if (kq > 0 && !mbar_wait(&empty_p[q], (int)((kq - 1) & 1), a.flags, abort)) {
                        ok = 0;
                        break;
                    }
                    mbar_expect_tx(&full_p[q], kTB);
                    tma_load_1d(smem + kRingOff + (size_t)q * kTB, a.b1 + (T ^ ((int64_t)1 << j)) * kTF, kTB,
                                &full_p[q]);
                    last_p[q] = (int)(kq & 1);
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
        }
        if (lane == 0) {
            for (int i = 0; i < kNS; ++i)
                if (last_s[i] >= 0) mbar_drain(&full_s[i], last_s[i] & 1, a.flags);
            for (int i = 0; i < kNP; ++i)
                if (last_p[i] >= 0) mbar_drain(&full_p[i], last_p[i], a.flags);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    // Thread constants: every energy term that involves only bits 0..10 of z, for the
    // four combinations of bit 9 (p) and bit 10 (tile parity b).
    int64_t K00, K01, K10, K11;  // K<b><p>
    {
        const int n = a.n;
        const int64_t* J = a.jq;
        const int64_t* hq = a.jq + (size_t)n * n;
        int64_t e_tau = 0, phi9 = hq[9], phi10 = hq[10];
        for (int i = 0; i <= 8; ++i) {
            const uint32_t bi = (t >> i) & 1;
            int64_t hi = hq[i];
            for (int j = i + 1; j <= 8; ++j) hi += sel((t >> j) & 1, J[i * n + j]);
            e_tau += sel(bi, hi);
            phi9 += sel(bi, J[i * n + 9]);
            phi10 += sel(bi, J[i * n + 10]);
        }
        const int64_t j910 = J[9 * n + 10];
        K00 = e_tau + phi9 + phi10 + j910;
        K01 = e_tau - phi9 + phi10 - j910;
        K10 = e_tau + phi9 - phi10 - j910;
        K11 = e_tau - phi9 - phi10 + j910;
    }
    const bool twice = a.scale != 1.f;
    const float gs2 = twice ? 2.f * a.g2 : a.g2, gs1 = twice ? 2.f * a.g1 : a.g1, gs0 = twice ? 2.f * a.g0 : a.g0;
    int it = 0;
    long long pj = 0;
    for (int64_t T = blockIdx.x; T < a.ntiles; T += gridDim.x, ++it) {
        const int s = it % kNS;
        if (!mbar_wait(&full_s[s], (it / kNS) & 1, a.flags, abort)) break;
        const float4* sb1 = (const float4*)(smem + (size_t)s * 3 * kTB);
        const float4* spsi = sb1 + kTF;
        const float4* sslot = sb1 + 2 * kTF;
        const int64_t* W = wall + s * kW;
        FFAcc S0, S1;
        S0.zero();
        S1.zero();
        // bits 10 .. 10+l-1: partner tiles from the ring
        bool ok = true;
        for (int j = 0; j < a.l; ++j, ++pj) {
            const int q = (int)(pj % kNP);
            if (!mbar_wait(&full_p[q], (int)((pj / kNP) & 1), a.flags, abort)) {
                ok = false;
                break;
            }
            const float4* pr = (const float4*)(smem + kRingOff + (size_t)q * kTB);
            S0.add(pr[t]);
            S1.add(pr[t + kCons]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_p[q]);
        }
        if (!ok) break;
        const float4 v0 = sb1[t], v1 = sb1[t + kCons];
        // bits 0..8 (partner threads' amplitudes in shared memory), then bit 9
#pragma unroll
        for (int j = 0; j <= 8; ++j) {
            S0.add(sb1[t ^ (1 << j)]);
            S1.add(sb1[(t ^ (1 << j)) + kCons]);
        }
        S0.add(v1);
        S1.add(v0);
        const int64_t base = W[t & 31] + W[32 + (t >> 5)];
        const bool b10 = (T & 1) != 0;
        const int64_t e0 = base + W[48] + (b10 ? K10 : K00);
        const int64_t e1 = base + W[49] + (b10 ? K11 : K01);
        const float4 ps0 = need_psi ? spsi[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ps1 = need_psi ? spsi[t + kCons] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q0 = need_slot ? sslot[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = need_slot ? sslot[t + kCons] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_s[s]);  // this warp is done with the stage
        // out = scale (D b_{k+1} + g S) + slot_coeff q + c_k psi: every term goes into one
        // accumulator (scale = 2 is folded into D and g exactly), renormalised once
        auto combine = [&](int64_t e, float4 v, const FFAcc& S, float4 q, float4 ps) -> FF2 {
            float d2, d1, d0;
            energy_words(e, a.Q, d2, d1, d0);
            if (twice) {
                d2 += d2;
                d1 += d1;
                d0 += d0;
            }
            FFAcc A;
            acc_start_energy(A, d2, d1, d0, f2(v.x, v.y), f2(v.z, v.w));
            acc_mul3(A, gs2, gs1, gs0, S.s, S.c);
            if (need_slot) {
                const float2 qh = f2(q.x, q.y), ql = f2(q.z, q.w);
                if (a.slot_coeff < 0.f)
                    A.add(ng(qh), ng(ql));
                else
                    A.add(qh, ql);
            }
            if (need_psi) {
                acc_mul2(A, a.crh, a.crl, f2(ps.x, ps.y), f2(ps.z, ps.w));
                acc_mul2(A, a.cih, a.cil, f2(-ps.y, ps.x), f2(-ps.w, ps.z));  // c_im (i psi)
            }
            return A.result();
        };
        const FF2 o0 = combine(e0, v0, S0, q0, ps0);
        const FF2 o1 = combine(e1, v1, S1, q1, ps1);
        if (a.out_f64) {
            double2* out = (double2*)a.out + T * kTF;
            out[t] = make_double2((double)o0.h.x + (double)o0.l.x, (double)o0.h.y + (double)o0.l.y);
            out[t + kCons] = make_double2((double)o1.h.x + (double)o1.l.x, (double)o1.h.y + (double)o1.l.y);
        } else {
            float4* out = (float4*)a.out + T * kTF;
            out[t] = pk(o0);
            out[t + kCons] = pk(o1);
        }
    }
}

// ---------------------------------------------------------------------------
// Strided pass over amplitude bits [lo, lo + H) with rows of 2^RB amplitudes (RB = 3:
// 128 B, RB = 4: 256 B). The float4 geometry is that of the FP32 strided pass with
// rows of 2^(RB+1) FP32 amplitudes, so the tile and ring sizes come from StridedWsCfg.
struct StridedFFArgs {
    const float4* b1;
    const float4* slot_in;
    float4* slot;
    int lo;
    int64_t ntiles;  // 2^(n - H - RB)
    float g2, g1, g0;  // scale * gamma / r as a normalised triple
    float sgn;       // coefficient of the slot's old content: -1, 0 or +1
    int* flags;
};

template <int H, int RB>
struct StridedFFCfg {
    static constexpr int kRowF4 = 1 << RB;
    static constexpr uint32_t kRowBytes = 16u * kRowF4;
    static constexpr int kRB = 9 - RB;  // row bits in the thread index
    static constexpr int kRows = 1 << H;
    static constexpr int kBox = kRows < 256 ? kRows : 256;
    static constexpr uint32_t kStageBytes = (uint32_t)kRows * kRowBytes;
    static constexpr int kP = 1 << (H - kRB);
    static constexpr int kChunkRows = 1 << kRB;
    static constexpr uint32_t kChunkBytes = (uint32_t)kChunkRows * kRowBytes;  // 8 KB
    static constexpr int kSR = 8;
    static constexpr uint32_t kRingBytes = kSR * kChunkBytes;
    static constexpr int kNSraw = (int)((200u * 1024u - kRingBytes) / kStageBytes);
    static constexpr int kNS = kNSraw < 6 ? kNSraw : 6;
    static constexpr size_t kRingOffS = (size_t)kNS * kStageBytes;
    static constexpr size_t kBarOffS = kRingOffS + kRingBytes;
    static constexpr size_t kSmem = kBarOffS + (2 * kNS + 2 * kSR) * sizeof(uint64_t) + 16;
    static_assert(kRowF4 * (1 << kRB) == kCons && H >= kRB, "thread layout");
};

template <int H, int RB>
__global__ void __launch_bounds__(kThreads, 1)
    k_strided_ff(const StridedFFArgs a, const __grid_constant__ CUtensorMap map,
                 const __grid_constant__ CUtensorMap smap) {
    using Cfg = StridedFFCfg<H, RB>;
    static_assert(H <= 9 && Cfg::kNS >= 2, "strided ring");
    static_assert(Cfg::kSmem <= 227 * 1024, "shared memory");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)(smem + Cfg::kBarOffS);
    uint64_t* empty = full + Cfg::kNS;
    uint64_t* sfull = empty + Cfg::kNS;
    uint64_t* sempty = sfull + Cfg::kSR;
    volatile int* abort = (volatile int*)(sempty + Cfg::kSR);
    unsigned char* ring = smem + Cfg::kRingOffS;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t row_stride = (int64_t)1 << a.lo;
    const int sh = a.lo - RB;
    const bool need_slot = a.sgn != 0.f;
    if (t == 0) {
        for (int i = 0; i < Cfg::kNS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kCons / 32);
        }
        for (int i = 0; i < Cfg::kSR; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], kCons / 32);
        }
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    pdl_trigger();
    if (warp == kCons / 32) {
        pdl_wait();
        if (lane != 0) return;
        int last[Cfg::kNS], slast[Cfg::kSR];
        for (int i = 0; i < Cfg::kNS; ++i) last[i] = -1;
        for (int i = 0; i < Cfg::kSR; ++i) slast[i] = -1;
        bool ok = true;
        int it = 0;
        for (int64_t T = blockIdx.x; ok && T < a.ntiles; T += gridDim.x, ++it) {
            const int s = it % Cfg::kNS, k = it / Cfg::kNS;
            if (k > 0 && !mbar_wait(&empty[s], (k - 1) & 1, a.flags, abort)) break;
            mbar_expect_tx(&full[s], Cfg::kStageBytes);
            last[s] = k;
            const int tlo = (int)(T & (((int64_t)1 << sh) - 1));
            const int thi = (int)(T >> sh);
            unsigned char* dst = smem + (size_t)s * Cfg::kStageBytes;
#pragma unroll
            for (int c = 0; c < Cfg::kRows / Cfg::kBox; ++c)
                tma_load_4d(dst + (size_t)c * Cfg::kBox * Cfg::kRowBytes, &map, 0, tlo, c * Cfg::kBox, thi, &full[s]);
            if (need_slot) {
                for (int p = 0; p < Cfg::kP; ++p) {
                    const int c = it * Cfg::kP + p, r = c % Cfg::kSR, kk = c / Cfg::kSR;
                    if (kk > 0 && !mbar_wait(&sempty[r], (kk - 1) & 1, a.flags, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&sfull[r], Cfg::kChunkBytes);
                    slast[r] = kk;
                    tma_load_4d(ring + (size_t)r * Cfg::kChunkBytes, &smap, 0, tlo, p * Cfg::kChunkRows, thi,
                                &sfull[r]);
                }
            }
        }
        for (int i = 0; i < Cfg::kNS; ++i)
            if (last[i] >= 0) mbar_drain(&full[i], last[i] & 1, a.flags);
        for (int i = 0; i < Cfg::kSR; ++i)
            if (slast[i] >= 0) mbar_drain(&sfull[i], slast[i] & 1, a.flags);
        return;
    }
    const int u = t & (Cfg::kRowF4 - 1);
    const int rlo = t >> RB;  // kRB bits
    bool ok = true;
    int it = 0;
    for (int64_t T = blockIdx.x; ok && T < a.ntiles; T += gridDim.x, ++it) {
        const int s = it % Cfg::kNS;
        const int64_t tlo = T & (((int64_t)1 << sh) - 1);
        const int64_t base = tlo * Cfg::kRowF4 + ((T >> sh) << (a.lo + H));
        if (!mbar_wait(&full[s], (it / Cfg::kNS) & 1, a.flags, abort)) break;
        const float4* tile = (const float4*)(smem + (size_t)s * Cfg::kStageBytes);
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            FFAcc S;
            S.zero();
            // partners in descending bit order of the range (as in the blocked pair, so the
            // two agree bit for bit)
#pragma unroll
            for (int b = Cfg::kP >> 1; b >= 1; b >>= 1) S.add(tile[(rlo | ((p ^ b) << Cfg::kRB)) * Cfg::kRowF4 + u]);
#pragma unroll
            for (int j = Cfg::kRB - 1; j >= 0; --j) S.add(tile[((rlo ^ (1 << j)) | (p << Cfg::kRB)) * Cfg::kRowF4 + u]);
            // q = g S + sgn slot in one accumulator, renormalised once
            FFAcc A;
            A.zero();
            if (need_slot) {
                const int c = it * Cfg::kP + p, r = c % Cfg::kSR;
                if (!mbar_wait(&sfull[r], (c / Cfg::kSR) & 1, a.flags, abort)) {
                    ok = false;
                    break;
                }
                const float4 w = ((const float4*)(ring + (size_t)r * Cfg::kChunkBytes))[rlo * Cfg::kRowF4 + u];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sempty[r]);
                if (a.sgn < 0.f)
                    A.start(f2(-w.x, -w.y), f2(-w.z, -w.w));
                else
                    A.start(f2(w.x, w.y), f2(w.z, w.w));
            }
            acc_mul3(A, a.g2, a.g1, a.g0, S.s, S.c);
            a.slot[base + (rlo | (p << Cfg::kRB)) * row_stride + u] = pk(A.result());
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// Arithmetic of the blocked strided pair (pair.cuh) for float-float vectors: the flip
// sum in the Sum2 accumulator, q = (s g) S + sgn w in one accumulator, exactly as in
// k_strided_ff.
struct ArithFF {
    static constexpr int kAmpShift = 0;  // one amplitude per float4
    static constexpr int kRowBits = 3;   // 8 amplitudes per 128-byte row
    using Acc = FFAcc;
    static constexpr bool kLanes = false;  // float-float sums need whole amplitudes
    struct Scale {
        float g2, g1, g0;
    };
    __device__ static Scale scale(const pairk::Args& a) { return {a.g2, a.g1, a.g0}; }
    __device__ static float4 finish(const Acc& S, float4 w, bool need, float sgn, const Scale& c) {
        FFAcc A;
        A.zero();
        if (need) {
            if (sgn < 0.f)
                A.start(f2(-w.x, -w.y), f2(-w.z, -w.w));
            else
                A.start(f2(w.x, w.y), f2(w.z, w.w));
        }
        acc_mul3(A, c.g2, c.g1, c.g0, S.s, S.c);
        return pk(A.result());
    }
};

// ---------------------------------------------------------------------------
// Conversions at the ends of a run (once per Clenshaw run, FP64 arithmetic).
__global__ void k_to_ff(int64_t N, double2* psi) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = psi[z];
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        const float rl = __double2float_rn(v.x - (double)rh), il = __double2float_rn(v.y - (double)ih);
        ((float4*)psi)[z] = make_float4(rh, ih, rl, il);
    }
}

// dst = c * src for float-float vectors, c = (crh + crl) + i (cih + cil).
__global__ void k_ff_scale(int64_t N, const float4* src, float4* dst, float crh, float crl, float cih, float cil) {
    for (int64_t z = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; z < N; z += (int64_t)gridDim.x * blockDim.x)
        dst[z] = pk(ff_cmul(crh, crl, cih, cil, ld(src[z])));
}

unsigned grid_1d(int64_t N) {
    int64_t b = (N + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (unsigned)std::max<int64_t>(b, 1);
}

// Tensor maps of a float-float strided pass over amplitude bits [lo, lo + H) with rows of
// 2^RB amplitudes: (row of 2^(RB+2) floats) x (rows below the range) x (rows in the
// range) x (rows above); b_{k+1} in boxes of box_rows rows, the slot in 8 KB chunks.
cudaError_t ff_maps(const StridedFFArgs& a, int n, int H, int RB, int box_rows, CUtensorMap* map, CUtensorMap* smap) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint32_t rf = 1u << (RB + 2);
    cuuint64_t dims[4] = {rf, (cuuint64_t)1 << (a.lo - RB), (cuuint64_t)1 << H, (cuuint64_t)1 << (n - a.lo - H)};
    cuuint64_t strides[3] = {(cuuint64_t)4 * rf, (cuuint64_t)1 << (a.lo + 4), (cuuint64_t)1 << (a.lo + H + 4)};
    cuuint32_t box[4] = {rf, 1, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)a.b1, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    *smap = *map;
    if (a.sgn != 0.f) {
        cuuint32_t sbox[4] = {rf, 1, 1u << (9 - RB), 1};
        if (enc(smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)a.slot_in, dims, strides, sbox, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <int H, int RB>
cudaError_t launch_strided_ff_t(const StridedFFArgs& a, int n, cudaStream_t s) {
    using Cfg = StridedFFCfg<H, RB>;
    CUtensorMap map, smap;
    cudaError_t e = ff_maps(a, n, H, RB, Cfg::kBox, &map, &smap);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_strided_ff<H, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.ntiles, num_sms());
    note_launch(kKindHigh);
    const int pi = prof_begin(kKindHigh, s);
    const cudaError_t le = launch_step_kernel(k_strided_ff<H, RB>, (unsigned)grid, kThreads, Cfg::kSmem, s, a, map, smap);
    prof_end(pi, s);
    return le;
}

// Rows of 2^RB amplitudes: 256-byte rows (RB = 4) for ranges of 5..8 bits whose rows
// are at least 2 MB apart, 128-byte rows (RB = 3) for 6..9 bits otherwise.
int ff_row_bits(int lo, int H) { return (H >= 5 && H <= 8 && lo >= 17) ? 4 : 3; }

cudaError_t launch_strided_ff(int H, int RB, const StridedFFArgs& a, int n, cudaStream_t s) {
    if (RB == 4) {
        switch (H) {
            case 5: return launch_strided_ff_t<5, 4>(a, n, s);
            case 6: return launch_strided_ff_t<6, 4>(a, n, s);
            case 7: return launch_strided_ff_t<7, 4>(a, n, s);
            case 8: return launch_strided_ff_t<8, 4>(a, n, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (H) {
        case 6: return launch_strided_ff_t<6, 3>(a, n, s);
        case 7: return launch_strided_ff_t<7, 3>(a, n, s);
        case 8: return launch_strided_ff_t<8, 3>(a, n, s);
        case 9: return launch_strided_ff_t<9, 3>(a, n, s);
    }
    return cudaErrorInvalidValue;
}

// Near-equal passes of the h strided bits above lo0; each pass must be 6..9 bits, or
// 5 bits when it runs on wide rows.
bool ff_passes(int lo0, int h, FusedPlan& p) {
    p.npass = 0;
    if (h == 0) return true;
    if (h < 5) return false;
    const int np = (h + kMaxStrided - 1) / kMaxStrided;
    if (np > 4) return false;
    int lo = lo0;
    for (int k = 0; k < np; ++k) {
        const int hb = h / np + (k < h % np ? 1 : 0);
        if (hb > kMaxStrided || (hb < 6 && !(hb == 5 && ff_row_bits(lo, hb) == 4))) return false;
        p.lo[k] = lo;
        p.hb[k] = hb;
        lo += hb;
    }
    p.npass = np;
    return true;
}

std::mutex g_ff_mu;
int g_ff_l[kMaxQubits + 1], g_ff_h[kMaxQubits + 1];
bool g_ff_init = false;

void ff_table_init() {
    if (!g_ff_init) {
        for (int i = 0; i <= kMaxQubits; ++i) g_ff_l[i] = g_ff_h[i] = -1;
        g_ff_init = true;
    }
}

// float-float of a double: hi = fl(x), lo = fl(x - hi); and a normalised triple.
void split2(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}
void split3(double x, float& a2, float& a1, float& a0) {
    a2 = (float)x;
    const double r = x - (double)a2;
    a1 = (float)r;
    a0 = (float)(r - (double)a1);
}

}  // namespace

bool ff_split_valid(int n, int l, int h) {
    if (n < kFFMinQubits || n > kMaxQubits || l < 0 || l > kMaxL || h < 0 || kLowBitsFF + l + h != n) return false;
    FusedPlan p;
    return ff_passes(kLowBitsFF + l, h, p);
}

bool ff_set_split(int n, int l, int h) {
    std::lock_guard<std::mutex> lk(g_ff_mu);
    ff_table_init();
    if (n < kFFMinQubits || n > kMaxQubits) return false;
    if (l < 0) {
        g_ff_l[n] = g_ff_h[n] = -1;
        return true;
    }
    if (!ff_split_valid(n, l, h)) return false;
    g_ff_l[n] = l;
    g_ff_h[n] = h;
    return true;
}

bool ff_supported(int n) { return n >= kFFMinQubits && n <= kMaxQubits; }

// Default split: at most four L2 partner bits; the fewest strided passes of 6..9 bits,
// then the fewest partner bits; a 9-bit top pass at bit 17 or above becomes an 8-bit
// pass of wide rows by taking one more partner bit (as in the FP32 plan).
FusedPlan ff_plan(int n) {
    FusedPlan p;
    p.n = n;
    p.prec = 1;
    p.M = kLowBitsFF;
    int l = -1, h = -1;
    {
        std::lock_guard<std::mutex> lk(g_ff_mu);
        ff_table_init();
        if (n >= kFFMinQubits && n <= kMaxQubits && g_ff_l[n] >= 0) {
            l = g_ff_l[n];
            h = g_ff_h[n];
        }
    }
    if (l < 0) {
        const int rest = n - kLowBitsFF;
        if (rest <= 5) {
            l = rest;
        } else {
            const int np = (std::max(rest - 4, 0) + kMaxStrided - 1) / kMaxStrided;
            l = std::max(0, rest - kMaxStrided * np);
            if (rest - l > 0 && rest - l < 6) l = rest - 6;
        }
        h = rest - l;
        FusedPlan q;
        if (h > kMaxStrided && l < 4 && ff_passes(kLowBitsFF + l, h, q) && q.hb[q.npass - 1] == kMaxStrided &&
            q.lo[q.npass - 1] >= 17 && ff_split_valid(n, l + 1, h - 1)) {
            ++l;
            --h;
        }
    }
    p.l = l;
    p.h = h;
    ff_passes(kLowBitsFF + l, h, p);
    return p;
}

cudaError_t launch_to_ff(int64_t N, void* psi, cudaStream_t s) {
    note_launch(kKindScale);
    k_to_ff<<<grid_1d(N), 256, 0, s>>>(N, (double2*)psi);
    return cudaGetLastError();
}

cudaError_t launch_ff_scale(int64_t N, const void* src, void* dst, double cr, double ci, cudaStream_t s) {
    float crh, crl, cih, cil;
    split2(cr, crh, crl);
    split2(ci, cih, cil);
    note_launch(kKindScale);
    k_ff_scale<<<grid_1d(N), 256, 0, s>>>(N, (const float4*)src, (float4*)dst, crh, crl, cih, cil);
    return cudaGetLastError();
}

bool ff_pair_eligible(const FusedPlan& plan) {
    return plan.prec == 1 && plan.n >= 22 && plan.npass == 2 && pairk::shape_ok(plan.hb[0], plan.hb[1]);
}

cudaError_t launch_step_ff(const FusedPlan& plan, const StepArgs& s, void* scratch, int* flags, bool out_f64,
                           cudaStream_t st) {
    if (plan.prec != 1 || plan.n != s.n || !ff_split_valid(s.n, plan.l, plan.h) || s.M != 11)
        return cudaErrorInvalidValue;
    float g2, g1, g0;
    split3(s.g * s.scale, g2, g1, g0);
    float slot_coeff = (float)s.sgn;
    float4* q = (s.out != s.psi && s.out != s.b1) ? (float4*)s.out : (float4*)s.b2;
    // the two strided passes of a two-pass split as one L2-blocked launch
    const bool pair = fused_blocking_for(1, s.n) == 2 && scratch != nullptr && ff_pair_eligible(plan) &&
                      s.out != s.b1;
    if (pair) {
        pairk::Args pa{};
        pa.b1 = (const float4*)s.b1;
        pa.slot_in = (const float4*)s.b2;
        pa.slot = q;
        pa.loA = plan.lo[0];
        pa.loB = plan.lo[1];
        pa.g2 = g2;
        pa.g1 = g1;
        pa.g0 = g0;
        pa.sgn = (float)s.sgn;
        pa.gbits = plan.lo[0] - ArithFF::kRowBits;
        const size_t group_bytes = (size_t)32 << (ArithFF::kRowBits + plan.hb[0] + plan.hb[1]);  // b_{k+1} and q
        pa.lag = (int)std::min<int64_t>(pair_lag(group_bytes), (int64_t)1 << pa.gbits);
        pa.work = (unsigned long long*)scratch;
        pa.done = (unsigned*)((unsigned char*)scratch + 8);
        pa.flags = flags;
        cudaError_t e = cudaMemsetAsync(scratch, 0, 8 + ((size_t)4 << pa.gbits), st);
        if (e != cudaSuccess) return e;
        e = pairk::launch<ArithFF>(plan.hb[0], plan.hb[1], pa, s.n, st);
        if (e != cudaSuccess) return e;
        slot_coeff = 1.0f;
    }
    for (int k = 0; k < (pair ? 0 : plan.npass); ++k) {
        StridedFFArgs sa;
        sa.b1 = (const float4*)s.b1;
        sa.slot_in = (k == 0) ? (const float4*)s.b2 : q;
        sa.slot = q;
        sa.lo = plan.lo[k];
        const int rb = ff_row_bits(plan.lo[k], plan.hb[k]);
        sa.ntiles = (int64_t)1 << (s.n - plan.hb[k] - rb);
        sa.g2 = g2;
        sa.g1 = g1;
        sa.g0 = g0;
        sa.sgn = (k == 0) ? (float)s.sgn : 1.0f;
        sa.flags = flags;
        cudaError_t e = launch_strided_ff(plan.hb[k], rb, sa, s.n, st);
        if (e != cudaSuccess) return e;
        slot_coeff = 1.0f;
    }
    LowFFArgs la;
    la.b1 = (const float4*)s.b1;
    la.slot = plan.npass > 0 ? q : (const float4*)s.b2;
    la.psi = (const float4*)s.psi;
    la.out = s.out;
    la.tiles = s.tiles;
    la.jq = s.jq;
    la.flags = flags;
    la.n = s.n;
    la.l = plan.l;
    la.Q = s.Q;
    la.out_f64 = out_f64 ? 1 : 0;
    la.ntiles = (int64_t)1 << (s.n - kLowBitsFF);
    la.scale = (float)s.scale;
    la.slot_coeff = slot_coeff;
    split3(s.g, la.g2, la.g1, la.g0);
    split2(s.ck_re, la.crh, la.crl);
    split2(s.ck_im, la.cih, la.cil);
    cudaError_t e = cudaFuncSetAttribute(k_low_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLowSmem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(la.ntiles, num_sms());
    note_launch(kKindLow);
    const int pi = prof_begin(kKindLow, st);
    const cudaError_t le = launch_step_kernel(k_low_ff, (unsigned)grid, kThreads, kLowSmem, st, la);
    prof_end(pi, st);
    return le;
}

}  // namespace cheb
