// Fused FP32 Clenshaw step: the matrix-free hypercube matvec of Sec. II.D fused
// with the recurrence b_k = 2 Ht b_{k+1} - b_{k+2} + c_k psi (Eq. recursion).
//
// One step needs every bit-flip partner of every amplitude. The flips are split
// over a few passes over memory:
//  * Strided passes (zero or more): bits [lo, lo + hb), hb in 3..9. A tile is
//    2^hb rows of 16 consecutive amplitudes (128 B) that differ only in those bits;
//    threads load their rows (coalesced 128-bit loads, prefetched one tile ahead),
//    exchange them through shared memory and form the flip sum over the hb bits.
//    The pass writes q = scale*g*S + sgn*slot into the slot of b_{k+2} (sgn = -1 or
//    0 on the first strided pass of a step, +1 on later ones).
//  * Low pass: bits [0, 11) from a 16 KB contiguous tile of b_{k+1}; bits [11, 11+l)
//    from the partner tiles T xor 2^j, which a producer warp fetches from L2 with TMA
//    into a 4-deep ring; psi and the slot tile travel with b_{k+1} in a 3-stage TMA
//    pipeline. The producer warp also forms the tile's energy partial sums. The 16
//    consumer warps rebuild the Ising diagonal (float-float, exact to ~2^-48) and
//    write out = scale*(Dt.*b1 + g*S) + slot_coeff*slot + c_k*psi.
//
// Consumer layout (512 threads, 4 amplitudes each): float4 p of thread t holds the
// amplitudes {2t + 1024p, 2t + 1024p + 1}: bit 0 inside the float4, bits 1..9 = t
// (partners read from shared memory; 8 consecutive threads read 8 consecutive
// 16-byte words, free of bank conflicts), bit 10 = p.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "cheb_internal.h"
#include "fused.cuh"
#include "mbar.cuh"
#include "pair.cuh"

namespace cheb {

namespace {

constexpr int kLowBits = kTileBits;                 // 11
constexpr int kTF = 1 << (kLowBits - 1);            // float4 per tile per stream (1024)
constexpr uint32_t kTB = kTF * 16;                  // 16 KB
constexpr int kNS = 3;                              // pipeline stages of {b1, psi, slot}
constexpr int kNP = 4;                              // partner-tile ring depth
constexpr int kCons = 512;                          // consumer threads
constexpr int kLowThreads = kCons + 32;             // + one producer warp
constexpr int kMaxL = 6;                            // L2 partner bits allowed in a plan
constexpr int kMaxStrided = 9;                      // bits per strided pass
constexpr int kW = 50;                              // per-tile energy scalars
static_assert(kTF == 2 * kCons, "two float4 per consumer thread");

// shared-memory map of the low pass
constexpr size_t kRingOff = (size_t)kNS * 3 * kTB;
constexpr size_t kWOff = kRingOff + (size_t)kNP * kTB;
constexpr size_t kBarOff = kWOff + (size_t)kNS * kW * sizeof(int64_t);
constexpr size_t kAbortOff = kBarOff + (size_t)(2 * kNS + 2 * kNP) * sizeof(uint64_t);
constexpr size_t kLowSmem = kAbortOff + 16;
static_assert(kLowSmem <= 227 * 1024, "k_low shared memory");

__device__ __forceinline__ int64_t sel(uint32_t bit, int64_t v) { return bit ? -v : v; }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

// Flip-sum accumulator of two complex numbers (a float4). C = false: plain packed
// FP32x2 adds. C = true: Kahan's compensated summation (a running correction holds
// the low-order part that each add rounds away and feeds it into the next term), so
// the sum of one pass's flip terms is accurate to about one rounding whatever their
// number.
template <bool C>
struct AccT;

template <>
struct AccT<false> {
    float2 a, b;
    __device__ __forceinline__ void zero() { a = b = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float4 v) {
        a = __fadd2_rn(a, lo2(v));
        b = __fadd2_rn(b, hi2(v));
    }
    __device__ __forceinline__ void add2(float4 v, float4 w) {
        a = __fadd2_rn(a, __fadd2_rn(lo2(v), lo2(w)));
        b = __fadd2_rn(b, __fadd2_rn(hi2(v), hi2(w)));
    }
    __device__ __forceinline__ float2 ra() const { return a; }
    __device__ __forceinline__ float2 rb() const { return b; }
};

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

// s + x with the correction c: y = x - c, t = s + y, c = (t - s) - y, s = t.
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 x) {
    const float2 y = __fadd2_rn(x, neg2(c));
    const float2 t = __fadd2_rn(s, y);
    c = __fadd2_rn(__fadd2_rn(t, neg2(s)), neg2(y));
    s = t;
}

template <>
struct AccT<true> {
    float2 a, b, ca, cb;
    __device__ __forceinline__ void zero() { a = b = ca = cb = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float4 v) {
        kahan2(a, ca, lo2(v));
        kahan2(b, cb, hi2(v));
    }
    __device__ __forceinline__ void add2(float4 v, float4 w) {
        add(v);
        add(w);
    }
    __device__ __forceinline__ void add_a(float2 x) { kahan2(a, ca, x); }
    __device__ __forceinline__ void add_b(float2 x) { kahan2(b, cb, x); }
    __device__ __forceinline__ float2 ra() const { return __fadd2_rn(a, neg2(ca)); }
    __device__ __forceinline__ float2 rb() const { return __fadd2_rn(b, neg2(cb)); }
};

// Flips of bit 0 (the other half of the float4) and of the register bit for the two
// float4 v0, v1 of a low-pass thread (the plain sum keeps its pairwise order).
template <bool C>
__device__ __forceinline__ void add_register_partners(AccT<C>& S0, AccT<C>& S1, float4 v0, float4 v1) {
    if constexpr (!C) {
        S0.a = __fadd2_rn(S0.a, __fadd2_rn(hi2(v0), lo2(v1)));
        S0.b = __fadd2_rn(S0.b, __fadd2_rn(lo2(v0), hi2(v1)));
        S1.a = __fadd2_rn(S1.a, __fadd2_rn(hi2(v1), lo2(v0)));
        S1.b = __fadd2_rn(S1.b, __fadd2_rn(lo2(v1), hi2(v0)));
    } else {
        S0.add_a(hi2(v0));
        S0.add_a(lo2(v1));
        S0.add_b(lo2(v0));
        S0.add_b(hi2(v1));
        S1.add_a(hi2(v1));
        S1.add_a(lo2(v0));
        S1.add_b(lo2(v1));
        S1.add_b(hi2(v0));
    }
}

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
    const int64_t* tiles;  // (kLowBits + 1) int64 per tile: f_0..f_10, A
    const int64_t* jq;     // J symmetric n*n, h[n], c
    int* flags;
    int n;
    int l;
    int Q;
    int64_t ntiles;
    float ck_re, ck_im, scale, slot_coeff, ghi, glo;
};

template <bool C>
__global__ void __launch_bounds__(kLowThreads, 1) k_low(const LowArgs a) {
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
    const bool need_psi = a.ck_re != 0.f || a.ck_im != 0.f;  // c_k = 0: the adjoint chain

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
        // Energy partial sums of a tile: W[x] = A + sum_{i=1..5} s_i f_i over the lane
        // bits x, W[32 + y] = sum_{i=6..9} s_i f_i over the warp bits y, f10 +- f0.
        // Each lane needs at most 6 table entries of a tile; they are loaded one tile
        // ahead so that the load latency never delays the copies issued below.
        int64_t r0[6], r1[4];  // this lane's entries of the current tile
        auto load_row = [&](int64_t Tt, int64_t* x0, int64_t* x1) {
            const int64_t* row = a.tiles + Tt * (kLowBits + 1);
            x0[0] = __ldg(row + kLowBits);
#pragma unroll
            for (int i = 1; i <= 5; ++i) x0[i] = __ldg(row + i);
            if (lane < 16) {
#pragma unroll
                for (int i = 6; i <= 9; ++i) x1[i - 6] = __ldg(row + i);
            } else {
                x1[0] = __ldg(row + 10);
                x1[1] = __ldg(row + 0);
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
                for (int i = 1; i <= 5; ++i) e += sel((lane >> (i - 1)) & 1, r0[i]);
                W[lane] = e;
                if (lane < 16) {
                    int64_t f = 0;
#pragma unroll
                    for (int i = 6; i <= 9; ++i) f += sel((lane >> (i - 6)) & 1, r1[i - 6]);
                    W[32 + lane] = f;
                } else if (lane == 16) {
                    W[48] = r1[0] + r1[1];
                } else if (lane == 17) {
                    W[49] = r1[0] - r1[1];
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
        // let every copy this warp issued land before the CTA can retire (bounded even
        // after an abort, so a stuck copy cannot keep the kernel alive)
        if (lane == 0) {
            for (int i = 0; i < kNS; ++i)
                if (last_s[i] >= 0) mbar_drain(&full_s[i], last_s[i] & 1, a.flags);
            for (int i = 0; i < kNP; ++i)
                if (last_p[i] >= 0) mbar_drain(&full_p[i], last_p[i], a.flags);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    // Thread constants of the energy split: every term of E that involves only bits
    // 0..10 of z (bits 1..9 = thread index, bit 0 = w, bit 10 = p).
    int64_t K00, K01, K10, K11;
    {
        const int n = a.n;
        const int64_t* J = a.jq;
        const int64_t* hq = a.jq + (size_t)n * n;
        int64_t e_tau = 0, phi0 = hq[0], phi10 = hq[10];
        for (int i = 1; i <= 9; ++i) {
            const uint32_t bi = (t >> (i - 1)) & 1;
            int64_t hi = hq[i];
            for (int j = i + 1; j <= 9; ++j) hi += sel((t >> (j - 1)) & 1, J[i * n + j]);
            e_tau += sel(bi, hi);
            phi0 += sel(bi, J[0 * n + i]);
            phi10 += sel(bi, J[10 * n + i]);
        }
        const int64_t j0b = J[0 * n + 10];
        K00 = e_tau + phi0 + phi10 + j0b;
        K01 = e_tau - phi0 + phi10 - j0b;
        K10 = e_tau + phi0 - phi10 - j0b;
        K11 = e_tau - phi0 - phi10 + j0b;
    }
    const float2 ckr = dup(a.ck_re), cki_s = make_float2(-a.ck_im, a.ck_im);
    const float2 gh = dup(a.ghi), gl = dup(a.glo), sc = dup(a.scale), cs = dup(a.slot_coeff);
    const int scale_hi = (127 + 32 - a.Q) << 23, scale_lo = (127 - a.Q) << 23;
    int it = 0;
    long long pj = 0;
    for (int64_t T = blockIdx.x; T < a.ntiles; T += gridDim.x, ++it) {
        const int s = it % kNS;
        if (!mbar_wait(&full_s[s], (it / kNS) & 1, a.flags, abort)) break;
        const float4* sb1 = (const float4*)(smem + (size_t)s * 3 * kTB);
        const float4* spsi = sb1 + kTF;
        const float4* sslot = sb1 + 2 * kTF;
        const int64_t* W = wall + s * kW;
        AccT<C> S0, S1;
        S0.zero();
        S1.zero();
        // bits 11 .. 11+l-1: partner tiles from the ring
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
        // bit 0 (other half of the float4) and bit 10 (the other register)
        add_register_partners<C>(S0, S1, v0, v1);
        // bits 1..9: the partner thread's float4s in shared memory
#pragma unroll
        for (int jj = 0; jj < 8; jj += 2) {
            const int pa = t ^ (1 << jj), pb = t ^ (2 << jj);
            S0.add2(sb1[pa], sb1[pb]);
            S1.add2(sb1[pa + kCons], sb1[pb + kCons]);
        }
        {
            const int pa = t ^ (1 << 8);
            S0.add(sb1[pa]);
            S1.add(sb1[pa + kCons]);
        }
        // energies: e(p, w) = W[t & 31] + W[32 + (t >> 5)] +- (f10 +- f0) + K[p][w]
        const int64_t base = W[t & 31] + W[32 + (t >> 5)];
        const int64_t up = W[48], um = W[49];
        const int64_t e00 = base + up + K00, e01 = base + um + K01;
        const int64_t e10 = base - um + K10, e11 = base - up + K11;
        const float4 ps0 = need_psi ? spsi[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ps1 = need_psi ? spsi[t + kCons] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q0 = need_slot ? sslot[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = need_slot ? sslot[t + kCons] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_s[s]);  // this warp is done with the stage
        auto dd = [&](int64_t e, float& hi, float& lo) {
            hi = __int2float_rn((int)(e >> 32)) * __int_as_float(scale_hi);
            lo = __uint2float_rn((unsigned)(e & 0xffffffffll)) * __int_as_float(scale_lo);
        };
        float dh, dl;
        dd(e00, dh, dl);
        const float2 o00 = combine(dh, dl, lo2(v0), gh, gl, S0.ra(), sc, cs, lo2(q0), ckr, cki_s, lo2(ps0));
        dd(e01, dh, dl);
        const float2 o01 = combine(dh, dl, hi2(v0), gh, gl, S0.rb(), sc, cs, hi2(q0), ckr, cki_s, hi2(ps0));
        dd(e10, dh, dl);
        const float2 o10 = combine(dh, dl, lo2(v1), gh, gl, S1.ra(), sc, cs, lo2(q1), ckr, cki_s, lo2(ps1));
        dd(e11, dh, dl);
        const float2 o11 = combine(dh, dl, hi2(v1), gh, gl, S1.rb(), sc, cs, hi2(q1), ckr, cki_s, hi2(ps1));
        a.out[T * kTF + t] = make_float4(o00.x, o00.y, o01.x, o01.y);
        a.out[T * kTF + t + kCons] = make_float4(o10.x, o10.y, o11.x, o11.y);
    }
}

// ---------------------------------------------------------------------------
// Strided pass over bits [lo, lo + H). Rows of 16 amplitudes (8 float4); row index
// rho in [0, 2^H) holds those bits. Thread t: u = t & 7 (float4 within the row),
// rho low bits = t >> 3 (up to 7 bits), rho high bits = register index p.
template <int H>
struct StridedCfg {
    static constexpr int kRowBitsT = H < 7 ? H : 7;          // row bits in the thread index
    static constexpr int kThreads = 8 << kRowBitsT;          // 64 .. 1024
    static constexpr int kP = 1 << (H - kRowBitsT);          // float4 registers per thread
    static constexpr int kRows = 1 << H;
};

struct StridedArgs {
    const float4* b1;
    const float4* slot_in;  // b_{k+2} or the partial q (may equal slot)
    float4* slot;           // receives q
    int lo;             // first bit of the range (>= 4)
    int64_t ntiles;     // 2^(n - H - 4)
    float scale_g;      // scale * (gamma / r), float-float hi part
    float scale_glo;    // lo part
    float sgn;          // coefficient of the slot's old content
    int* flags_ws;      // status word (bounded waits of the warp-specialised variant)
};

template <int H>
__device__ __forceinline__ int64_t strided_base(const StridedArgs& a, int64_t T) {
    const int sh = a.lo - 4;
    const int64_t tlo = T & (((int64_t)1 << sh) - 1);
    const int64_t thi = T >> sh;
    return tlo * 8 + (thi << (a.lo + H - 1));
}

template <int H, bool C>
__global__ void __launch_bounds__(StridedCfg<H>::kThreads, 1) k_strided(const StridedArgs a) {
    using Cfg = StridedCfg<H>;
    extern __shared__ __align__(16) float4 tiles2[];  // 2 x kRows * 8 float4 (double-buffered)
    const int t = threadIdx.x;
    const int u = t & 7;
    const int rlo = t >> 3;
    const int64_t row_stride_f4 = (int64_t)1 << (a.lo - 1);  // 2^lo amplitudes
    const bool need_slot = a.sgn != 0.f;
    const float2 g_hi = dup(a.scale_g), g_lo = dup(a.scale_glo), sg = dup(a.sgn);
    float4 nxt[Cfg::kP];
    int64_t T = blockIdx.x;
    pdl_trigger();
    pdl_wait();
    if (T < a.ntiles) {
        const int64_t base = strided_base<H>(a, T);
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            const int rho = rlo | (p << Cfg::kRowBitsT);
            nxt[p] = __ldg(a.b1 + base + rho * row_stride_f4 + u);
        }
    }
    for (int it = 0; T < a.ntiles; T += gridDim.x, ++it) {
        // With two buffers one barrier per tile suffices: the buffer written now was
        // last read two iterations ago, before the previous iteration's barrier.
        float4* tile = tiles2 + (it & 1) * (Cfg::kRows * 8);
        const int64_t base = strided_base<H>(a, T);
        float4 w[Cfg::kP];
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            const int rho = rlo | (p << Cfg::kRowBitsT);
            tile[rho * 8 + u] = nxt[p];
            if (need_slot) w[p] = a.slot_in[base + rho * row_stride_f4 + u];
        }
        const int64_t Tn = T + gridDim.x;
        if (Tn < a.ntiles) {
            const int64_t bn = strided_base<H>(a, Tn);
#pragma unroll
            for (int p = 0; p < Cfg::kP; ++p) {
                const int rho = rlo | (p << Cfg::kRowBitsT);
                nxt[p] = __ldg(a.b1 + bn + rho * row_stride_f4 + u);
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            AccT<C> S;
            S.zero();
            // partners in descending bit order of the range
#pragma unroll
            for (int b = Cfg::kP >> 1; b >= 1; b >>= 1) {
                const int rho = rlo | ((p ^ b) << Cfg::kRowBitsT);
                S.add(tile[rho * 8 + u]);
            }
#pragma unroll
            for (int j = Cfg::kRowBitsT - 1; j >= 0; --j) {
                const int rho = (rlo ^ (1 << j)) | (p << Cfg::kRowBitsT);
                S.add(tile[rho * 8 + u]);
            }
            const int rho = rlo | (p << Cfg::kRowBitsT);
            const int64_t idx = base + rho * row_stride_f4 + u;
            float2 q0 = __ffma2_rn(g_hi, S.ra(), __fmul2_rn(g_lo, S.ra()));
            float2 q1 = __ffma2_rn(g_hi, S.rb(), __fmul2_rn(g_lo, S.rb()));
            if (need_slot) {
                q0 = __ffma2_rn(sg, lo2(w[p]), q0);
                q1 = __ffma2_rn(sg, hi2(w[p]), q1);
            }
            a.slot[idx] = make_float4(q0.x, q0.y, q1.x, q1.y);
        }
    }
}

// Warp-specialised strided pass for 5..9 bits. The vector is viewed as a 4-D tensor
// of float32: (one row of 2^RB amplitudes: 128 B for RB = 4, 256 B for RB = 5) x
// (2^(lo-RB) rows below the range) x (2^H rows of the range) x (rows above it). A
// producer lane copies each tile's 2^H rows of b_{k+1} with one or two tensor TMA
// copies (boxes of up to 256 rows) into a ring of stages, and the slot rows in 8 KB
// chunks (2^(10-RB) rows, one chunk per row group p) into a second ring, so that the
// consumers only read shared memory. 512 consumer threads (u = float4 within the
// row, rho low bits = the rest of the thread index, rho high bits = p) form the flip
// sums from the partner rows, in descending bit order, and write q. Wide rows halve
// the rows per byte, which pays where the range sits at large strides (rows many
// MB apart); a 9-bit tile of wide rows would not fit, so RB = 5 takes H <= 8.
template <int H, int RB = 4>
struct StridedWsCfg {
    static constexpr int kRowF4 = 1 << (RB - 1);             // float4 per row
    static constexpr uint32_t kRowBytes = 16u * kRowF4;
    static constexpr int kRB = 10 - RB;                       // row bits in the thread index
    static constexpr int kRows = 1 << H;
    static constexpr int kBox = kRows < 256 ? kRows : 256;
    static constexpr uint32_t kStageBytes = (uint32_t)kRows * kRowBytes;
    static constexpr int kP = 1 << (H - kRB);                 // row groups of 2^kRB rows
    static constexpr int kChunkRows = 1 << kRB;
    static constexpr uint32_t kChunkBytes = (uint32_t)kChunkRows * kRowBytes;  // 8 KB
    static constexpr int kSR = 8;                             // slot chunk ring depth
    static constexpr uint32_t kRingBytes = kSR * kChunkBytes;
    static constexpr int kNSraw = (int)((200u * 1024u - kRingBytes) / kStageBytes);
    static constexpr int kNS = kNSraw < 6 ? kNSraw : 6;      // b_{k+1} stages
    static constexpr size_t kRingOff = (size_t)kNS * kStageBytes;
    static constexpr size_t kBarOff = kRingOff + kRingBytes;
    static constexpr size_t kSmem = kBarOff + (2 * kNS + 2 * kSR) * sizeof(uint64_t) + 16;
    static_assert(kRowF4 * (1 << kRB) == kCons && H >= kRB, "thread layout");
};

// Start of tile T (in float4) of a strided pass with rows of 2^RB amplitudes.
template <int H, int RB>
__device__ __forceinline__ int64_t strided_base_rb(const StridedArgs& a, int64_t T) {
    const int sh = a.lo - RB;
    const int64_t tlo = T & (((int64_t)1 << sh) - 1);
    const int64_t thi = T >> sh;
    return tlo * (1 << (RB - 1)) + (thi << (a.lo + H - 1));
}


template <int H, int RB, bool C>
__global__ void __launch_bounds__(kLowThreads, 1)
    k_strided_ws(const StridedArgs a, const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap smap) {
    using Cfg = StridedWsCfg<H, RB>;
    static_assert(H >= Cfg::kRB && H <= 9 && Cfg::kNS >= 2, "strided ring");
    static_assert(Cfg::kSmem <= 227 * 1024, "shared memory");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)(smem + Cfg::kBarOff);
    uint64_t* empty = full + Cfg::kNS;
    uint64_t* sfull = empty + Cfg::kNS;
    uint64_t* sempty = sfull + Cfg::kSR;
    volatile int* abort = (volatile int*)(sempty + Cfg::kSR);
    unsigned char* ring = smem + Cfg::kRingOff;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t row_stride_f4 = (int64_t)1 << (a.lo - 1);
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
            if (k > 0 && !mbar_wait(&empty[s], (k - 1) & 1, a.flags_ws, abort)) break;
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
                    if (kk > 0 && !mbar_wait(&sempty[r], (kk - 1) & 1, a.flags_ws, abort)) {
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
        // let every issued copy land before the CTA exits
        for (int i = 0; i < Cfg::kNS; ++i)
            if (last[i] >= 0) mbar_drain(&full[i], last[i] & 1, a.flags_ws);
        for (int i = 0; i < Cfg::kSR; ++i)
            if (slast[i] >= 0) mbar_drain(&sfull[i], slast[i] & 1, a.flags_ws);
        return;
    }
    const int u = t & (Cfg::kRowF4 - 1);
    const int rlo = t >> (RB - 1);  // kRB bits
    const float2 g_hi = dup(a.scale_g), g_lo = dup(a.scale_glo), sg = dup(a.sgn);
    bool ok = true;
    int it = 0;
    for (int64_t T = blockIdx.x; ok && T < a.ntiles; T += gridDim.x, ++it) {
        const int s = it % Cfg::kNS;
        const int64_t base = strided_base_rb<H, RB>(a, T);
        if (!mbar_wait(&full[s], (it / Cfg::kNS) & 1, a.flags_ws, abort)) break;
        const float4* tile = (const float4*)(smem + (size_t)s * Cfg::kStageBytes);
#pragma unroll
        for (int p = 0; p < Cfg::kP; ++p) {
            AccT<C> S;
            S.zero();
            // partners in descending bit order of the range (the same order for both
            // row widths, the blocked tail and the blocked pair, so all of them agree
            // bit for bit)
#pragma unroll
            for (int b = Cfg::kP >> 1; b >= 1; b >>= 1) S.add(tile[(rlo | ((p ^ b) << Cfg::kRB)) * Cfg::kRowF4 + u]);
#pragma unroll
            for (int j = Cfg::kRB - 1; j >= 0; --j) S.add(tile[((rlo ^ (1 << j)) | (p << Cfg::kRB)) * Cfg::kRowF4 + u]);
            float2 q0 = __ffma2_rn(g_hi, S.ra(), __fmul2_rn(g_lo, S.ra()));
            float2 q1 = __ffma2_rn(g_hi, S.rb(), __fmul2_rn(g_lo, S.rb()));
            if (need_slot) {
                const int c = it * Cfg::kP + p, r = c % Cfg::kSR;
                if (!mbar_wait(&sfull[r], (c / Cfg::kSR) & 1, a.flags_ws, abort)) {
                    ok = false;
                    break;
                }
                const float4 w = ((const float4*)(ring + (size_t)r * Cfg::kChunkBytes))[rlo * Cfg::kRowF4 + u];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sempty[r]);  // this warp's reads of the chunk are done
                q0 = __ffma2_rn(sg, lo2(w), q0);
                q1 = __ffma2_rn(sg, hi2(w), q1);
            }
            a.slot[base + (rlo | (p << Cfg::kRB)) * row_stride_f4 + u] = make_float4(q0.x, q0.y, q1.x, q1.y);
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp's shared-memory reads are done
    }
}

// ---------------------------------------------------------------------------
// L2-blocked tail of a step: the last strided pass (bits [lo, n), lo + H = n) and the
// low pass in one persistent launch. Amplitudes are grouped by their bits [11, lo):
// group g holds 2^(n - lo + 11) amplitudes, 128 strided tiles (bits 4..10 of the
// tile index free) and 2^H low tiles (bits lo..n-1 free). A low tile of group g reads
// the partial q that the strided tiles of group g wrote, and b_{k+1} of groups g and
// g ^ 1 that those strided tiles read; scheduling the strided tiles of group g + 1
// between them and the low tiles of group g keeps that data in L2, so the low tiles
// read b_{k+1} and q from L2 and their in-place write of the output replaces the
// q lines still in L2 before they go back to DRAM.
//
// Work items in order: S(0) .. S(D - 1), then S(s) followed by L(s - D) for
// s = D .. G - 1, then L(G - D) .. L(G - 1), where S(g) are the 128 strided tiles and
// L(g) the 2^H low tiles of group g, and the lag D (host-chosen) puts several items
// per SM between the strided tiles of a group and its low tiles. CTAs take items
// from a global counter, so an item only ever waits for items taken before it:
// before loading a low tile the producer waits until all 128 strided tiles of its
// group are published (a notifier warp per CTA fences each finished tile's q stores
// and then raises the group's count). Every wait is bounded (status flag, abort,
// clean exit).
//
// Measured on B300: DRAM traffic of the tail drops from 56 to ~32.5 B per amplitude
// (n = 26), but the combined kernel is limited by shared-memory traffic and latency
// (a 9-bit strided tile moves ~783 KB through shared memory, a low tile ~277 KB), so
// the step is within a few percent of the separate launches (faster at n = 28,
// slower at n = 26 and 30); it is off by default.
template <int H>
struct MixedCfg {
    static constexpr int kRows = 1 << H;
    static constexpr int kBox = kRows < 256 ? kRows : 256;
    static constexpr uint32_t kS = (uint32_t)kRows * 128;    // b_{k+1} of a strided tile
    static constexpr int kP = 1 << (H - 6);                   // q chunks of 64 rows
    static constexpr uint32_t kChunk = 64 * 128;
    // a whole strided tile's q chunks fit the ring (a ring of 4 stalls 9-bit tiles
    // mid-tile for one DRAM round trip); the rest of shared memory holds the stages
    static constexpr int kSR = kP > 4 ? 8 : 4;
    static constexpr uint32_t kStage = 4 * kTB;              // {b1, psi, q, partner} of a low tile
    static constexpr int kNS = kSR == 8 ? 2 : 3;
    static constexpr int kNR = 8;                             // completion records in flight
    static constexpr size_t kRingOff = (size_t)kNS * kStage;
    static constexpr size_t kWOff = kRingOff + (size_t)kSR * kChunk;
    static constexpr size_t kItemOff = kWOff + (size_t)kNS * kW * sizeof(int64_t);
    static constexpr size_t kNoteOff = kItemOff + 32;
    static constexpr size_t kBarOff = kNoteOff + (size_t)kNR * sizeof(int64_t);
    static constexpr size_t kAbortOff = kBarOff + (size_t)(2 * kNS + 2 * kSR + 2 * kNR) * sizeof(uint64_t);
    static constexpr size_t kSmem = kAbortOff + 16;
    static_assert(kS <= kStage && kNS * sizeof(int64_t) <= 32, "stage map");
};

// Consumer warps, the producer warp and a notifier warp that publishes finished
// strided tiles (fence + count) so that the consumers never wait on a memory fence.
constexpr int kMixedThreads = kCons + 64;

struct MixedArgs {
    StridedArgs sa;               // last strided pass: slot_in = slot = q, sgn = 1
    LowArgs la;                   // low pass: slot = q, slot_coeff = 1, l = 0 or 1
    unsigned long long* work;     // item counter (zero at launch)
    unsigned* done;               // per group: strided tiles done (zero at launch)
    int gbits;                    // lo - 11 (2^gbits groups)
    int lag;                      // D, 1 <= D <= 2^gbits
};

constexpr int kItemStrided = 0, kItemLow = 1, kItemEnd = 2;

struct MixedItem {
    int kind;
    int64_t g;    // group
    int64_t idx;  // strided tile within the group (0..127) or low tile (0..2^H - 1)
};

__device__ __forceinline__ MixedItem mixed_decode(unsigned long long i, int gbits, int H, int lag) {
    const unsigned long long G = 1ull << gbits, D = (unsigned long long)lag, NS = 128, NL = 1ull << H;
    const unsigned long long seg = NS + NL, head = D * NS;
    if (i < head) return {kItemStrided, (int64_t)(i / NS), (int64_t)(i % NS)};
    const unsigned long long j = i - head, s = D + j / seg;
    if (s < G) {
        const unsigned long long r = j % seg;
        return r < NS ? MixedItem{kItemStrided, (int64_t)s, (int64_t)r}
                      : MixedItem{kItemLow, (int64_t)(s - D), (int64_t)(r - NS)};
    }
    const unsigned long long k = j - (G - D) * seg, g = G - D + k / NL;
    if (g < G) return {kItemLow, (int64_t)g, (int64_t)(k % NL)};
    return {kItemEnd, 0, 0};
}

template <int H, bool C>
__global__ void __launch_bounds__(kMixedThreads, 1)
    k_mixed(const MixedArgs m, const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap smap) {
    using Cfg = MixedCfg<H>;
    static_assert(H >= 6 && H <= 9, "strided range");
    static_assert(Cfg::kSmem <= 227 * 1024, "shared memory");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)(smem + Cfg::kBarOff);
    uint64_t* empty = full + Cfg::kNS;
    uint64_t* sfull = empty + Cfg::kNS;
    uint64_t* sempty = sfull + Cfg::kSR;
    uint64_t* cdone = sempty + Cfg::kSR;   // a strided tile's q stores are issued (16 warps)
    uint64_t* cempty = cdone + Cfg::kNR;   // the notifier has published that record
    volatile int* abort = (volatile int*)(smem + Cfg::kAbortOff);
    int64_t* wall = (int64_t*)(smem + Cfg::kWOff);
    long long* item = (long long*)(smem + Cfg::kItemOff);
    volatile long long* note = (volatile long long*)(smem + Cfg::kNoteOff);
    unsigned char* ring = smem + Cfg::kRingOff;
    const StridedArgs& a = m.sa;
    const LowArgs& la = m.la;
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const bool need_psi = la.ck_re != 0.f || la.ck_im != 0.f;
    if (t == 0) {
        for (int i = 0; i < Cfg::kNS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kCons / 32);
        }
        for (int i = 0; i < Cfg::kSR; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], kCons / 32);
        }
        for (int i = 0; i < Cfg::kNR; ++i) {
            mbar_init(&cdone[i], kCons / 32);
            mbar_init(&cempty[i], 1);
        }
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kCons / 32 + 1) {
        // ---------------- notifier warp ----------------
        // Record j: the consumers' q stores of this CTA's j-th strided tile (or the end
        // marker, group < 0). The mbarrier wait observes every consumer warp's stores;
        // the GPU-scope fence then publishes them before the group count is raised.
        if (lane != 0) return;
        for (long long j = 0;; ++j) {
            const int r = (int)(j % Cfg::kNR);
            if (!mbar_wait(&cdone[r], (uint32_t)((j / Cfg::kNR) & 1), a.flags_ws, abort)) break;
            const long long g = note[r];
            if (g < 0) break;
            __threadfence();
            atomicAdd(m.done + g, 1u);
            mbar_arrive(&cempty[r]);
        }
        return;
    }

    if (warp == kCons / 32) {
        // ---------------- producer warp ----------------
        int last[Cfg::kNS], slast[Cfg::kSR];
        for (int i = 0; i < Cfg::kNS; ++i) last[i] = -1;
        for (int i = 0; i < Cfg::kSR; ++i) slast[i] = -1;
        long long cc = 0;  // q chunks issued
        auto grab = [&]() -> unsigned long long {
            unsigned long long v = 0;
            if (lane == 0) v = atomicAdd(m.work, 1ull);
            return __shfl_sync(0xffffffffu, v, 0);
        };
        // this lane's tile-table entries (as in k_low), loaded one item ahead
        auto load_row = [&](int64_t Tt, int64_t* x0, int64_t* x1) {
            const int64_t* row = la.tiles + Tt * (kLowBits + 1);
            x0[0] = __ldg(row + kLowBits);
#pragma unroll
            for (int i = 1; i <= 5; ++i) x0[i] = __ldg(row + i);
            if (lane < 16) {
#pragma unroll
                for (int i = 6; i <= 9; ++i) x1[i - 6] = __ldg(row + i);
            } else {
                x1[0] = __ldg(row + 10);
                x1[1] = __ldg(row + 0);
            }
        };
        int64_t r0[6], r1[4];
        // the strided tiles' b_{k+1} and q are read again by the low tiles of their group
        const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
        unsigned long long nxt = grab();
        MixedItem ni = mixed_decode(nxt, m.gbits, H, m.lag);
        if (ni.kind == kItemLow) load_row(ni.g + (ni.idx << m.gbits), r0, r1);
        for (int it = 0;; ++it) {
            const unsigned long long cur = nxt;
            const MixedItem ci = ni;
            int64_t c0[6], c1[4];
#pragma unroll
            for (int i = 0; i < 6; ++i) c0[i] = r0[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) c1[i] = r1[i];
            if (ci.kind != kItemEnd) {
                nxt = grab();
                ni = mixed_decode(nxt, m.gbits, H, m.lag);
                if (ni.kind == kItemLow) load_row(ni.g + (ni.idx << m.gbits), r0, r1);
            }
            const int s = it % Cfg::kNS, k = it / Cfg::kNS;
            int ok = 1;
            if (lane == 0 && k > 0) ok = mbar_wait(&empty[s], (k - 1) & 1, a.flags_ws, abort);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (ci.kind == kItemEnd) {
                if (lane == 0) {
                    item[s] = -1;
                    mbar_arrive(&full[s]);
                    last[s] = k;
                }
                break;
            }
            if (ci.kind == kItemLow) {
                int64_t* W = wall + s * kW;
                int64_t e = c0[0];
#pragma unroll
                for (int i = 1; i <= 5; ++i) e += sel((lane >> (i - 1)) & 1, c0[i]);
                W[lane] = e;
                if (lane < 16) {
                    int64_t f = 0;
#pragma unroll
                    for (int i = 6; i <= 9; ++i) f += sel((lane >> (i - 6)) & 1, c1[i - 6]);
                    W[32 + lane] = f;
                } else if (lane == 16) {
                    W[48] = c1[0] + c1[1];
                } else if (lane == 17) {
                    W[49] = c1[0] - c1[1];
                }
                __syncwarp();
                if (lane == 0) {
                    ok = wait_count(m.done + ci.g, 128u, a.flags_ws, abort);
                    if (ok) {
                        // q was written through the generic proxy by other SMs; order
                        // those writes before this thread's bulk copies read it
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                        __threadfence_block();
                        const int64_t T = ci.g + (ci.idx << m.gbits);
                        item[s] = (long long)cur;
                        unsigned char* d = smem + (size_t)s * Cfg::kStage;
                        const uint32_t bytes = (2u + (need_psi ? 1u : 0u) + (uint32_t)la.l) * kTB;
                        mbar_expect_tx(&full[s], bytes);
                        // psi and q are not read again in this step: evict them first
                        tma_load_1d(d, la.b1 + T * kTF, kTB, &full[s]);
                        if (need_psi) tma_load_1d_hint(d + kTB, la.psi + T * kTF, kTB, &full[s], pol_first);
                        tma_load_1d_hint(d + 2 * kTB, la.slot + T * kTF, kTB, &full[s], pol_first);
                        if (la.l) tma_load_1d(d + 3 * kTB, la.b1 + (T ^ 1) * kTF, kTB, &full[s]);
                        last[s] = k;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            } else {
                if (lane == 0) {
                    const int T = (int)((ci.g << 7) | ci.idx);  // tile index below the range
                    item[s] = (long long)cur;
                    unsigned char* d = smem + (size_t)s * Cfg::kStage;
                    mbar_expect_tx(&full[s], Cfg::kS);
#pragma unroll
                    for (int c = 0; c < Cfg::kRows / Cfg::kBox; ++c)
                        tma_load_4d_hint(d + (size_t)c * Cfg::kBox * 128, &map, 0, T, c * Cfg::kBox, 0, &full[s],
                                         pol_last);
                    last[s] = k;
                    for (int p = 0; p < Cfg::kP; ++p, ++cc) {
                        const int r = (int)(cc % Cfg::kSR);
                        const long long kk = cc / Cfg::kSR;
                        if (kk > 0 && !mbar_wait(&sempty[r], (int)((kk - 1) & 1), a.flags_ws, abort)) {
                            ok = 0;
                            break;
                        }
                        mbar_expect_tx(&sfull[r], Cfg::kChunk);
                        slast[r] = (int)(kk & 1);
                        tma_load_4d_hint(ring + (size_t)r * Cfg::kChunk, &smap, 0, T, p * 64, 0, &sfull[r], pol_last);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            }
        }
        if (lane == 0) {
            for (int i = 0; i < Cfg::kNS; ++i)
                if (last[i] >= 0) mbar_drain(&full[i], last[i] & 1, a.flags_ws);
            for (int i = 0; i < Cfg::kSR; ++i)
                if (slast[i] >= 0) mbar_drain(&sfull[i], slast[i], a.flags_ws);
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const int u = t & 7;
    const int rlo = t >> 3;
    const int64_t row_stride_f4 = (int64_t)1 << (a.lo - 1);
    const float2 g_hi = dup(a.scale_g), g_lo = dup(a.scale_glo);
    // low-pass thread constants (every energy term that involves only bits 0..10)
    int64_t K00, K01, K10, K11;
    {
        const int n = la.n;
        const int64_t* J = la.jq;
        const int64_t* hq = la.jq + (size_t)n * n;
        int64_t e_tau = 0, phi0 = hq[0], phi10 = hq[10];
        for (int i = 1; i <= 9; ++i) {
            const uint32_t bi = (t >> (i - 1)) & 1;
            int64_t hi = hq[i];
            for (int j = i + 1; j <= 9; ++j) hi += sel((t >> (j - 1)) & 1, J[i * n + j]);
            e_tau += sel(bi, hi);
            phi0 += sel(bi, J[0 * n + i]);
            phi10 += sel(bi, J[10 * n + i]);
        }
        const int64_t j0b = J[0 * n + 10];
        K00 = e_tau + phi0 + phi10 + j0b;
        K01 = e_tau - phi0 + phi10 - j0b;
        K10 = e_tau + phi0 - phi10 - j0b;
        K11 = e_tau - phi0 - phi10 + j0b;
    }
    const float2 ckr = dup(la.ck_re), cki_s = make_float2(-la.ck_im, la.ck_im);
    const float2 gh = dup(la.ghi), gl = dup(la.glo), sc = dup(la.scale), cs = dup(la.slot_coeff);
    const int scale_hi = (127 + 32 - la.Q) << 23, scale_lo = (127 - la.Q) << 23;
    const uint64_t pol_out = policy_evict_first();
    long long cc = 0;  // q chunks consumed
    long long sj = 0;  // completion records sent
    // Send record sj (group g, or -1 for the end) to the notifier once this warp's
    // stores are issued; records are reused after the notifier has published them.
    auto record = [&](long long g) -> bool {
        __syncwarp();
        bool ok = true;
        if (lane == 0) {
            const int r = (int)(sj % Cfg::kNR);
            if (sj >= Cfg::kNR) ok = mbar_wait(&cempty[r], (uint32_t)(((sj / Cfg::kNR) - 1) & 1), a.flags_ws, abort);
            if (ok) {
                if (warp == 0) note[r] = g;
                mbar_arrive(&cdone[r]);
            }
        }
        ++sj;
        return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    };
    for (int it = 0;; ++it) {
        const int s = it % Cfg::kNS;
        if (!mbar_wait(&full[s], (it / Cfg::kNS) & 1, a.flags_ws, abort)) break;
        const long long cur = item[s];
        if (cur < 0) {
            record(-1);
            break;
        }
        const MixedItem ci = mixed_decode((unsigned long long)cur, m.gbits, H, m.lag);
        const unsigned char* d = smem + (size_t)s * Cfg::kStage;
        if (ci.kind == kItemStrided) {
            const int64_t T = (ci.g << 7) | ci.idx;
            const int64_t base = T * 8;  // the range is the top H bits: no tile bits above it
            const float4* tile = (const float4*)d;
            bool ok = true;
#pragma unroll
            for (int p = 0; p < Cfg::kP; ++p) {
                AccT<C> S;
                S.zero();
#pragma unroll
                for (int b = Cfg::kP >> 1; b >= 1; b >>= 1) S.add(tile[((rlo | ((p ^ b) << 6))) * 8 + u]);
#pragma unroll
                for (int j = 5; j >= 0; --j) S.add(tile[((rlo ^ (1 << j)) | (p << 6)) * 8 + u]);
                float2 q0 = __ffma2_rn(g_hi, S.ra(), __fmul2_rn(g_lo, S.ra()));
                float2 q1 = __ffma2_rn(g_hi, S.rb(), __fmul2_rn(g_lo, S.rb()));
                const int r = (int)(cc % Cfg::kSR);
                if (!mbar_wait(&sfull[r], (int)((cc / Cfg::kSR) & 1), a.flags_ws, abort)) {
                    ok = false;
                    break;
                }
                ++cc;
                const float4 w = ((const float4*)(ring + (size_t)r * Cfg::kChunk))[rlo * 8 + u];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sempty[r]);
                q0 = __fadd2_rn(lo2(w), q0);
                q1 = __fadd2_rn(hi2(w), q1);
                a.slot[base + (rlo | (p << 6)) * row_stride_f4 + u] = make_float4(q0.x, q0.y, q1.x, q1.y);
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (!record(ci.g)) break;
        } else {
            const int64_t T = ci.g + (ci.idx << m.gbits);
            const float4* sb1 = (const float4*)d;
            const float4* spsi = sb1 + kTF;
            const float4* sslot = sb1 + 2 * kTF;
            const float4* spart = sb1 + 3 * kTF;
            const int64_t* W = wall + s * kW;
            AccT<C> S0, S1;
            S0.zero();
            S1.zero();
            if (la.l) {
                S0.add(spart[t]);
                S1.add(spart[t + kCons]);
            }
            const float4 v0 = sb1[t], v1 = sb1[t + kCons];
            add_register_partners<C>(S0, S1, v0, v1);
#pragma unroll
            for (int jj = 0; jj < 8; jj += 2) {
                const int pa = t ^ (1 << jj), pb = t ^ (2 << jj);
                S0.add2(sb1[pa], sb1[pb]);
                S1.add2(sb1[pa + kCons], sb1[pb + kCons]);
            }
            {
                const int pa = t ^ (1 << 8);
                S0.add(sb1[pa]);
                S1.add(sb1[pa + kCons]);
            }
            const int64_t base = W[t & 31] + W[32 + (t >> 5)];
            const int64_t up = W[48], um = W[49];
            const int64_t e00 = base + up + K00, e01 = base + um + K01;
            const int64_t e10 = base - um + K10, e11 = base - up + K11;
            const float4 ps0 = need_psi ? spsi[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 ps1 = need_psi ? spsi[t + kCons] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 q0 = sslot[t];
            const float4 q1 = sslot[t + kCons];
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            auto dd = [&](int64_t e, float& hi, float& lo) {
                hi = __int2float_rn((int)(e >> 32)) * __int_as_float(scale_hi);
                lo = __uint2float_rn((unsigned)(e & 0xffffffffll)) * __int_as_float(scale_lo);
            };
            float dh, dl;
            dd(e00, dh, dl);
            const float2 o00 = combine(dh, dl, lo2(v0), gh, gl, S0.ra(), sc, cs, lo2(q0), ckr, cki_s, lo2(ps0));
            dd(e01, dh, dl);
            const float2 o01 = combine(dh, dl, hi2(v0), gh, gl, S0.rb(), sc, cs, hi2(q0), ckr, cki_s, hi2(ps0));
            dd(e10, dh, dl);
            const float2 o10 = combine(dh, dl, lo2(v1), gh, gl, S1.ra(), sc, cs, lo2(q1), ckr, cki_s, lo2(ps1));
            dd(e11, dh, dl);
            const float2 o11 = combine(dh, dl, hi2(v1), gh, gl, S1.rb(), sc, cs, hi2(q1), ckr, cki_s, hi2(ps1));
            // the output is next step's b_{k+1}, not read again in this launch
            st_hint(la.out + T * kTF + t, make_float4(o00.x, o00.y, o01.x, o01.y), pol_out);
            st_hint(la.out + T * kTF + t + kCons, make_float4(o10.x, o10.y, o11.x, o11.y), pol_out);
        }
    }
}

// Arithmetic of the blocked strided pair (pair.cuh) for complex64 vectors: plain FP32
// flip sums, q = s g S (float-float s g) + sgn w, exactly as in k_strided_ws.
struct ArithF32 {
    static constexpr int kAmpShift = 1;  // two amplitudes per float4
    static constexpr int kRowBits = 4;   // 16 amplitudes per 128-byte row
    using Acc = AccT<false>;
    struct Scale {
        float2 ghi, glo;
    };
    __device__ static Scale scale(const pairk::Args& a) { return {dup(a.scale_g), dup(a.scale_glo)}; }
    __device__ static float4 finish(const Acc& S, float4 w, bool need, float sgn, const Scale& c) {
        float2 q0 = __ffma2_rn(c.ghi, S.ra(), __fmul2_rn(c.glo, S.ra()));
        float2 q1 = __ffma2_rn(c.ghi, S.rb(), __fmul2_rn(c.glo, S.rb()));
        if (need) {
            const float2 sg = dup(sgn);
            q0 = __ffma2_rn(sg, lo2(w), q0);
            q1 = __ffma2_rn(sg, hi2(w), q1);
        }
        return make_float4(q0.x, q0.y, q1.x, q1.y);
    }
    // the pair's one-float-per-lane tiles: S and w hold the same float of two rows
    static constexpr bool kLanes = true;
    __device__ static float2 finish2(float2 S, float2 w, bool need, float sgn, const Scale& c) {
        float2 q = __ffma2_rn(c.ghi, S, __fmul2_rn(c.glo, S));
        if (need) q = __ffma2_rn(dup(sgn), w, q);
        return q;
    }
};

}  // namespace

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

// Flip sums with Kahan compensation (cheb_set_fused_compensated); off by default.
static int g_comp = 0;

template <int H, bool C>
cudaError_t launch_strided_c(const StridedArgs& a, cudaStream_t s) {
    using Cfg = StridedCfg<H>;
    const size_t smem = 2 * (size_t)Cfg::kRows * 8 * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_strided<H, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_strided<H, C>, Cfg::kThreads, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)num_sms() * per_sm);
    if (grid < 1) grid = 1;
    note_launch(kKindHigh);
    const int pi = prof_begin(kKindHigh, s);
    const cudaError_t le = launch_step_kernel(k_strided<H, C>, (unsigned)grid, Cfg::kThreads, smem, s, a);
    prof_end(pi, s);
    return le;
}

template <int H>
cudaError_t launch_strided_t(const StridedArgs& a, cudaStream_t s) {
    return g_comp ? launch_strided_c<H, true>(a, s) : launch_strided_c<H, false>(a, s);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

namespace {

// Tensor maps of a strided pass over bits [lo, lo + H) with rows of 2^RB amplitudes:
// b_{k+1} in boxes of `box` rows of the range, the slot in 8 KB chunks of 2^(10-RB)
// rows (only encoded when sgn != 0).
cudaError_t strided_maps(const StridedArgs& a, int n, int H, int RB, int box_rows, CUtensorMap* map,
                         CUtensorMap* smap) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    // (row of 2^(RB+1) floats) x (rows below the range) x (rows in the range) x (rows above)
    const cuuint32_t rf = 1u << (RB + 1);
    cuuint64_t dims[4] = {rf, (cuuint64_t)1 << (a.lo - RB), (cuuint64_t)1 << H, (cuuint64_t)1 << (n - a.lo - H)};
    cuuint64_t strides[3] = {(cuuint64_t)4 * rf, (cuuint64_t)1 << (a.lo + 3), (cuuint64_t)1 << (a.lo + H + 3)};
    cuuint32_t box[4] = {rf, 1, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)a.b1, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    *smap = *map;
    if (a.sgn != 0.f) {
        cuuint32_t sbox[4] = {rf, 1, 1u << (10 - RB), 1};
        if (enc(smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)a.slot_in, dims, strides, sbox, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <int H, int RB, bool C>
cudaError_t launch_strided_ws_c(const StridedArgs& a, int n, cudaStream_t s) {
    using Cfg = StridedWsCfg<H, RB>;
    CUtensorMap map, smap;
    cudaError_t e = strided_maps(a, n, H, RB, Cfg::kBox, &map, &smap);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_strided_ws<H, RB, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(a.ntiles, num_sms());
    note_launch(kKindHigh);
    const int pi = prof_begin(kKindHigh, s);
    const cudaError_t le =
        launch_step_kernel(k_strided_ws<H, RB, C>, (unsigned)grid, kLowThreads, Cfg::kSmem, s, a, map, smap);
    prof_end(pi, s);
    return le;
}

template <int H, int RB>
cudaError_t launch_strided_ws_t(const StridedArgs& a, int n, cudaStream_t s) {
    return g_comp ? launch_strided_ws_c<H, RB, true>(a, n, s) : launch_strided_ws_c<H, RB, false>(a, n, s);
}

// Rows of 2^RB amplitudes for a strided pass over [lo, lo + H): wide rows (RB = 5)
// for ranges of 6..8 bits whose rows are at least 2 MB apart (lo >= 18), where the
// 128-byte rows of RB = 4 measured ~19% slower per byte than at small strides.
int strided_row_bits(int lo, int H) { return (H >= 6 && H <= 8 && lo >= 18) ? 5 : 4; }

// Passes of 6..9 bits use the warp-specialised TMA kernel, narrower ones the
// register-prefetch kernel. a.ntiles must be 2^(n - H - RB).
cudaError_t launch_strided(int H, int RB, const StridedArgs& a, int n, cudaStream_t s) {
    if (RB == 5) {
        switch (H) {
            case 6: return launch_strided_ws_t<6, 5>(a, n, s);
            case 7: return launch_strided_ws_t<7, 5>(a, n, s);
            case 8: return launch_strided_ws_t<8, 5>(a, n, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (H) {
        case 3: return launch_strided_t<3>(a, s);
        case 4: return launch_strided_t<4>(a, s);
        case 5: return launch_strided_t<5>(a, s);
        case 6: return launch_strided_ws_t<6, 4>(a, n, s);
        case 7: return launch_strided_ws_t<7, 4>(a, n, s);
        case 8: return launch_strided_ws_t<8, 4>(a, n, s);
        case 9: return launch_strided_ws_t<9, 4>(a, n, s);
    }
    return cudaErrorInvalidValue;
}

template <int H, bool C>
cudaError_t launch_mixed_c(const MixedArgs& m, int n, cudaStream_t s) {
    using Cfg = MixedCfg<H>;
    CUtensorMap map, smap;
    cudaError_t e = strided_maps(m.sa, n, H, 4, Cfg::kBox, &map, &smap);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mixed<H, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    if (e != cudaSuccess) return e;
    note_launch(kKindMixed);
    const int pi = prof_begin(kKindMixed, s);
    k_mixed<H, C><<<(unsigned)num_sms(), kMixedThreads, Cfg::kSmem, s>>>(m, map, smap);
    prof_end(pi, s);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_mixed_t(const MixedArgs& m, int n, cudaStream_t s) {
    return g_comp ? launch_mixed_c<H, true>(m, n, s) : launch_mixed_c<H, false>(m, n, s);
}

cudaError_t launch_mixed(int H, const MixedArgs& m, int n, cudaStream_t s) {
    switch (H) {
        case 6: return launch_mixed_t<6>(m, n, s);
        case 7: return launch_mixed_t<7>(m, n, s);
        case 8: return launch_mixed_t<8>(m, n, s);
        case 9: return launch_mixed_t<9>(m, n, s);
    }
    return cudaErrorInvalidValue;
}

// Split h strided bits above bit lo0 into near-equal passes of 3..9 bits.
bool make_passes(int lo0, int h, FusedPlan& p) {
    p.npass = 0;
    if (h == 0) return true;
    if (h < 3) return false;
    const int np = (h + kMaxStrided - 1) / kMaxStrided;
    if (np > 4) return false;
    int lo = lo0;
    for (int k = 0; k < np; ++k) {
        const int hb = h / np + (k < h % np ? 1 : 0);
        if (hb < 3 || hb > kMaxStrided) return false;
        p.lo[k] = lo;
        p.hb[k] = hb;
        lo += hb;
    }
    p.npass = np;
    return true;
}

}  // namespace

// The L2-blocked launches need an item counter and one counter per group of
// amplitudes: at most 2^(n - 17) groups for the blocked tail (its strided range has at
// least 6 bits), 2^(n - 16) for the blocked pair (bits [4, loA), loA <= n - 12).
constexpr int kMixedMinN = 22;
size_t mixed_counter_bytes(int gbits) { return 8 + ((size_t)4 << gbits); }

size_t fused_scratch_bytes(int n, int prec) {
    if (n < kMixedMinN || n > kMaxQubits) return 0;
    // float-float rows are 8 amplitudes: the pair's groups are bits [3, loA), one more bit
    return (mixed_counter_bytes(prec == 0 ? n - 16 : n - 15) + 255) / 256 * 256;
}

// Lag D of the blocked pair in groups: the B-tiles of group g follow the A-tiles of group
// g + D, so about D + 1 groups of b_{k+1} and q are live in L2. Measured at n = 28..30,
// the best D keeps that near 48 MB: D = 1 for 32 MB groups, D = 2 for 16 MB groups (one
// more group cost 10-27%). CHEB_PAIR_LAG (1..16) overrides the rule.
int pair_lag(size_t group_bytes) {
    static int env = -1;
    if (env < 0) {
        const char* e = std::getenv("CHEB_PAIR_LAG");
        const int v = e ? std::atoi(e) : 0;
        env = (v >= 1 && v <= 16) ? v : 0;
    }
    if (env > 0) return env;
    const int d = (int)((size_t)48 * 1024 * 1024 / std::max<size_t>(group_bytes, 1)) - 1;
    return std::min(std::max(d, 1), 8);
}

// 0: separate launches, 1: L2-blocked tail, 2: L2-blocked strided pair, -1: automatic:
// the strided pair from n = 26 on for FP32 (12-18% faster per step at n = 26..30) and
// from n = 28 on for the float-float path; separate launches below, where the vectors
// partly stay in L2 anyway.
static int g_blocking = -1;
void fused_set_blocking(int mode) { g_blocking = (mode >= -1 && mode <= 2) ? mode : -1; }
int fused_get_blocking() { return g_blocking; }
constexpr int kPairAutoMinN[2] = {26, 28};  // FP32, float-float

// Per-n choices of the autotuner (-1: not tuned): the blocked tail, and the AUTO path.
static int g_block_n[2][kMaxQubits + 1];
static int g_auto_path[2][kMaxQubits + 1];
static bool g_tuned_init = false;

static void tuned_init() {
    if (!g_tuned_init) {
        for (int i = 0; i <= kMaxQubits; ++i)
            g_block_n[0][i] = g_block_n[1][i] = g_auto_path[0][i] = g_auto_path[1][i] = -1;
        g_tuned_init = true;
    }
}

void tuned_set(int prec, int n, int path, int blocking) {
    std::lock_guard<std::mutex> lk(g_mu);
    tuned_init();
    if (n < 0 || n > kMaxQubits || prec < 0 || prec > 1) return;
    g_auto_path[prec][n] = path;
    g_block_n[prec][n] = blocking;
}

int tuned_auto_path(int prec, int n) {
    std::lock_guard<std::mutex> lk(g_mu);
    tuned_init();
    if (n < 0 || n > kMaxQubits || prec < 0 || prec > 1) return -1;
    return g_auto_path[prec][n];
}

int fused_blocking_for(int prec, int n) {
    std::lock_guard<std::mutex> lk(g_mu);
    tuned_init();
    if (prec < 0 || prec > 1) return 0;
    int m = (n >= 0 && n <= kMaxQubits && g_block_n[prec][n] >= 0) ? g_block_n[prec][n] : g_blocking;
    if (m < 0) m = n >= kPairAutoMinN[prec] ? 2 : 0;
    return (prec == 1 && m == 1) ? 0 : m;  // the blocked tail is FP32 only
}
static int blocking_for(int n) { return fused_blocking_for(0, n); }

bool fused_blocking_eligible(const FusedPlan& plan) {
    const int lastp = plan.npass - 1;
    return plan.prec == 0 && plan.n >= kMixedMinN && plan.npass >= 2 && plan.l <= 1 && plan.hb[lastp] >= 6 &&
           plan.hb[lastp] <= kMaxStrided;
}
bool fused_pair_eligible(const FusedPlan& plan) {
    return plan.prec == 0 && plan.n >= kMixedMinN && plan.npass == 2 && pairk::shape_ok(plan.hb[0], plan.hb[1]);
}
void fused_set_compensated(int on) { g_comp = on ? 1 : 0; }
int fused_get_compensated() { return g_comp; }

bool fused_supported(int n, int prec) { return prec == 0 && n >= kLowBits && n <= kMaxQubits; }

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
    if (n < kLowBits || n > kMaxQubits || l < 0 || l > kMaxL || h < 0 || kLowBits + l + h != n) return false;
    FusedPlan p;
    return make_passes(kLowBits + l, h, p);
}

bool fused_set_split(int n, int l, int h) {
    std::lock_guard<std::mutex> lk(g_mu);
    split_table_init();
    if (n < kLowBits || n > kMaxQubits) return false;
    if (l < 0) {
        g_split_l[n] = g_split_h[n] = -1;
        return true;
    }
    if (!fused_split_valid(n, l, h)) return false;
    g_split_l[n] = l;
    g_split_h[n] = h;
    return true;
}

// Default split: the fewest strided passes reachable with at most 4 L2 partner bits
// (each partner bit costs 8 B per amplitude of L2 reads, which saturate the L2 -> SM
// path beyond ~4 bits), then the fewest partner bits for that number of passes. If
// the top pass would then be a 9-bit range at bit 18 or above, one more partner bit
// (up to 4) makes it an 8-bit range of wide rows: at n = 30, (2, 17) with passes of
// 9 + 8 bits ran 6% faster per step than (1, 18) with 9 + 9.
FusedPlan fused_plan(int n, int prec) {
    FusedPlan p;
    p.n = n;
    p.prec = prec;
    p.M = kLowBits;
    int l = -1, h = -1;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        split_table_init();
        if (n >= kLowBits && n <= kMaxQubits && g_split_l[n] >= 0) {
            l = g_split_l[n];
            h = g_split_h[n];
        }
    }
    if (l < 0) {
        const int rest = n - kLowBits;
        if (rest <= 3) {
            l = rest;
        } else {
            const int np = (std::max(rest - 4, 0) + kMaxStrided - 1) / kMaxStrided;
            l = std::max(0, rest - kMaxStrided * np);
            if (rest - l > 0 && rest - l < 3) l = rest - 3;
        }
        h = rest - l;
        FusedPlan q;
        if (h > kMaxStrided && l < 4 && make_passes(kLowBits + l, h, q) && q.hb[q.npass - 1] == kMaxStrided &&
            q.lo[q.npass - 1] >= 18 && fused_split_valid(n, l + 1, h - 1)) {
            ++l;
            --h;
        }
        // 9 + 8 strided ranges over a low pass without L2 partner bits (n = 28): one bit
        // moves to the low pass, which costs it nothing there (1.29 ms either way), and
        // the blocked pair runs two 8-bit ranges on one-float tiles (2.85 against 2.93 ms
        // per step)
        if (l == 0 && h == 2 * 8 + 1 && fused_split_valid(n, 1, h - 1)) {
            l = 1;
            --h;
        }
    }
    p.l = l;
    p.h = h;
    make_passes(kLowBits + l, h, p);
    return p;
}

cudaError_t launch_step_fused(const FusedPlan& plan, const StepArgs& s, void* scratch, int* flags, cudaStream_t st) {
    if (plan.prec != 0 || plan.n != s.n || !fused_split_valid(s.n, plan.l, plan.h) || s.M != kLowBits)
        return cudaErrorInvalidValue;
    const float ghi = (float)s.g;
    const float glo = (float)(s.g - (double)ghi);
    float slot_coeff = (float)s.sgn;
    // The strided passes build the partial q in `out` when out is a separate
    // buffer (b2 is then left intact), else in place in b2.
    float4* q = (s.out != s.psi && s.out != s.b1) ? (float4*)s.out : (float4*)s.b2;
    // The last strided pass and the low pass run as one L2-blocked launch when enabled
    // and the plan allows it (an earlier strided pass, at most one L2 partner bit, a
    // last range of 6..9 bits, scratch for the counters).
    const int lastp = plan.npass - 1;
    const int mode = blocking_for(s.n);
    const bool mixed = mode == 1 && scratch != nullptr && s.n >= kMixedMinN && plan.npass >= 2 && plan.l <= 1 &&
                       plan.hb[lastp] >= 6 && plan.hb[lastp] <= kMaxStrided && s.out != s.b1;
    // The two strided passes of a two-pass plan run as one L2-blocked launch (plain
    // flip sums only).
    const bool pair = mode == 2 && !g_comp && scratch != nullptr && fused_pair_eligible(plan) && s.out != s.b1;
    if (pair) {
        pairk::Args pa{};
        pa.b1 = (const float4*)s.b1;
        pa.slot_in = (const float4*)s.b2;
        pa.slot = q;
        pa.loA = plan.lo[0];
        pa.loB = plan.lo[1];
        pa.scale_g = (float)s.scale * ghi;
        pa.scale_glo = (float)s.scale * glo;
        pa.sgn = (float)s.sgn;
        pa.gbits = plan.lo[0] - ArithF32::kRowBits;
        const size_t group_bytes = (size_t)16 << (4 + plan.hb[0] + plan.hb[1]);  // b_{k+1} and q
        pa.lag = (int)std::min<int64_t>(pair_lag(group_bytes), (int64_t)1 << pa.gbits);
        pa.work = (unsigned long long*)scratch;
        pa.done = (unsigned*)((unsigned char*)scratch + 8);
        pa.flags = flags;
        cudaError_t e = cudaMemsetAsync(scratch, 0, mixed_counter_bytes(pa.gbits), st);
        if (e != cudaSuccess) return e;
        e = pairk::launch<ArithF32>(plan.hb[0], plan.hb[1], pa, s.n, st);
        if (e != cudaSuccess) return e;
        slot_coeff = 1.0f;
    }
    const int nsep = pair ? 0 : (mixed ? lastp : plan.npass);  // strided passes launched on their own
    for (int k = 0; k < nsep; ++k) {
        StridedArgs sa;
        sa.b1 = (const float4*)s.b1;
        sa.slot_in = (k == 0) ? (const float4*)s.b2 : q;
        sa.slot = q;
        sa.lo = plan.lo[k];
        const int rb = strided_row_bits(plan.lo[k], plan.hb[k]);
        sa.ntiles = (int64_t)1 << (s.n - plan.hb[k] - rb);
        sa.scale_g = (float)s.scale * ghi;
        sa.scale_glo = (float)s.scale * glo;
        sa.sgn = (k == 0) ? (float)s.sgn : 1.0f;
        sa.flags_ws = flags;
        cudaError_t e = launch_strided(plan.hb[k], rb, sa, s.n, st);
        if (e != cudaSuccess) return e;
        slot_coeff = 1.0f;  // the slot now holds q
    }
    LowArgs la;
    la.b1 = (const float4*)s.b1;
    la.slot = plan.npass > 0 ? q : (const float4*)s.b2;
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
    if (mixed) {
        MixedArgs m;
        m.sa.b1 = (const float4*)s.b1;
        m.sa.slot_in = q;
        m.sa.slot = q;
        m.sa.lo = plan.lo[lastp];
        m.sa.ntiles = (int64_t)1 << (s.n - plan.hb[lastp] - 4);
        m.sa.scale_g = (float)s.scale * ghi;
        m.sa.scale_glo = (float)s.scale * glo;
        m.sa.sgn = 1.0f;
        m.sa.flags_ws = flags;
        m.la = la;
        m.gbits = plan.lo[lastp] - kLowBits;
        // about six items per SM between a group's strided tiles and its low tiles;
        // the groups in that window (b_{k+1} and q, 2^(15 + H) bytes each) stay in L2
        {
            const int per_seg = 128 + (1 << plan.hb[lastp]);
            const int want = (6 * num_sms() + per_seg - 1) / per_seg;
            m.lag = std::min(std::max(want, 2), 8);
            m.lag = (int)std::min<int64_t>(m.lag, (int64_t)1 << m.gbits);
        }
        m.work = (unsigned long long*)scratch;
        m.done = (unsigned*)((unsigned char*)scratch + 8);
        cudaError_t e = cudaMemsetAsync(scratch, 0, mixed_counter_bytes(m.gbits), st);
        if (e != cudaSuccess) return e;
        return launch_mixed(plan.hb[lastp], m, s.n, st);
    }
    auto kern = g_comp ? k_low<true> : k_low<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLowSmem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(la.ntiles, num_sms());
    note_launch(kKindLow);
    const int pi = prof_begin(kKindLow, st);
    const cudaError_t le = launch_step_kernel(kern, (unsigned)grid, kLowThreads, kLowSmem, st, la);
    prof_end(pi, st);
    return le;
}

}  // namespace cheb
