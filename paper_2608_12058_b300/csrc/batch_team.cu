// One persistent launch for a whole batch of independent FP32 instances (Sec. III.A
// batches many problems per launch so that no instance pays for launches of its own).
//
// The launch has one CTA of 512 threads per SM (a cooperative launch, so that every CTA
// is resident).
// Work is a list of slots, instances sorted longest first (2^n K) by the host; a CTA
// takes the next slot from a global counter, runs it, and takes another:
//  * n <= 12: one slot, the whole Clenshaw run in the CTA's shared memory (psi, b_{k+1},
//    b_{k+2}: 96 KB at n = 12).
//  * n >= 13: `team` consecutive slots (2^(n-14) CTAs, 1..64); the team runs the
//    instance step by step with the vectors in global memory (L2-resident at these
//    sizes) and a bounded team barrier after every pass. A step is
//      - for n >= 16 a strided pass over bits [11, n): tiles of 2^(n-11) rows of 16
//        amplitudes in shared memory, q = scale g S + sgn b_{k+2} written over b_{k+2};
//      - a low pass over bits [0, 11) from a shared-memory tile of 2048 amplitudes (and
//        for n = 12..15 bits [11, n) from the partner tiles in L2), with the Ising
//        diagonal rebuilt from the tile's energy table row, writing
//        out = scale (Dt b_{k+1} + g S) + q + c_k psi.
//    Team members share data only through L2: every load of a team-shared vector
//    bypasses L1 (ld.global.cg), and a barrier is a release fence, an atomic arrival
//    and a bounded acquire spin. A CTA loads the next low tile's data into registers
//    while it computes the current one.
// Slots are handed out in order, so at most the last team being formed is incomplete
// and every earlier team can finish: the schedule cannot deadlock. Every wait gives up
// after ~2 s with the timeout flag set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "batch_team.cuh"
#include "fused.cuh"
#include "cheb_internal.h"
#include "kernels.cuh"
#include "kernels_dev.cuh"
#include "mbar.cuh"

namespace cheb {
namespace {

constexpr int kTeamThreads = 512;
constexpr int kTileF4 = 1024;  // float4 per 2048-amplitude low tile
// Whole-run items keep psi, b_{k+1}, b_{k+2} in shared memory, up to n = 12 (96 KB); a
// team of one CTA stepping through L2 was measured faster for n = 13 than a whole run in
// 192 KB (whose 16 amplitudes per thread spill registers).
constexpr int small_max(int ctas_per_sm) { return ctas_per_sm >= 2 ? 12 : 12; }
constexpr size_t team_smem(int ctas_per_sm) { return 3 * ((size_t)1 << small_max(ctas_per_sm)) * 8; }

__device__ __forceinline__ float4 ldcg4(const float4* p) { return __ldcg(p); }

// Bounded team barrier: every thread's writes of this CTA are released, the CTA arrives,
// and thread 0 waits (acquire) until `target` arrivals are counted.
__device__ bool team_barrier(unsigned* bar, unsigned target, int* flags, int* s_ok, long long limit = kWaitCycles) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int good = 1;
        const long long t0 = clock64();
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > limit) {
                atomicOr(flags, kFlagTimeout);
                good = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        *s_ok = good;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 dupf(float x) { return make_float2(x, x); }

// o = scale (d v + g s) + sgn q + c p for one complex amplitude (d = dh + dl, g = gh + gl).
__device__ __forceinline__ float2 combine1(float dh, float dl, float2 v, float2 gh, float2 gl, float2 s, float2 sc,
                                           float2 sg, float2 q, float2 cr, float2 ci_s, float2 p) {
    float2 h = __ffma2_rn(dupf(dh), v, __fmul2_rn(dupf(dl), v));
    h = add2(h, __ffma2_rn(gh, s, __fmul2_rn(gl, s)));
    float2 o = __ffma2_rn(sc, h, __fmul2_rn(sg, q));
    o = __ffma2_rn(cr, p, o);
    return __ffma2_rn(ci_s, make_float2(p.y, p.x), o);  // ci_s = (-ci, ci)
}

// Strided pass of a team over bits [11, 11 + H), H = 6..9: 128 tiles of 2^H rows x 8 float4
// (rows 1024 float4 apart); this CTA takes tiles r, r + T, ... Thread t owns float4
// t & 7 of the 2^(H-6) rows whose bits 0..5 are t >> 3: it loads them (and their slot
// b_{k+2}, in two halves) in batches of L2-only loads, keeps them in registers for the
// flips of row bits 6..H-1 and reads only the flips of bits 0..5 from shared memory.
// Writes q = scale g S + sgn b_{k+2} over b_{k+2}.
template <int H>
__device__ __noinline__ void team_strided(const float4* b1, float4* b2, float4* st, int r, int T, float2 g2h,
                                             float2 g2l, float sgn) {
    constexpr int P = 1 << (H - 6);
    const int t = threadIdx.x;
    const int u = t & 7, rq = t >> 3;
    const bool need = sgn != 0.f;
    const float2 sg = dupf(sgn);
    constexpr int PH = P > 1 ? P / 2 : 1;  // slot values loaded in two halves (registers)
    for (int tile = r; tile < 128; tile += T) {
        float4 v[P], w[PH];
#pragma unroll
        for (int i = 0; i < P; ++i) v[i] = ldcg4(b1 + tile * 8 + (int64_t)(rq + 64 * i) * kTileF4 + u);
        if (need) {
#pragma unroll
            for (int i = 0; i < PH; ++i) w[i] = ldcg4(b2 + tile * 8 + (int64_t)(rq + 64 * i) * kTileF4 + u);
        }
#pragma unroll
        for (int i = 0; i < P; ++i) st[((rq + 64 * i) << 3) + u] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (need && i == PH) {
#pragma unroll
                for (int m = 0; m < PH; ++m)
                    w[m] = ldcg4(b2 + tile * 8 + (int64_t)(rq + 64 * (PH + m)) * kTileF4 + u);
            }
            float2 Sa = make_float2(0.f, 0.f), Sb = Sa;
#pragma unroll
            for (int b = P >> 1; b >= 1; b >>= 1) {  // row bits H-1 .. 6 from registers
                Sa = add2(Sa, lo2(v[i ^ b]));
                Sb = add2(Sb, hi2(v[i ^ b]));
            }
#pragma unroll
            for (int j = 5; j >= 0; --j) {  // row bits 5 .. 0 from shared memory
                const float4 pv = st[(((rq ^ (1 << j)) + 64 * i) << 3) + u];
                Sa = add2(Sa, lo2(pv));
                Sb = add2(Sb, hi2(pv));
            }
            float2 qa = __ffma2_rn(g2h, Sa, __fmul2_rn(g2l, Sa));
            float2 qb = __ffma2_rn(g2h, Sb, __fmul2_rn(g2l, Sb));
            if (need) {
                const float4 wi = w[i % PH];
                qa = __ffma2_rn(sg, lo2(wi), qa);
                qb = __ffma2_rn(sg, hi2(wi), qb);
            }
            b2[tile * 8 + (int64_t)(rq + 64 * i) * kTileF4 + u] = make_float4(qa.x, qa.y, qb.x, qb.y);
        }
        __syncthreads();
    }
}

// One instance on a team of CTAs (rank r of T). Returns false after a timeout.
// Low pass layout (as the fused low pass): thread t holds float4 t and t + 512 of a
// tile, i.e. amplitudes 2t + 1024 p + w: bit 0 = w, bits 1..9 = t, bit 10 = p.
__device__ bool team_run(const TeamInst& I, int r, unsigned char* smem, int* flags) {
    __shared__ int s_ok;
    __shared__ int64_t W[50];
    const int t = threadIdx.x;
    const int n = I.n, T = I.team, l = I.l, H = I.H;
    const int64_t nlow = (int64_t)1 << (n - 11);  // low tiles
    float4* psi = I.psi;
    float4* B[2] = {I.v0, I.v1};
    float4* st = (float4*)smem;
    unsigned target = 0;
    const float ghi = (float)I.g, glo = (float)(I.g - (double)ghi);
    const int scale_hi = (127 + 32 - I.Q) << 23, scale_lo = (127 - I.Q) << 23;
    // energy terms among bits 0..10 for this thread's four amplitudes (p, w)
    const int64_t el00 = __ldg(I.elow + 2 * t), el01 = __ldg(I.elow + 2 * t + 1);
    const int64_t el10 = __ldg(I.elow + 1024 + 2 * t), el11 = __ldg(I.elow + 1024 + 2 * t + 1);
    // b_K = c_K psi into B[1]
    {
        const double2 cK = I.coef[I.K];
        const float2 cr = dupf((float)cK.x), ci_s = make_float2(-(float)cK.y, (float)cK.y);
        for (int64_t T0 = r; T0 < nlow; T0 += T) {
            for (int p = 0; p < 2; ++p) {
                const int64_t z = T0 * kTileF4 + t + 512 * p;
                const float4 v = ldcg4(psi + z);
                const float2 a = __ffma2_rn(cr, lo2(v), __fmul2_rn(ci_s, make_float2(v.y, v.x)));
                const float2 b = __ffma2_rn(cr, hi2(v), __fmul2_rn(ci_s, make_float2(v.w, v.z)));
                B[1][z] = make_float4(a.x, a.y, b.x, b.y);
            }
        }
    }
    target += T;
    if (!team_barrier(I.bar, target, flags, &s_ok)) return false;
    int cur = 1;
    for (int k = I.K - 1; k >= 0; --k) {
        const float4* b1 = B[cur];
        float4* b2 = B[cur ^ 1];
        float4* out = (k == 0) ? psi : b2;
        const float sc = (k == 0) ? 1.f : 2.f;
        float sgn = (k == I.K - 1) ? 0.f : -1.f;
        if (H >= 6) {
            // strided pass over bits [11, n) with rows held in registers (team_strided)
            const float2 g2h = dupf(sc * ghi), g2l = dupf(sc * glo);
            switch (H) {
                case 6: team_strided<6>(b1, b2, st, r, T, g2h, g2l, sgn); break;
                case 7: team_strided<7>(b1, b2, st, r, T, g2h, g2l, sgn); break;
                case 8: team_strided<8>(b1, b2, st, r, T, g2h, g2l, sgn); break;
                default: team_strided<9>(b1, b2, st, r, T, g2h, g2l, sgn); break;
            }
            target += T;
            if (!team_barrier(I.bar, target, flags, &s_ok)) return false;
            sgn = 1.f;  // b_{k+2} now holds q
        } else if (H > 0) {
            // strided pass over bits [11, n): 128 tiles of 2^H rows x 8 float4, rows 1024
            // float4 apart; q = scale g S + sgn b_{k+2} written over b_{k+2}
            const int elems = 8 << H;
            const float2 g2h = dupf(sc * ghi), g2l = dupf(sc * glo), sg = dupf(sgn);
            for (int tile = r; tile < 128; tile += T) {
                for (int idx = t; idx < elems; idx += kTeamThreads)
                    st[idx] = ldcg4(b1 + tile * 8 + (int64_t)(idx >> 3) * kTileF4 + (idx & 7));
                __syncthreads();
                for (int idx = t; idx < elems; idx += kTeamThreads) {
                    const int row = idx >> 3, u = idx & 7;
                    const int64_t z = tile * 8 + (int64_t)row * kTileF4 + u;
                    const float4 w = (sgn != 0.f) ? ldcg4(b2 + z) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float2 Sa = make_float2(0.f, 0.f), Sb = Sa;
                    for (int j = 0; j < H; ++j) {
                        const float4 pv = st[((row ^ (1 << j)) << 3) + u];
                        Sa = add2(Sa, lo2(pv));
                        Sb = add2(Sb, hi2(pv));
                    }
                    const float2 qa = __ffma2_rn(sg, lo2(w), __ffma2_rn(g2h, Sa, __fmul2_rn(g2l, Sa)));
                    const float2 qb = __ffma2_rn(sg, hi2(w), __ffma2_rn(g2h, Sb, __fmul2_rn(g2l, Sb)));
                    b2[z] = make_float4(qa.x, qa.y, qb.x, qb.y);
                }
                __syncthreads();
            }
            target += T;
            if (!team_barrier(I.bar, target, flags, &s_ok)) return false;
            sgn = 1.f;  // b_{k+2} now holds q
        }
        const double2 ck = I.coef[k];
        const float2 cr = dupf((float)ck.x), ci_s = make_float2(-(float)ck.y, (float)ck.y);
        const float2 gh = dupf(ghi), gl = dupf(glo), scv = dupf(sc), sg = dupf(sgn);
        const bool need_q = sgn != 0.f;
        // the next tile's b_{k+1}, psi and q are loaded while this one is computed
        float4 nv0, nv1, np0, np1, nq0, nq1;
        auto fetch = [&](int64_t T0) {
            const int64_t z = T0 * kTileF4 + t;
            nv0 = ldcg4(b1 + z);
            nv1 = ldcg4(b1 + z + 512);
            np0 = ldcg4(psi + z);
            np1 = ldcg4(psi + z + 512);
            if (need_q) {
                nq0 = ldcg4(b2 + z);
                nq1 = ldcg4(b2 + z + 512);
            } else {
                nq0 = nq1 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        if (r < nlow) fetch(r);
        for (int64_t T0 = r; T0 < nlow; T0 += T) {
            const float4 v0 = nv0, v1 = nv1, ps0 = np0, ps1 = np1, q0 = nq0, q1 = nq1;
            if (T0 + T < nlow) fetch(T0 + T);
            st[t] = v0;
            st[t + 512] = v1;
            // energy partial sums of the tile (as in the fused low pass)
            if (t < 50) {
                const int64_t* row = I.tiles + T0 * 12;
                int64_t e = 0;
                if (t < 32) {
                    e = __ldg(row + 11);
#pragma unroll
                    for (int i = 1; i <= 5; ++i) {
                        const int64_t f = __ldg(row + i);
                        e += ((t >> (i - 1)) & 1) ? -f : f;
                    }
                } else if (t < 48) {
#pragma unroll
                    for (int i = 6; i <= 9; ++i) {
                        const int64_t f = __ldg(row + i);
                        e += (((t - 32) >> (i - 6)) & 1) ? -f : f;
                    }
                } else {
                    const int64_t f10 = __ldg(row + 10), f0 = __ldg(row);
                    e = (t == 48) ? f10 + f0 : f10 - f0;
                }
                W[t] = e;
            }
            float2 S0a = make_float2(0.f, 0.f), S0b = S0a, S1a = S0a, S1b = S0a;
            for (int j = 0; j < l; ++j) {  // bits 11..: partner tiles in L2
                const int64_t pz = (T0 ^ ((int64_t)1 << j)) * kTileF4 + t;
                const float4 p0 = ldcg4(b1 + pz), p1 = ldcg4(b1 + pz + 512);
                S0a = add2(S0a, lo2(p0));
                S0b = add2(S0b, hi2(p0));
                S1a = add2(S1a, lo2(p1));
                S1b = add2(S1b, hi2(p1));
            }
            __syncthreads();
            // bit 0 (other half of the float4) and bit 10 (the other float4)
            S0a = add2(S0a, add2(hi2(v0), lo2(v1)));
            S0b = add2(S0b, add2(lo2(v0), hi2(v1)));
            S1a = add2(S1a, add2(hi2(v1), lo2(v0)));
            S1b = add2(S1b, add2(lo2(v1), hi2(v0)));
#pragma unroll
            for (int j = 0; j < 9; ++j) {  // bits 1..9: partner threads
                const float4 p0 = st[t ^ (1 << j)], p1 = st[(t ^ (1 << j)) + 512];
                S0a = add2(S0a, lo2(p0));
                S0b = add2(S0b, hi2(p0));
                S1a = add2(S1a, lo2(p1));
                S1b = add2(S1b, hi2(p1));
            }
            const int64_t base = W[t & 31] + W[32 + (t >> 5)];
            const int64_t up = W[48], um = W[49];
            const int64_t e00 = base + up + el00, e01 = base + um + el01;
            const int64_t e10 = base - um + el10, e11 = base - up + el11;
            auto dd = [&](int64_t e, float& dh, float& dl) {
                dh = __int2float_rn((int)(e >> 32)) * __int_as_float(scale_hi);
                dl = __uint2float_rn((unsigned)(e & 0xffffffffll)) * __int_as_float(scale_lo);
            };
            float dh, dl;
            dd(e00, dh, dl);
            const float2 o00 = combine1(dh, dl, lo2(v0), gh, gl, S0a, scv, sg, lo2(q0), cr, ci_s, lo2(ps0));
            dd(e01, dh, dl);
            const float2 o01 = combine1(dh, dl, hi2(v0), gh, gl, S0b, scv, sg, hi2(q0), cr, ci_s, hi2(ps0));
            dd(e10, dh, dl);
            const float2 o10 = combine1(dh, dl, lo2(v1), gh, gl, S1a, scv, sg, lo2(q1), cr, ci_s, lo2(ps1));
            dd(e11, dh, dl);
            const float2 o11 = combine1(dh, dl, hi2(v1), gh, gl, S1b, scv, sg, hi2(q1), cr, ci_s, hi2(ps1));
            const int64_t z = T0 * kTileF4 + t;
            out[z] = make_float4(o00.x, o00.y, o01.x, o01.y);
            out[z + 512] = make_float4(o10.x, o10.y, o11.x, o11.y);
            __syncthreads();
        }
        if (k > 0) {
            target += T;
            if (!team_barrier(I.bar, target, flags, &s_ok)) return false;
        }
        cur ^= 1;
    }
    return true;
}

// MB: CTAs per SM the kernel is compiled for (1: 128 registers per thread, the default;
// 2: 64 registers, with spills); cheb_set_batch_persistent picks the variant.
template <int MB>
__global__ void __launch_bounds__(kTeamThreads, MB)
    k_batch_team(const TeamInst* __restrict__ inst, int ninst, int nslots, unsigned* slot_counter, int* flags) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_slot;
    while (true) {
        if (threadIdx.x == 0) s_slot = (int)atomicAdd(slot_counter, 1u);
        __syncthreads();
        const int slot = s_slot;
        __syncthreads();
        if (slot >= nslots) return;
        // the instance that owns this slot: the last one whose first slot is <= slot
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].first_slot <= slot) lo = mid;
            else hi = mid - 1;
        }
        const TeamInst& I = inst[lo];
        if (I.team == 0) {
            small_run<float, 1 << (small_max(MB) - 9)>(I.n, I.K, I.coef, I.Q, I.tiles, I.elow, I.g,
                                                       (float2*)I.psi, smem);
            __syncthreads();
        } else if (!team_run(I, slot - I.first_slot, smem, flags)) {
            return;
        }
    }
}

// One CTA of a team of two: its barrier waits for a teammate that never comes.
__global__ void k_team_barrier_selftest(unsigned* bar, int* flags, long long limit) {
    __shared__ int s_ok;
    team_barrier(bar, 2u, flags, &s_ok, limit);
}

}  // namespace

cudaError_t launch_team_barrier_selftest(unsigned* bar, int* flags, long long limit, cudaStream_t s) {
    note_launch(kKindReduce);
    k_team_barrier_selftest<<<1, 32, 0, s>>>(bar, flags, limit);
    return cudaGetLastError();
}

// Larger teams measured faster on the 512-instance workload (teams of 2^(n-14) against
// 2^(n-15): 782 against 945 ms): more CTAs per instance keep fewer instances, and so
// fewer vectors, in flight in L2.
int team_size(int n, int ctas_per_sm) {
    if (n <= small_max(ctas_per_sm)) return 0;
    const int e = n - 14;
    return e <= 0 ? 1 : std::min(64, 1 << e);
}

void team_split(int n, int* l, int* H) {
    if (n <= 11) {
        *l = 0;
        *H = 0;
    } else if (n <= 15) {
        *l = n - 11;
        *H = 0;
    } else {
        *l = 0;
        *H = n - 11;
    }
}

cudaError_t launch_batch_team(const TeamInst* inst, int ninst, int nslots, unsigned* slot_counter, int* flags,
                              int ctas_per_sm, cudaStream_t s) {
    if (ninst <= 0) return cudaSuccess;
    const int mb = ctas_per_sm >= 2 ? 2 : 1;
    const void* kern = mb == 2 ? (const void*)k_batch_team<2> : (const void*)k_batch_team<1>;
    const size_t smem = team_smem(mb);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTeamThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    per_sm = std::min(per_sm, mb);
    const int grid = std::min(num_sms() * per_sm, nslots);
    void* args[] = {(void*)&inst, (void*)&ninst, (void*)&nslots, (void*)&slot_counter, (void*)&flags};
    note_launch(kKindSmall);
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kTeamThreads), args, smem, s);
}

}  // namespace cheb
