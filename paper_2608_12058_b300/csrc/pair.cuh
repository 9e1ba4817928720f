// L2-blocked pair of strided passes (the flips of the hypercube matvec, Sec. II.D, over
// the two strided ranges of a step), generic over the arithmetic: FP32 complex64
// vectors (fused.cu) and float-float vectors of the FP64 path (fused_ff.cu) share the
// schedule, the pipeline and the tile layout; Arith supplies the flip-sum accumulator
// and the final q = s g S + sgn slot.
//
// The two ranges A = [loA, loB) and B = [loB, n) run in one persistent launch, on rows
// of 128 bytes (2^kRowBits amplitudes: 16 complex64 or 8 float-float). The amplitudes are
// grouped by their bits [kRowBits, loA): a group holds 2^(kRowBits + HA + HB) amplitudes,
// 2^HB A-tiles (one per value of the bits of B) and 2^HA B-tiles (one per value of the
// bits of A). A-tiles read b_{k+1} and the slot (b_{k+2}) from DRAM and write
// q = s g S_A + sgn slot; the B-tiles of the same group, D groups later, read b_{k+1}
// and q back from L2 and write q + s g S_B, so the two strided passes of a step move
// half the DRAM bytes of two separate passes.
//
// Work items in order: A(0) .. A(D - 1), then A(s) followed by B(s - D) for
// s = D .. G - 1, then B(G - D) .. B(G - 1). CTAs take items from a global counter (one
// ahead); before loading a B-tile the producer waits (bounded) until all A-tiles of its
// group are published by the notifier warps (fence, then the group count), so an item
// only waits on items taken before it. The producer decodes each item once and leaves
// kind, group and index in shared memory for the consumers.
//
// Consumers: 512 threads. In a tile of 2^H rows (8 float4 each) thread t holds float4
// u = t & 7 of the 2^(H-6) rows whose bits 0..5 are t >> 3: the flips of row bits
// 6..H-1 come from registers and those of bits 0..5 from shared memory, 8 shared-memory
// reads per float4 (the TMA fill, the own value, six partners) against 10 in the
// one-pass kernels. An A-tile's slot is read with L2-only loads, or by TMA with the tile
// when tiles have at most 8 bits (a stage then holds both); so is a B-tile's q, which
// other SMs wrote in this launch. FP32 tiles whose slot is staged take a layout with
// one float per lane (tile_lanes), which reads four flips from shared memory instead of
// six. The flip sum runs in descending bit order, as in the one-pass kernels, so the
// pair and two separate passes agree bit for bit.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cheb_internal.h"
#include "fused.cuh"
#include "kernels.cuh"
#include "mbar.cuh"

namespace cheb {
namespace pairk {

constexpr int kCons = 512;
constexpr int kThreads = kCons + 64;  // + producer warp + notifier warp
constexpr int kItemA = 0, kItemB = 1, kItemEnd = 2;

struct Item {
    int kind;
    int64_t g;    // group
    int64_t idx;  // A: value of the bits of B; B: value of the bits of A
};

struct Args {
    const float4* b1;
    const float4* slot_in;  // b_{k+2} (read by the A-tiles when sgn != 0)
    float4* slot;           // receives q (may equal slot_in)
    int loA, loB;           // loB = loA + HA, n = loB + HB
    float scale_g, scale_glo;  // FP32: s g as a float-float pair
    float g2, g1, g0;          // float-float path: s g as a normalised triple
    float sgn;
    unsigned long long* work;  // item counter (zero at launch)
    unsigned* done;            // per group: A-tiles published (zero at launch)
    int gbits;                 // loA - kRowBits (2^gbits groups)
    int lag;                   // D, 1 <= D <= 2^gbits
    int* flags;
};

__host__ __device__ __forceinline__ Item decode(unsigned long long i, int gbits, int HA, int HB, int lag) {
    const unsigned long long G = 1ull << gbits, D = (unsigned long long)lag, NA = 1ull << HB, NB = 1ull << HA;
    const unsigned long long seg = NA + NB, head = D * NA;
    if (i < head) return {kItemA, (int64_t)(i / NA), (int64_t)(i % NA)};
    const unsigned long long j = i - head, s = D + j / seg;
    if (s < G) {
        const unsigned long long r = j % seg;
        return r < NA ? Item{kItemA, (int64_t)s, (int64_t)r} : Item{kItemB, (int64_t)(s - D), (int64_t)(r - NA)};
    }
    const unsigned long long k = j - (G - D) * seg, g = G - D + k / NB;
    if (g < G) return {kItemB, (int64_t)g, (int64_t)(k % NB)};
    return {kItemEnd, 0, 0};
}

template <int HA, int HB>
struct Cfg {
    static constexpr int kHMax = HA > HB ? HA : HB;
    static constexpr uint32_t kTileMax = (uint32_t)128 << kHMax;  // largest tile
    static constexpr uint32_t kBytesA = (uint32_t)128 << HA;
    static constexpr uint32_t kBytesB = (uint32_t)128 << HB;
    // Tiles of up to 8 bits: a stage holds a tile and its slot rows (three stages of
    // 64 KB), so the consumers read nothing from global memory and FP32 tiles take the
    // one-float-per-lane layout. With 9-bit tiles a stage holds the tile alone and both
    // slots come by L2-only loads (staging a narrower B-tile's q in the free half of its
    // stage, and ordering the narrower range first so that its b_{k+2} can be staged,
    // both measured slower at n=30, FP32).
    static constexpr bool kFull = kHMax <= 8;
    static constexpr uint32_t kStage = kFull ? 2 * kTileMax : kTileMax;
    static constexpr uint32_t kSlotOff = kTileMax;
    static constexpr int kNSraw = (int)((200u * 1024u) / kStage);
    static constexpr int kNS = kNSraw < 6 ? kNSraw : 6;
    static constexpr int kNR = 8;  // completion records in flight
    static constexpr size_t kItemOff = (size_t)kNS * kStage;  // per stage: kind, group, index
    static constexpr size_t kNoteOff = kItemOff + 3 * 8 * sizeof(long long);
    static constexpr size_t kBarOff = kNoteOff + (size_t)kNR * sizeof(int64_t);
    static constexpr size_t kAbortOff = kBarOff + (size_t)(2 * kNS + 2 * kNR) * sizeof(uint64_t);
    static constexpr size_t kSmem = kAbortOff + 16;
    static_assert(kNS >= 2 && kNS <= 8, "pair stages");
};

// One strided tile of 2^H rows (in shared memory, rows of 8 float4) on the 512
// consumer threads: q = s g S + sgn w for the rows' amplitudes, written to slot. The
// slot comes from qtile (shared memory, same layout as the tile) when it is not null,
// else from slot_in with L2-only loads.
template <int H, class Arith>
__device__ __forceinline__ void tile(const float4* __restrict__ t4, const float4* __restrict__ qtile,
                                     const float4* slot_in, float4* slot, int64_t base, int64_t row_stride_f4,
                                     const typename Arith::Scale& sc, float sgn, bool need_slot, uint64_t pol_store) {
    constexpr int P = 1 << (H - 6);
    const int t = threadIdx.x;
    const int u = t & 7, rq = t >> 3;
    float4 v[P];
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = t4[(rq | (i << 6)) * 8 + u];
    typename Arith::Acc S[P];
    // register bits H-1 .. 6 first (descending)
#pragma unroll
    for (int i = 0; i < P; ++i) {
        S[i].zero();
#pragma unroll
        for (int b = P >> 1; b >= 1; b >>= 1) S[i].add(v[i ^ b]);
    }
    float4 w[P];
    if (need_slot && !qtile) {
#pragma unroll
        for (int i = 0; i < P; ++i) w[i] = ld_cg4(slot_in + base + (int64_t)(rq | (i << 6)) * row_stride_f4 + u);
    }
    // then row bits 5 .. 0 from shared memory
#pragma unroll
    for (int i = 0; i < P; ++i) {
#pragma unroll
        for (int j = 5; j >= 0; --j) S[i].add(t4[((rq ^ (1 << j)) | (i << 6)) * 8 + u]);
    }
    if (need_slot && qtile) {
#pragma unroll
        for (int i = 0; i < P; ++i) w[i] = qtile[(rq | (i << 6)) * 8 + u];
    }
#pragma unroll
    for (int i = 0; i < P; ++i)
        st_hint(slot + base + (int64_t)(rq | (i << 6)) * row_stride_f4 + u,
                Arith::finish(S[i], w[i], need_slot, sgn, sc), pol_store);
}

// The same tile with one float per lane, for FP32 vectors (whose flip sums and final
// q = s g S + sgn slot act on each float alone) with the slot rows staged in shared
// memory (qf, same layout as the tile): warp w holds row bits 0..3, the lane the float
// within the row and the register index row bits 4..H-1, 2^(H-4) rows kept as float2
// pairs of rows m and m + 2^(H-5). The flips of bits H-1..4 come from registers and those
// of bits 3..0 from shared memory: per 128-byte row 6 shared-memory wavefronts for the
// tile (TMA fill, own values, four partners) against 8 for the float4 layout. The flip
// sum runs in the same descending bit order, so both layouts give the same bits.
// Pointers and offsets are in floats.
template <int H, class Arith>
__device__ __forceinline__ void tile_lanes(const float* __restrict__ tf, const float* __restrict__ qf, float* slot,
                                           int64_t base, int64_t row_stride, const typename Arith::Scale& sc,
                                           float sgn, bool need_slot, uint64_t pol_store) {
    constexpr int P2 = 1 << (H - 5);  // row pairs per thread
    const int t = threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    auto lo_row = [&](int m) { return w | (m << 4); };
    auto hi_row = [&](int m) { return w | ((m + P2) << 4); };
    float2 v[P2];
#pragma unroll
    for (int m = 0; m < P2; ++m) v[m] = make_float2(tf[lo_row(m) * 32 + lane], tf[hi_row(m) * 32 + lane]);
    float2 S[P2];
    // register bits H-1 .. 4 first (descending); the top one swaps the rows of a pair
#pragma unroll
    for (int m = 0; m < P2; ++m) {
        S[m] = __fadd2_rn(make_float2(0.f, 0.f), make_float2(v[m].y, v[m].x));
#pragma unroll
        for (int b = P2 >> 1; b >= 1; b >>= 1) S[m] = __fadd2_rn(S[m], v[m ^ b]);
    }
    // then row bits 3 .. 0 from shared memory
#pragma unroll
    for (int m = 0; m < P2; ++m) {
#pragma unroll
        for (int j = 3; j >= 0; --j)
            S[m] = __fadd2_rn(S[m], make_float2(tf[(lo_row(m) ^ (1 << j)) * 32 + lane],
                                                tf[(hi_row(m) ^ (1 << j)) * 32 + lane]));
    }
#pragma unroll
    for (int m = 0; m < P2; ++m) {
        const float2 q = need_slot ? make_float2(qf[lo_row(m) * 32 + lane], qf[hi_row(m) * 32 + lane])
                                   : make_float2(0.f, 0.f);
        const float2 o = Arith::finish2(S[m], q, need_slot, sgn, sc);
        st_hint1(slot + base + (int64_t)lo_row(m) * row_stride + lane, o.x, pol_store);
        st_hint1(slot + base + (int64_t)hi_row(m) * row_stride + lane, o.y, pol_store);
    }
}

template <int HA, int HB, class Arith>
__global__ void __launch_bounds__(kThreads, 1)
    k_pair(const Args a, const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
           const __grid_constant__ CUtensorMap smapA, const __grid_constant__ CUtensorMap qmapB) {
    using C = Cfg<HA, HB>;
    static_assert(HA >= 6 && HA <= 9 && HB >= 6 && HB <= 9, "pair ranges");
    static_assert(C::kSmem <= 227 * 1024, "shared memory");
    constexpr int kAmpShift = Arith::kAmpShift;  // log2(amplitudes per float4)
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = (uint64_t*)(smem + C::kBarOff);
    uint64_t* empty = full + C::kNS;
    uint64_t* cdone = empty + C::kNS;   // an A-tile's q stores are issued (16 warps)
    uint64_t* cempty = cdone + C::kNR;  // the notifier has published that record
    volatile int* abort = (volatile int*)(smem + C::kAbortOff);
    // the producer decodes each item once: kind, group and index per stage
    long long* item = (long long*)(smem + C::kItemOff);
    volatile long long* note = (volatile long long*)(smem + C::kNoteOff);
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int sha = a.loA - Arith::kRowBits;
    if (t == 0) {
        for (int i = 0; i < C::kNS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kCons / 32);
        }
        for (int i = 0; i < C::kNR; ++i) {
            mbar_init(&cdone[i], kCons / 32);
            mbar_init(&cempty[i], 1);
        }
        *abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kCons / 32 + 1) {
        // ---------------- notifier warp ----------------
        if (lane != 0) return;
        for (long long j = 0;; ++j) {
            const int r = (int)(j % C::kNR);
            if (!mbar_wait(&cdone[r], (uint32_t)((j / C::kNR) & 1), a.flags, abort)) break;
            const long long g = note[r];
            if (g < 0) break;
            __threadfence();
            atomicAdd(a.done + g, 1u);
            mbar_arrive(&cempty[r]);
        }
        return;
    }

    if (warp == kCons / 32) {
        // ---------------- producer warp ----------------
        if (lane != 0) return;
        int last[C::kNS];
        for (int i = 0; i < C::kNS; ++i) last[i] = -1;
        // the A-tiles' b_{k+1} is read again by the B-tiles of their group
        const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
        // the next item is taken one ahead, so the counter's round trip overlaps the
        // current item (it is later in the order, so holding it cannot block anyone)
        unsigned long long nxt = atomicAdd(a.work, 1ull);
        constexpr int boxA = HA < 8 ? (1 << HA) : 256;
        constexpr int boxB = HB < 8 ? (1 << HB) : 256;
        for (int it = 0;; ++it) {
            const unsigned long long cur = nxt;
            const Item ci = decode(cur, a.gbits, HA, HB, a.lag);
            if (ci.kind != kItemEnd) nxt = atomicAdd(a.work, 1ull);
            const int s = it % C::kNS, k = it / C::kNS;
            if (k > 0 && !mbar_wait(&empty[s], (k - 1) & 1, a.flags, abort)) break;
            unsigned char* d = smem + (size_t)s * C::kStage;
            if (ci.kind == kItemEnd) {
                item[3 * s] = kItemEnd;
                mbar_arrive(&full[s]);
                last[s] = k;
                break;
            }
            if (ci.kind == kItemA) {
                // A-tile: bits [kRowBits, loA) = g, bits of B = idx
                item[3 * s] = kItemA;
                item[3 * s + 1] = ci.g;
                item[3 * s + 2] = ci.idx;
                const bool slot_tma = C::kFull && a.sgn != 0.f;
                mbar_expect_tx(&full[s], slot_tma ? 2 * C::kBytesA : C::kBytesA);
#pragma unroll
                for (int c = 0; c < (1 << HA) / boxA; ++c) {
                    tma_load_4d_hint(d + (size_t)c * boxA * 128, &mapA, 0, (int)ci.g, c * boxA, (int)ci.idx, &full[s],
                                     pol_last);
                    // the slot lines become q, which the group's B-tiles read back
                    if (slot_tma)
                        tma_load_4d_hint(d + C::kSlotOff + (size_t)c * boxA * 128, &smapA, 0, (int)ci.g, c * boxA,
                                         (int)ci.idx, &full[s], pol_last);
                }
                last[s] = k;
            } else {
                if (!wait_count(a.done + ci.g, 1u << HB, a.flags, abort)) break;
                // q of the group was written through the generic proxy by other SMs
                asm volatile("fence.proxy.async.global;" ::: "memory");
                item[3 * s] = kItemB;
                item[3 * s + 1] = ci.g;
                item[3 * s + 2] = ci.idx;
                mbar_expect_tx(&full[s], C::kFull ? 2 * C::kBytesB : C::kBytesB);
                const int tlo = (int)(ci.g | (ci.idx << sha));  // bits [kRowBits, loB)
#pragma unroll
                for (int c = 0; c < (1 << HB) / boxB; ++c) {
                    tma_load_4d_hint(d + (size_t)c * boxB * 128, &mapB, 0, tlo, c * boxB, 0, &full[s], pol_first);
                    if (C::kFull)
                        tma_load_4d_hint(d + C::kSlotOff + (size_t)c * boxB * 128, &qmapB, 0, tlo, c * boxB, 0,
                                         &full[s], pol_first);
                }
                last[s] = k;
            }
        }
        for (int i = 0; i < C::kNS; ++i)
            if (last[i] >= 0) mbar_drain(&full[i], last[i] & 1, a.flags);
        return;
    }

    // ---------------- consumer warps ----------------
    const typename Arith::Scale sc = Arith::scale(a);
    const bool need_a = a.sgn != 0.f;
    const uint64_t pol_last = policy_evict_last(), pol_first = policy_evict_first();
    // float4 strides of a row of each range: 2^lo amplitudes
    const int64_t rsA = (int64_t)1 << (a.loA - kAmpShift), rsB = (int64_t)1 << (a.loB - kAmpShift);
    long long sj = 0;  // completion records sent
    auto record = [&](long long g) -> bool {
        __syncwarp();
        bool ok = true;
        if (lane == 0) {
            const int r = (int)(sj % C::kNR);
            if (sj >= C::kNR) ok = mbar_wait(&cempty[r], (uint32_t)(((sj / C::kNR) - 1) & 1), a.flags, abort);
            if (ok) {
                if (warp == 0) note[r] = g;
                mbar_arrive(&cdone[r]);
            }
        }
        ++sj;
        return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    };
    for (int it = 0;; ++it) {
        const int s = it % C::kNS;
        if (!mbar_wait(&full[s], (it / C::kNS) & 1, a.flags, abort)) break;
        const Item ci = {(int)item[3 * s], item[3 * s + 1], item[3 * s + 2]};
        if (ci.kind == kItemEnd) {
            record(-1);
            break;
        }
        const float4* t4 = (const float4*)(smem + (size_t)s * C::kStage);
        const float4* qt = C::kFull ? t4 + (C::kSlotOff / 16) : nullptr;
        if (ci.kind == kItemA) {
            // first row of the tile: bits [kRowBits, loA) = g, bits of B = idx
            const int64_t base = ci.g * 8 + (ci.idx << (a.loB - kAmpShift));
            if constexpr (Arith::kLanes && C::kFull)
                tile_lanes<HA, Arith>((const float*)t4, (const float*)qt, (float*)a.slot, base * 4, rsA * 4, sc, a.sgn,
                                      need_a, pol_last);
            else
                tile<HA, Arith>(t4, qt, a.slot_in, a.slot, base, rsA, sc, a.sgn, need_a, pol_last);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (!record(ci.g)) break;
        } else {
            const int64_t base = (ci.g | (ci.idx << sha)) * 8;
            if constexpr (Arith::kLanes && C::kFull)
                tile_lanes<HB, Arith>((const float*)t4, (const float*)qt, (float*)a.slot, base * 4, rsB * 4, sc, 1.f, true,
                                      pol_first);
            else
                tile<HB, Arith>(t4, qt, a.slot, a.slot, base, rsB, sc, 1.f, true, pol_first);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
}

// Tensor map of a 128-byte-row strided view of a vector with `amp_bytes` per amplitude:
// (row: 32 floats) x (rows below the range: 2^(lo - rbits)) x (rows in the range: 2^H) x
// (rows above it), in boxes of box_rows rows.
inline cudaError_t encode_rows(const void* base, int n, int lo, int H, int rbits, int amp_bytes, int box_rows,
                               CUtensorMap* map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const int ab = amp_bytes == 16 ? 4 : 3;  // log2(amp_bytes)
    cuuint64_t dims[4] = {32, (cuuint64_t)1 << (lo - rbits), (cuuint64_t)1 << H, (cuuint64_t)1 << (n - lo - H)};
    cuuint64_t strides[3] = {128, (cuuint64_t)1 << (lo + ab), (cuuint64_t)1 << (lo + H + ab)};
    cuuint32_t box[4] = {32, 1, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <int HA, int HB, class Arith>
cudaError_t launch_t(const Args& a, int n, cudaStream_t s) {
    using C = Cfg<HA, HB>;
    constexpr int ab = Arith::kAmpShift == 1 ? 8 : 16;  // bytes per amplitude
    constexpr int rb = Arith::kRowBits;
    CUtensorMap mapA, mapB, smapA, qmapB;
    cudaError_t e = encode_rows(a.b1, n, a.loA, HA, rb, ab, HA < 8 ? (1 << HA) : 256, &mapA);
    if (e == cudaSuccess) e = encode_rows(a.slot_in, n, a.loA, HA, rb, ab, HA < 8 ? (1 << HA) : 256, &smapA);
    if (e == cudaSuccess) e = encode_rows(a.b1, n, a.loB, HB, rb, ab, HB < 8 ? (1 << HB) : 256, &mapB);
    if (e == cudaSuccess) e = encode_rows(a.slot, n, a.loB, HB, rb, ab, HB < 8 ? (1 << HB) : 256, &qmapB);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_pair<HA, HB, Arith>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    if (e != cudaSuccess) return e;
    note_launch(kKindPair);
    const int pi = prof_begin(kKindPair, s);
    k_pair<HA, HB, Arith><<<(unsigned)num_sms(), kThreads, C::kSmem, s>>>(a, mapA, mapB, smapA, qmapB);
    prof_end(pi, s);
    return cudaGetLastError();
}

// The range sizes of two-pass plans (the first pass takes the extra bit).
inline bool shape_ok(int HA, int HB) { return HA >= 6 && HA <= 9 && HB >= 6 && (HB == HA || HB == HA - 1); }

template <class Arith>
cudaError_t launch(int HA, int HB, const Args& a, int n, cudaStream_t s) {
    switch (HA * 16 + HB) {
        case 6 * 16 + 6: return launch_t<6, 6, Arith>(a, n, s);
        case 7 * 16 + 6: return launch_t<7, 6, Arith>(a, n, s);
        case 7 * 16 + 7: return launch_t<7, 7, Arith>(a, n, s);
        case 8 * 16 + 7: return launch_t<8, 7, Arith>(a, n, s);
        case 8 * 16 + 8: return launch_t<8, 8, Arith>(a, n, s);
        case 9 * 16 + 8: return launch_t<9, 8, Arith>(a, n, s);
        case 9 * 16 + 9: return launch_t<9, 9, Arith>(a, n, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pairk
}  // namespace cheb
