// cheb_expmv_batched: many independent instances psi_i <- exp(-i t_i H_i) psi_i,
// each with its own couplings, gamma_i, t_i and size n_i (the batching of
// Sec. III.A). Unlike the padding to the largest radius suggested there, every
// instance keeps its own spectral interval and polynomial.
//
//  1. Spectral bounds of all instances, one host synchronisation.
//  2. Host: centre, radius, fixed-point tables and coefficients per instance.
//  3. FP32: every instance runs in one persistent cooperative launch (batch_team.cu):
//     CTAs take work slots longest first, instances up to n = 12 whole in one CTA's
//     shared memory, larger ones on teams of CTAs with bounded team barriers.
//     FP64 (or with cheb_set_batch_persistent(0)): instances small enough for one
//     CTA's shared memory (n <= 13 FP32, <= 12 FP64) run in a single launch, one CTA
//     each; the next four sizes run whole on a thread-block cluster each (cluster.cu),
//     one launch per size. Larger instances run their Clenshaw step loops on a pool
//     of streams, longest first, joined back into the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>
#include <numeric>
#include <vector>

#include "batch_team.cuh"
#include "kernels.cuh"
#include "pipeline.h"

namespace cheb {
namespace {

constexpr int kPoolStreams = 8;
constexpr int kMaxDev = 64;

std::mutex g_pool_mu;
cudaStream_t g_pool[kMaxDev][kPoolStreams];
bool g_pool_ready[kMaxDev] = {};

cheb_status_t stream_pool(cudaStream_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return CHEB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready[dev]) {
        for (int i = 0; i < kPoolStreams; ++i)
            if (cudaStreamCreateWithFlags(&g_pool[dev][i], cudaStreamNonBlocking) != cudaSuccess) return CHEB_ERR_CUDA;
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return CHEB_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// FP32 batches run as one persistent launch (batch_team.cu) with one CTA per SM (1, the
// default), with two CTAs per SM (2), or as per-size launches (0).
int g_persistent = 1;

// An event destroyed when the call returns, on every path.
struct ScopedEvent {
    cudaEvent_t e = nullptr;
    ~ScopedEvent() {
        if (e) cudaEventDestroy(e);
    }
};

struct BatchLayout {
    size_t res_i64 = 0;   // 2 int64 per instance: energy bounds
    size_t res_f64 = 0;   // 2 double per instance: norm^2, energy
    size_t res_flag = 0;  // 1 int per instance
    size_t descs = 0;     // SmallDesc per instance
    size_t team = 0;      // TeamInst per instance (persistent launch)
    size_t bars = 0;      // team barrier counter per instance, then the slot counter
    std::vector<size_t> inst;
    size_t total = 0;
};

bool batch_layout(int B, const int* n, int prec, BatchLayout& L) {
    if (B < 1 || !n || (prec != CHEB_FP32 && prec != CHEB_FP64)) return false;
    size_t off = 256;
    L.res_i64 = off;
    off = align256(off + 2 * sizeof(int64_t) * (size_t)B);
    L.res_f64 = off;
    off = align256(off + 2 * sizeof(double) * (size_t)B);
    L.res_flag = off;
    off = align256(off + sizeof(int) * (size_t)B);
    L.descs = off;
    off = align256(off + sizeof(SmallDesc) * (size_t)B);
    L.team = off;
    off = align256(off + sizeof(TeamInst) * (size_t)B);
    L.bars = off;
    off = align256(off + sizeof(unsigned) * ((size_t)B + 1));
    L.inst.resize(B);
    for (int i = 0; i < B; ++i) {
        if (n[i] < 1 || n[i] > kMaxQubits) return false;
        L.inst[i] = off;
        off = align256(off + make_layout(n[i], prec).total);
    }
    L.total = off;
    return true;
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" cheb_status_t cheb_set_batch_persistent(int on) {
    if (on < 0 || on > 2) return CHEB_ERR_INVALID_ARG;
    g_persistent = on;
    return CHEB_OK;
}

extern "C" int cheb_get_batch_persistent(void) { return g_persistent; }

extern "C" size_t cheb_batched_workspace_bytes(int B, const int* n, cheb_precision_t precision) {
    BatchLayout L;
    return batch_layout(B, n, precision, L) ? L.total : 0;
}

extern "C" cheb_status_t cheb_expmv_batched(int B, const int* n, const int64_t* offsets, const double* h_cat,
                                            const double* J_cat, const double* gamma, const double* t,
                                            void* psi_cat, cheb_precision_t precision, double tol,
                                            cheb_method_t method, void* workspace, size_t ws_bytes, void* stream,
                                            cheb_info_t* infos) {
    BatchLayout BL;
    if (!batch_layout(B, n, precision, BL)) return CHEB_ERR_INVALID_ARG;
    if (!offsets || !h_cat || !J_cat || !gamma || !t || !psi_cat) return CHEB_ERR_INVALID_ARG;
    if (!(tol > 0) || !std::isfinite(tol)) return CHEB_ERR_INVALID_ARG;
    if (method != CHEB_METHOD_CHEBYSHEV && method != CHEB_METHOD_CF && method != CHEB_METHOD_REMEZ)
        return CHEB_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || ws_bytes < BL.total) return CHEB_ERR_WORKSPACE;
    const size_t cb = precision == CHEB_FP32 ? 8 : 16;
    std::vector<size_t> hoff(B), joff(B);
    {
        size_t ho = 0, jo = 0;
        for (int i = 0; i < B; ++i) {
            hoff[i] = ho;
            joff[i] = jo;
            ho += n[i];
            jo += (size_t)n[i] * n[i];
            if (offsets[i] < 0 || ((uintptr_t)psi_cat + (size_t)offsets[i] * cb) % 16 != 0) return CHEB_ERR_INVALID_ARG;
            if (!std::isfinite(gamma[i]) || !std::isfinite(t[i])) return CHEB_ERR_INVALID_ARG;
            if (!finite_all(h_cat + hoff[i], n[i]) || !finite_all(J_cat + joff[i], (size_t)n[i] * n[i]))
                return CHEB_ERR_INVALID_ARG;
        }
    }
    unsigned char* ws = (unsigned char*)workspace;
    cudaStream_t s0 = (cudaStream_t)stream;
    auto ctx = [&](int i, cudaStream_t s) { return Ctx{n[i], precision, make_layout(n[i], precision), ws + BL.inst[i], s}; };
    auto psi_i = [&](int i) { return (void*)((unsigned char*)psi_cat + (size_t)offsets[i] * cb); };

    // 1. bounds of every instance, one synchronisation
    std::vector<int> qb(B);
    for (int i = 0; i < B; ++i) {
        Ctx C = ctx(i, s0);
        CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s0));
        FixedOp F = make_fixed(n[i], h_cat + hoff[i], J_cat + joff[i], 0.0, 1.0);
        qb[i] = F.Q;
        cheb_status_t st = upload_tables(C, F);
        if (st != CHEB_OK) return st;
        launch_minmax(n[i], C.L.M, C.tiles(), C.elow(), (int64_t*)C.part(), C.i64out(), s0);
        CUDA_TRY(cudaMemcpyAsync(ws + BL.res_i64 + 16 * (size_t)i, C.i64out(), 16, cudaMemcpyDeviceToDevice, s0));
    }
    std::vector<int64_t> mm(2 * (size_t)B);
    CUDA_TRY(cudaMemcpyAsync(mm.data(), ws + BL.res_i64, 16 * (size_t)B, cudaMemcpyDeviceToHost, s0));
    CUDA_TRY(cudaStreamSynchronize(s0));

    // 2. per-instance operator tables and coefficients
    struct Inst {
        double emin, emax, c, r, g, err;
        int Q, K, slices;
        std::vector<std::complex<double>> coef;
        bool small;
        bool team = false;
    };
    std::vector<Inst> in(B);
    std::vector<SmallDesc> descs;
    int small_max_n = 0;
    const int small_lim = precision == CHEB_FP32 ? kSmallMaxF32 : kSmallMaxF64;
    // mid-size instances run whole on a thread-block cluster, grouped by size
    const int cl_sb = cluster_slice_bits(precision);
    const int cl_lim = cl_sb + 4;
    std::vector<std::vector<SmallDesc>> cdescs(cl_lim + 1);
    std::vector<std::vector<int>> cidx(cl_lim + 1);
    for (int i = 0; i < B; ++i) {
        Inst& x = in[i];
        x.emin = std::ldexp((double)mm[2 * i], -qb[i]);
        x.emax = std::ldexp((double)mm[2 * i + 1], -qb[i]);
        x.c = 0.5 * (x.emax + x.emin);
        x.r = 0.5 * (x.emax - x.emin) + std::fabs(gamma[i]) * n[i];
        if (!(x.r > 0)) x.r = 1.0;
        x.g = gamma[i] / x.r;
        FixedOp F = make_fixed(n[i], h_cat + hoff[i], J_cat + joff[i], x.c, x.r,
                               precision == CHEB_FP32 ? kMaxQF32 : 62);
        if (F.Q < 24) return CHEB_ERR_UNSUPPORTED;
        x.Q = F.Q;
        Ctx C = ctx(i, s0);
        cheb_status_t st = upload_tables(C, F);
        if (st != CHEB_OK) return st;
        st = slice_coefficients(t[i], x.c, x.r, tol, method, 0, x.coef, &x.K, &x.slices, &x.err);
        if (st != CHEB_OK) return st;
        if (g_persistent && precision == CHEB_FP32 && x.slices == 1 && x.K > 0) {
            // every instance goes into the persistent launch below
            CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.coef, x.coef.data(), x.coef.size() * sizeof(std::complex<double>),
                                     cudaMemcpyHostToDevice, s0));
            x.small = true;
            x.team = true;
            continue;
        }
        x.small = n[i] <= small_lim && x.slices == 1 && x.K > 0;
        const bool clus = !x.small && n[i] > cl_sb && n[i] <= cl_lim && x.slices == 1 && x.K > 0;
        if (x.small || clus) {
            CUDA_TRY(cudaMemcpyAsync(C.ws + C.L.coef, x.coef.data(), x.coef.size() * sizeof(std::complex<double>),
                                     cudaMemcpyHostToDevice, s0));
            SmallDesc d{};
            d.n = n[i];
            d.K = x.K;
            d.Q = x.Q;
            d.g = x.g;
            d.coef = (const double*)(C.ws + C.L.coef);
            d.tiles = C.tiles();
            d.elow = C.elow();
            d.psi = psi_i(i);
            if (x.small) {
                descs.push_back(d);
                small_max_n = std::max(small_max_n, n[i]);
            } else {
                cdescs[n[i]].push_back(d);
                cidx[n[i]].push_back(i);
                x.small = true;  // handled by its cluster launch (or taken back below)
            }
        } else if (x.K == 0) {
            for (int q = 0; q < x.slices; ++q)
                launch_scale(precision, (int64_t)1 << n[i], psi_i(i), psi_i(i), x.coef[0].real(), x.coef[0].imag(), s0);
            x.small = true;  // done
        }
    }
    // the stream pool forks here, so that the large instances overlap the small ones
    ScopedEvent fork_ev;
    CUDA_TRY(cudaEventCreateWithFlags(&fork_ev.e, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(fork_ev.e, s0));
    const cudaEvent_t fork = fork_ev.e;
    // 3. FP32: every instance in one persistent launch, longest first
    {
        std::vector<int> tl;
        for (int i = 0; i < B; ++i)
            if (in[i].team) tl.push_back(i);
        if (!tl.empty()) {
            std::stable_sort(tl.begin(), tl.end(), [&](int a, int b) {
                return std::ldexp((double)in[a].K, n[a]) > std::ldexp((double)in[b].K, n[b]);
            });
            std::vector<TeamInst> ti(tl.size());
            unsigned* bars = (unsigned*)(ws + BL.bars);
            int slots = 0;
            for (size_t q = 0; q < tl.size(); ++q) {
                const int i = tl[q];
                Ctx C = ctx(i, s0);
                TeamInst& d = ti[q];
                d.n = n[i];
                d.K = in[i].K;
                d.Q = in[i].Q;
                d.team = team_size(n[i], g_persistent == 2 ? 2 : 1);
                team_split(n[i], &d.l, &d.H);
                d.first_slot = slots;
                d.pad = 0;
                d.g = in[i].g;
                d.coef = (const double2*)(C.ws + C.L.coef);
                d.tiles = C.tiles();
                d.elow = C.elow();
                d.psi = (float4*)psi_i(i);
                d.v0 = (float4*)(C.ws + C.L.b0);
                d.v1 = (float4*)(C.ws + C.L.b1);
                d.bar = bars + q;
                slots += std::max(d.team, 1);
            }
            CUDA_TRY(cudaMemcpyAsync(ws + BL.team, ti.data(), ti.size() * sizeof(TeamInst), cudaMemcpyHostToDevice,
                                     s0));
            CUDA_TRY(cudaMemsetAsync(bars, 0, sizeof(unsigned) * ((size_t)B + 1), s0));
            // the status word of the first instance's workspace collects timeouts
            int* flags = ctx(tl[0], s0).flags();
            const cudaError_t e = launch_batch_team((const TeamInst*)(ws + BL.team), (int)ti.size(), slots, bars + B,
                                                    flags, g_persistent == 2 ? 2 : 1, s0);
            if (e != cudaSuccess) return CHEB_ERR_CUDA;
        }
    }
    // 3a. all small instances in one launch, mid-size ones in one cluster launch per size
    // (the descriptor region holds B entries: small ones first, then the clustered)
    size_t dpos = 0;
    if (!descs.empty()) {
        CUDA_TRY(cudaMemcpyAsync(ws + BL.descs, descs.data(), descs.size() * sizeof(SmallDesc), cudaMemcpyHostToDevice,
                                 s0));
        CUDA_TRY(launch_small_batched(precision, (int)descs.size(), small_max_n, (const SmallDesc*)(ws + BL.descs), s0));
        dpos = descs.size();
    }
    for (int nn = cl_sb + 1; nn <= cl_lim; ++nn) {
        if (cdescs[nn].empty()) continue;
        const SmallDesc* dd = (const SmallDesc*)(ws + BL.descs) + dpos;
        CUDA_TRY(cudaMemcpyAsync((void*)dd, cdescs[nn].data(), cdescs[nn].size() * sizeof(SmallDesc),
                                 cudaMemcpyHostToDevice, s0));
        dpos += cdescs[nn].size();
        const cudaError_t e = launch_cluster_batched(precision, nn, (int)cdescs[nn].size(), dd, s0);
        if (e == cudaErrorNotSupported) {
            (void)cudaGetLastError();
            for (int i : cidx[nn]) in[i].small = false;  // no room for such clusters: step kernels
        } else if (e != cudaSuccess) {
            return CHEB_ERR_CUDA;
        }
    }
    // 3b. larger instances on the stream pool, longest first onto the least loaded stream
    std::vector<int> big;
    for (int i = 0; i < B; ++i)
        if (!in[i].small) big.push_back(i);
    if (!big.empty()) {
        std::sort(big.begin(), big.end(), [&](int a, int b) {
            return std::ldexp((double)in[a].K * in[a].slices, n[a]) > std::ldexp((double)in[b].K * in[b].slices, n[b]);
        });
        cudaStream_t* pool = nullptr;
        cheb_status_t st = stream_pool(&pool);
        if (st != CHEB_OK) return st;
        double load[kPoolStreams] = {0};
        bool used[kPoolStreams] = {false};
        for (int i : big) {
            int j = (int)(std::min_element(load, load + kPoolStreams) - load);
            if (!used[j]) {
                CUDA_TRY(cudaStreamWaitEvent(pool[j], fork, 0));
                used[j] = true;
            }
            load[j] += std::ldexp((double)in[i].K * in[i].slices, n[i]);
            Ctx C = ctx(i, pool[j]);
            for (int q = 0; q < in[i].slices; ++q) {
                st = clenshaw_run(C, CHEB_PATH_AUTO, psi_i(i), in[i].coef, in[i].Q, in[i].g);
                if (st != CHEB_OK) return st;
            }
        }
        for (int j = 0; j < kPoolStreams; ++j) {
            if (!used[j]) continue;
            ScopedEvent join;
            CUDA_TRY(cudaEventCreateWithFlags(&join.e, cudaEventDisableTiming));
            CUDA_TRY(cudaEventRecord(join.e, pool[j]));
            CUDA_TRY(cudaStreamWaitEvent(s0, join.e, 0));
        }
    }
    // 4. per-instance results
    if (infos) {
        for (int i = 0; i < B; ++i) {
            Ctx C = ctx(i, s0);
            launch_norm_energy(precision, n[i], C.L.M, in[i].Q, C.tiles(), C.elow(), in[i].c, in[i].r, psi_i(i), C.part(),
                               C.f64out(), s0);
            CUDA_TRY(cudaMemcpyAsync(ws + BL.res_f64 + 16 * (size_t)i, C.f64out(), 16, cudaMemcpyDeviceToDevice, s0));
            CUDA_TRY(cudaMemcpyAsync(ws + BL.res_flag + 4 * (size_t)i, C.flags(), 4, cudaMemcpyDeviceToDevice, s0));
        }
        std::vector<double> ne(2 * (size_t)B);
        std::vector<int> fl(B);
        CUDA_TRY(cudaMemcpyAsync(ne.data(), ws + BL.res_f64, 16 * (size_t)B, cudaMemcpyDeviceToHost, s0));
        CUDA_TRY(cudaMemcpyAsync(fl.data(), ws + BL.res_flag, 4 * (size_t)B, cudaMemcpyDeviceToHost, s0));
        CUDA_TRY(cudaStreamSynchronize(s0));
        bool nonfinite = false;
        for (int i = 0; i < B; ++i) {
            if (fl[i] & kFlagTimeout) return CHEB_ERR_TIMEOUT;
            cheb_info_t& o = infos[i];
            o.K = in[i].K;
            o.time_splits = in[i].slices;
            o.matvecs = (int64_t)in[i].K * in[i].slices;
            o.emin = in[i].emin;
            o.emax = in[i].emax;
            o.center = in[i].c;
            o.radius = in[i].r;
            o.a = (t[i] / in[i].slices) * in[i].r;
            o.trunc_bound = in[i].err * in[i].slices;
            o.norm = std::sqrt(ne[2 * i]);
            o.energy = ne[2 * i + 1];
            o.eval_bound = -1.0;
            nonfinite |= !std::isfinite(ne[2 * i]) || !std::isfinite(ne[2 * i + 1]);
        }
        if (nonfinite) return CHEB_ERR_NONFINITE;
    }
    CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}
