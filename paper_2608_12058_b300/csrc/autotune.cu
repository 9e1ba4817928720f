// Autotuner for the Clenshaw step configuration (no counterpart in the paper).
//
// The fastest way to run a Clenshaw step depends on n and the precision: the plain
// one-pass kernel or the fused passes, how the n bit flips are split between the
// shared-memory tile, L2 partner tiles and strided passes (Sec. II.D matvec), and for
// FP32 whether the last strided pass and the low pass run as one L2-blocked launch.
// The built-in choices come from a few measurements; cheb_autotune measures every
// candidate on the calling device instead (a few steps each on a synthetic problem of
// the same size, CUDA events on the caller's stream) and installs the fastest one
// process-wide. With CHEB_AUTOTUNE_CACHE set to a file name, results are appended to
// that file and entries recorded for the current device's name are applied the first
// time a call needs one (or by cheb_autotune_load).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/cheb_expmv.h"
#include "cheb_internal.h"
#include "fused.cuh"
#include "fused_ff.cuh"
#include "kernels.cuh"
#include "pipeline.h"

namespace cheb {
namespace {

struct Candidate {
    int path;  // CHEB_PATH_PLAIN or CHEB_PATH_FUSED
    int l, h;
    int blocking;
};

std::vector<Candidate> candidates(int n, int prec) {
    std::vector<Candidate> out;
    const int plain_max = prec == CHEB_FP32 ? 24 : 26;  // the plain kernel is far behind above
    if (n <= plain_max) out.push_back({CHEB_PATH_PLAIN, 0, 0, 0});
    if (prec == CHEB_FP32) {
        for (int l = 0; l <= 4 && 11 + l <= n; ++l) {
            const int h = n - 11 - l;
            if (!fused_split_valid(n, l, h)) continue;
            out.push_back({CHEB_PATH_FUSED, l, h, 0});
            FusedPlan p;
            fused_set_split(n, l, h);
            p = fused_plan(n, 0);
            if (fused_blocking_eligible(p)) out.push_back({CHEB_PATH_FUSED, l, h, 1});
            if (fused_pair_eligible(p)) out.push_back({CHEB_PATH_FUSED, l, h, 2});
        }
        fused_set_split(n, -1, 0);
    } else {
        for (int l = 0; l <= 5 && 10 + l <= n; ++l) {
            const int h = n - 10 - l;
            if (!ff_split_valid(n, l, h)) continue;
            out.push_back({CHEB_PATH_FUSED, l, h, 0});
            ff_set_split(n, l, h);
            if (ff_pair_eligible(ff_plan(n))) out.push_back({CHEB_PATH_FUSED, l, h, 2});
        }
        ff_set_split(n, -1, 0);
    }
    return out;
}

void apply(int prec, int n, const Candidate& c) {
    if (c.path == CHEB_PATH_FUSED) {
        if (prec == CHEB_FP32)
            fused_set_split(n, c.l, c.h);
        else
            ff_set_split(n, c.l, c.h);
    }
    tuned_set(prec, n, c.path, c.blocking);
}

std::string device_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s(prop.name);
    for (char& ch : s)
        if (ch == ' ') ch = '_';
    return s;
}

std::mutex g_tune_mu;
bool g_cache_loaded = false;

// Apply the entries of a cache file recorded for `device` (later lines win).
int load_file(const char* path, const std::string& device) {
    FILE* f = std::fopen(path, "r");
    if (!f) return -1;
    char line[512];
    int applied = 0;
    while (std::fgets(line, sizeof line, f)) {
        char dev[256];
        int prec, n, pathc, l, h, blk;
        double ms;
        if (std::sscanf(line, "cheb-tune-1 %255s %d %d %d %d %d %d %lf", dev, &prec, &n, &pathc, &l, &h, &blk,
                        &ms) != 8)
            continue;
        if (device != dev || (prec != 0 && prec != 1) || n < 11 || n > kMaxQubits) continue;
        if (pathc != CHEB_PATH_PLAIN && pathc != CHEB_PATH_FUSED) continue;
        if (pathc == CHEB_PATH_FUSED &&
            !(prec == 0 ? fused_split_valid(n, l, h) : ff_split_valid(n, l, h)))
            continue;
        apply(prec, n, {pathc, l, h, blk ? 1 : 0});
        ++applied;
    }
    std::fclose(f);
    return applied;
}

}  // namespace

// Applies the cache named by CHEB_AUTOTUNE_CACHE once per process (for the current device).
void autotune_cache_once() {
    static std::atomic<bool> done{false};
    if (done.load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    done.store(true, std::memory_order_release);
    const char* path = std::getenv("CHEB_AUTOTUNE_CACHE");
    if (path && *path) load_file(path, device_name());
}

}  // namespace cheb

using namespace cheb;

extern "C" size_t cheb_autotune_workspace_bytes(int n, cheb_precision_t precision) {
    const size_t base = cheb_workspace_bytes(n, precision);
    if (base == 0) return 0;
    const size_t vb = (((size_t)1 << n) * (precision == CHEB_FP32 ? 8 : 16) + 255) / 256 * 256;
    return base + vb;
}

extern "C" cheb_status_t cheb_autotune(int n, cheb_precision_t precision, int steps, void* workspace,
                                       size_t workspace_bytes, void* stream, cheb_tune_result_t* result) {
    if (precision != CHEB_FP32 && precision != CHEB_FP64) return CHEB_ERR_INVALID_ARG;
    if (n < (precision == CHEB_FP32 ? 14 : 13) || n > kMaxQubits || steps < 2 || steps > 64 || !result)
        return CHEB_ERR_INVALID_ARG;
    const size_t base = cheb_workspace_bytes(n, precision);
    if (!workspace || ((uintptr_t)workspace & 255) != 0 ||
        workspace_bytes < cheb_autotune_workspace_bytes(n, precision))
        return CHEB_ERR_WORKSPACE;
    autotune_cache_once();
    cudaStream_t s = (cudaStream_t)stream;
    Ctx C{n, precision, make_layout(n, precision), (unsigned char*)workspace, s};
    void* psi = (unsigned char*)workspace + base;
    const size_t vbytes = ((size_t)1 << n) * (precision == CHEB_FP32 ? 8 : 16);
    // a synthetic SK-like problem of this size (fixed seed): timing does not depend on values
    std::mt19937_64 rng(12345);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> h(n), J((size_t)n * n, 0.0);
    double l1 = 0.0;
    for (int i = 0; i < n; ++i) {
        h[i] = nd(rng);
        l1 += std::fabs(h[i]);
        for (int j = i + 1; j < n; ++j) {
            J[(size_t)i * n + j] = nd(rng) / std::sqrt((double)n);
            l1 += std::fabs(J[(size_t)i * n + j]);
        }
    }
    const double gamma = 1.0, radius = l1 + n;
    CUDA_TRY(cudaMemsetAsync(C.flags(), 0, sizeof(int), s));
    FixedOp F = make_fixed(n, h.data(), J.data(), 0.0, radius, precision == CHEB_FP32 ? kMaxQF32 : 62);
    cheb_status_t st = upload_tables(C, F);
    if (st != CHEB_OK) return st;
    std::vector<std::complex<double>> coef(steps + 1);
    for (auto& c : coef) c = std::complex<double>(nd(rng), nd(rng)) / (4.0 * steps);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CHEB_ERR_CUDA;
    }
    // the state: a fixed normal bit pattern (0x3c bytes), reset before every run
    auto run = [&](int path, float* ms) -> cheb_status_t {
        if (cudaMemsetAsync(psi, 0x3c, vbytes, s) != cudaSuccess) return CHEB_ERR_CUDA;
        if (cudaEventRecord(e0, s) != cudaSuccess) return CHEB_ERR_CUDA;
        cheb_status_t r = clenshaw_run(C, path, psi, coef, F.Q, gamma / radius);
        if (r != CHEB_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return CHEB_ERR_CUDA;
        return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess ? CHEB_OK : CHEB_ERR_CUDA;
    };
    // the built-in choice first (the reference), then every candidate
    tuned_set(precision, n, -1, -1);
    if (precision == CHEB_FP32)
        fused_set_split(n, -1, 0);
    else
        ff_set_split(n, -1, 0);
    float ms = 0.f;
    double default_ms = 0.0;
    st = run(CHEB_PATH_AUTO, &ms);
    if (st == CHEB_OK) st = run(CHEB_PATH_AUTO, &ms);
    default_ms = ms;
    const std::vector<Candidate> cand = candidates(n, precision);
    double best = 1e300;
    Candidate bestc{CHEB_PATH_PLAIN, 0, 0, 0};
    for (size_t i = 0; st == CHEB_OK && i < cand.size(); ++i) {
        apply(precision, n, cand[i]);
        st = run(cand[i].path, &ms);  // warm-up (tensor maps, function attributes)
        if (st == CHEB_OK) st = run(cand[i].path, &ms);
        if (st == CHEB_OK && ms < best) {
            best = ms;
            bestc = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == CHEB_OK) st = read_flags(C);
    if (st != CHEB_OK || cand.empty()) {
        tuned_set(precision, n, -1, -1);
        if (precision == CHEB_FP32)
            fused_set_split(n, -1, 0);
        else
            ff_set_split(n, -1, 0);
        return st != CHEB_OK ? st : CHEB_ERR_UNSUPPORTED;
    }
    apply(precision, n, bestc);
    result->path = bestc.path;
    result->l = bestc.l;
    result->h = bestc.h;
    result->blocking = bestc.blocking;
    result->candidates = (int)cand.size();
    result->best_ms_per_step = best / steps;
    result->default_ms_per_step = default_ms / steps;
    const char* path = std::getenv("CHEB_AUTOTUNE_CACHE");
    if (path && *path) {
        FILE* f = std::fopen(path, "a");
        if (f) {
            std::fprintf(f, "cheb-tune-1 %s %d %d %d %d %d %d %.6f\n", device_name().c_str(), (int)precision, n,
                         bestc.path, bestc.l, bestc.h, bestc.blocking, best / steps);
            std::fclose(f);
        }
    }
    return CHEB_OK;
}

extern "C" cheb_status_t cheb_autotune_load(const char* path, const char* device, int* applied) {
    if (!path) return CHEB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int a = load_file(path, device ? std::string(device) : device_name());
    if (a < 0) return CHEB_ERR_INVALID_ARG;
    if (applied) *applied = a;
    return CHEB_OK;
}

extern "C" cheb_status_t cheb_autotune_reset(void) {
    for (int n = 0; n <= kMaxQubits; ++n) {
        tuned_set(0, n, -1, -1);
        tuned_set(1, n, -1, -1);
        if (n >= 11) {
            fused_set_split(n, -1, 0);
            ff_set_split(n, -1, 0);
        }
    }
    return CHEB_OK;
}
