// Internal declarations shared by the host orchestration (api.cu), the kernels
// (kernels.cu, fused.cu) and the host coefficient generator (coeffs.cpp).
#pragma once
#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace cheb {

// ---- host coefficient generator (coeffs.cpp) ------------------------------
void bessel_jn(double a, int mmax, std::vector<double>& out);
double cf_correct_real(const std::vector<double>& a, int K, std::vector<double>& p);
// method: 0 Chebyshev, 1 CF. Returns K or -1 (K would exceed max_K).
double remez_real(bool odd, double a, int K, std::vector<double>& p);
void monomial_to_chebyshev(int K, const std::complex<double>* a, std::complex<double>* c);
int make_coefficients(double a, std::complex<double> phase, double tol, int method, int max_K,
                      std::vector<std::complex<double>>& c, double* err_bound);

// ---- constants ------------------------------------------------------------
constexpr int kMaxQubits = 33;        // 3 complex64 vectors of 2^33 fit in 270 GB
constexpr int kTileBits = 11;         // low bits of the per-tile energy decomposition
constexpr int kMaxK = 1 << 16;        // coefficient table length per time slice
constexpr int kSmallMaxF32 = 13;      // whole-vector-in-SMEM kernel limits
constexpr int kSmallMaxF64 = 12;
constexpr int kPlainMaxF32 = 19;      // AUTO uses the one-pass kernel up to this n (FP32)
constexpr int kFFAutoMinF64 = 17;     // AUTO uses the float-float fused step from this n (FP64)
constexpr int kFormatFF = 2;          // vector format code of float-float vectors (kernels)
constexpr int kRedBlocks = 1184;      // partial-sum slots for two-stage reductions (8 x 148)
// Largest fixed-point scale for the FP32 kernels: with |Dt| <= 1 the high 32-bit
// word of a 2^-56 fixed-point value fits a float mantissa exactly.
constexpr int kMaxQF32 = 56;

// Status word written by kernels (bit flags), read by the host after a sync.
enum DeviceFlag : int {
    kFlagTimeout = 1,
    kFlagNonFinite = 2,
    kFlagBadLaunch = 4,
};

// ---- workspace layout -----------------------------------------------------
struct Layout {
    int n = 0;
    int M = 0;              // tile bits (min(n, kTileBits))
    size_t cbytes = 0;      // bytes per complex element (8 or 16)
    size_t status = 0;      // int[64]
    size_t part = 0;        // 4 * kRedBlocks doubles / int64
    size_t jq = 0;          // int64 [n*n + n + 1]: J (symmetric), h, c
    size_t tiles = 0;       // int64 [2^(n-M) * (M+1)]: f_0..f_{M-1}, A
    size_t elow = 0;        // int64 [2^M]
    size_t coef = 0;        // double2 [kMaxK + 1]
    size_t b0 = 0, b1 = 0;  // Clenshaw vectors
    size_t total = 0;
};
Layout make_layout(int n, int precision);

}  // namespace cheb
