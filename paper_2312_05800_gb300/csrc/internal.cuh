// internal.cuh -- device-side mechanism layout and helpers shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "chemgb.h"

#define CHEMGB_STR2(x) #x
#define CHEMGB_STR(x) CHEMGB_STR2(x)

namespace chemgb {

constexpr double kR = 8.314462618;        // J/mol/K
constexpr int kMaxSpecies = 64;
constexpr int kMaxReactions = 4096;

// Device tables of one mechanism. Every pointer is device memory owned by the
// chem_mech handle. Square per-pair tables are stored row k, column j with a
// padded row length Np (a multiple of 4) so that rows start on 16 bytes.
template <typename real>
struct PropTables {
    const real *invW;      // [N] 1 / W_k
    const real *nasa_cp;   // [2][N][5] cp/R Horner coefficients, range 0 = low, 1 = high
    const real *nasa_h;    // [2][N][6] H/RT: a1, a2/2, a3/3, a4/4, a5/5, a6
    const real *visc;      // [N][5] ln mu_k polynomial in x = ln(T/1000)
    const real *wilke;     // [3][N][Np] T0 = c_kj, T1 = 2 c_kj w_jk, T2 = c_kj w_jk^2
    const real *diff;      // [N][Np][5]... stored as [5][N][Np]: coefficient n of g_jk at (k, j)
};

struct DevMech {
    int N, R, Np, n_tb;
    double P_std, T_mid;
    PropTables<float> f32;
    PropTables<double> f64;
    // FP64 kinetics
    const double *W;        // [N]
    const double *nasa;     // [2][N][7] raw NASA-7 rows (low, high)
    const int *rtype;       // [R]
    const int *reac;        // [R][3]
    const int *prod;        // [R][3]
    const double *lnA;      // [R]
    const double *beta;     // [R]
    const double *EaR;      // [R] Ea / R (K)
    const double *lnA0;     // [R]
    const double *beta0;    // [R]
    const double *Ea0R;     // [R]
    const double *troe;     // [R][4]
    const int *tb_row;      // [R] row in eff, or -1
    const double *eff;      // [n_tb][N]
    const int *inc_ptr;     // [N+1] species -> reactions incidence (CSR)
    const int2 *inc;        // (reaction, signed nu)
    const int *dnu;         // [R] sum of nu over the reaction
    // derived FP64 tables of the stiff integrator
    const double *nasa_s;   // [2][N][6] S/R: a1 (times ln T), a2, a3/2, a4/3, a5/4, a7
    const double *troe_r;   // [R][4] a, 1/T***, 1/T*, T**
    const int *rsp;         // [R][6] distinct species of reaction j (first-occurrence order), -1 pad
    const int *rnu;         // [R][6] their net stoichiometric coefficients
    const int *tb_list;     // [n_tb] reactions with a third body, ascending
    double lnPR;            // ln(P_std / R)
    unsigned int *counters; // [kNumCounters] work-queue counters (scratch) and error words
};

constexpr int kNumCounters = 8;
constexpr int kPropsErrCounter = 7;       // props_eval's staged thermo pass: a copy wait ran out

}  // namespace chemgb

struct chem_mech {
    int N, R, E, bath;
    double P_std, T_lo, T_mid, T_hi;
    chemgb::DevMech dev;
    void *blob;            // single device allocation holding every table
    size_t blob_bytes;
    int device;
};

namespace chemgb {
int set_error(int code, const std::string &msg);
// opt-in per-kernel timing (chem_prof_enable): events around tagged launches
bool prof_on();
void *prof_begin(cudaStream_t st);
void prof_end(void *begin, cudaStream_t st, const std::string &tag, double flops, double bytes);
int check_cuda(cudaError_t e, const char *what);
bool device_ok(std::string *why);
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Precision conversions by integer operations. On this part the FP64 pipe (which
// also converts between FP32 and FP64) runs at 1/64 of the FP32 rate, so the
// per-species conversions of the cell kernels are done on the integer pipe.
// FP64 -> FP32 by truncating the mantissa (relative error < 2^-23); magnitudes
// below 2^-126 become signed zero, at or above 2^128 infinity; NaN stays NaN.
// For |x| in range the FP32 bits are the double's high word with the exponent
// rebased (- (1023 - 127) << 20) and the 20 + 3 leading mantissa bits shifted
// into place, one funnel shift of the two words.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const unsigned int hi = static_cast<unsigned int>(__double2hiint(x));
    const unsigned int lo = static_cast<unsigned int>(__double2loint(x));
    const unsigned int a = hi & 0x7FFFFFFFu;
    unsigned int r = __funnelshift_l(lo, a - 0x38000000u, 3);      // exponent - 896, mantissa 23 bits
    r = (a < 0x38100000u) ? 0u : r;                                  // below 2^-126
    if (a >= 0x47F00000u)                                            // 2^128 and above, infinity, NaN
        r = (a > 0x7FF00000u || (a == 0x7FF00000u && lo != 0u)) ? 0x7FC00000u : 0x7F800000u;
    return __uint_as_float(r | (hi & 0x80000000u));
}
// FP32 -> FP64, exact for normal numbers and zero; FP32 subnormals (below 2^-126)
// become signed zero; infinities and NaN are kept.
__device__ __forceinline__ double f32_to_f64_int(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned long long sign = static_cast<unsigned long long>(b & 0x80000000u) << 32;
    const unsigned int e = (b >> 23) & 0xFFu;
    if (e == 0) return __longlong_as_double(static_cast<long long>(sign));
    const unsigned long long ed = (e == 0xFFu) ? 0x7FFull : static_cast<unsigned long long>(e) + 896ull;
    const unsigned long long mant = static_cast<unsigned long long>(b & 0x7FFFFFu) << 29;
    return __longlong_as_double(static_cast<long long>(sign | (ed << 52) | mant));
}
}  // namespace chemgb
