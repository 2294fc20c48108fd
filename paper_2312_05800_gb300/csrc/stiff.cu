// stiff.cu -- chem_step_stiff: FP64 constant-pressure reactor integration over
// dt for every cell (Sec. 3.1: the compositions are integrated over dt = 1 us;
// Sec. 4.2: direct integration, "CPU-DI", is the plain method the network
// replaces).
//
// Design for sm_103a:
//  - One warp per cell. Cells are popped from a device work queue (one atomic
//    per cell), so cells with very different step counts balance across the
//    persistent grid (one block of kWarps warps per resident slot).
//  - Few cells (at most one per SM, e.g. the learned step's out-of-distribution
//    cells): a team of the block's kWarps warps integrates each cell. The FP64
//    pipe is per SM sub-partition, so a lone warp leaves three of them idle.
//    The team splits the reaction pass (reactions over all 128 lanes) and the
//    LU trailing updates (rows over warps); the rest runs redundantly in every
//    warp on identical data, and one warp writes the shared results. Every
//    value is computed by the same operations in the same order as by a lone
//    warp, so the results are bitwise those of one warp per cell.
//  - The state vector y = (T, Y_1..Y_N) is distributed over the lanes:
//    component c lives in lane c % 32, register slot c / 32 (N <= 63).
//  - Species work runs lane-per-species, reaction work lane-per-reaction; the
//    dense Jacobian and its LU factors (n x n FP64, n = N + 1) live in the
//    warp's shared-memory slice. The LU is right-looking with partial pivoting;
//    its rank-1 updates are column-parallel (each lane owns columns c % 32).
//  - Integrator: Rodas3 (Sandu et al. 1997), an embedded L-stable Rosenbrock
//    method of order 3(2), in the transformed form
//      (I/(h g) - J) K_i = f(y + sum_j a_ij K_j) + sum_j (c_ij / h) K_j,
//    y_new = y + sum_i m_i K_i, error estimate sum_i e_i K_i, with the
//    step-size controller of chem_ode_opts. Everything is FP64.
#include <math_constants.h>

#include <cmath>
#include <mutex>

#include "internal.cuh"

namespace chemgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;
constexpr size_t kSmemHeader = 16;   // the team's queue ticket, ahead of the warp slices
constexpr double kMixedMinRtol = 1e-5;   // tightest rtol the mixed mode integrates (below it: FP64)

// Rodas3 coefficients (g = 1/2 on the diagonal)
constexpr double kGam = 0.5;
constexpr double kA31 = 2.0, kA41 = 2.0, kA43 = 1.0;      // a21 = a32 = a42 = 0
constexpr double kC21 = 4.0, kC31 = 1.0, kC32 = -1.0, kC41 = 1.0, kC42 = -1.0, kC43 = -8.0 / 3.0;
// m = (2, 0, 1, 1), e = (0, 0, 0, 1)

__device__ __forceinline__ double warp_sum(double v) {
    // butterfly: every lane ends with the same bits (addition is commutative)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// The warps integrating one cell: W = 1 (a lone warp) or W = kWarps (the block).
template <int W>
struct Team {
    int wt;                    // rank of this warp in the team
    __device__ __forceinline__ void sync() const {
        if (W == 1) __syncwarp();
        else asm volatile("bar.sync 1, %0;" ::"n"(W * 32) : "memory");
    }
    __device__ __forceinline__ bool lead() const { return W == 1 || wt == 0; }
};

struct Slice {                 // one warp's shared-memory slice
    double *G;                 // [n][n] Jacobian, then its LU factors
    double *bsw;               // [n] permutation buffer
    double *invd;              // [n] reciprocal diagonal of U
    double *C, *HRT, *SR, *cpR, *wdot, *wT, *JCC, *U, *V;   // [N]
    double *rq, *rdqT, *rc3;   // [R] rate of progress, d q / dT, third-body coefficient
    double *rdq;               // [R][6] d q / d C_l for the reaction's distinct species
    int *piv;                  // [n]
};

__host__ __device__ inline size_t slice_doubles(int N, int R) {
    int n = N + 1;
    return (size_t)n * n + 2 * (size_t)n + 9 * (size_t)N + 9 * (size_t)R;
}
__host__ __device__ inline size_t slice_bytes(int N, int R) {
    size_t b = slice_doubles(N, R) * sizeof(double) + (size_t)(N + 1) * sizeof(int);
    return (b + 15) & ~size_t(15);
}

__device__ Slice make_slice(char *base, int N, int R) {
    Slice s;
    int n = N + 1;
    double *d = reinterpret_cast<double *>(base);
    s.G = d; d += (size_t)n * n;
    s.bsw = d; d += n;
    s.invd = d; d += n;
    s.C = d; d += N; s.HRT = d; d += N; s.SR = d; d += N; s.cpR = d; d += N; s.wdot = d; d += N;
    s.wT = d; d += N; s.JCC = d; d += N; s.U = d; d += N; s.V = d; d += N;
    s.rq = d; d += R; s.rdqT = d; d += R; s.rc3 = d; d += R;
    s.rdq = d; d += 6 * (size_t)R;
    s.piv = reinterpret_cast<int *>(d);
    return s;
}

// values of the last right-hand-side evaluation needed by the Jacobian
struct EvalInfo {
    double T, invT, rho, invrho, cp, dcpdT, Wbar, Q;
};

__device__ __forceinline__ double sel(const double v[2], int slot) { return slot ? v[1] : v[0]; }

// Troe blending function F(T, Pr) (Gilbert, Luther and Troe 1983), with
// glg = d log10 F / d log10 Pr and dF/dT at fixed Pr. tp = (a, 1/T***, 1/T*, T**).
__device__ void troe_F(const double *tp, double T, double invT, double Prd, double &F, double &glg,
                       double &dFdT_atPr) {
    const double a = __ldg(tp), r3 = __ldg(tp + 1), r1 = __ldg(tp + 2), T2 = __ldg(tp + 3);
    const double e3 = exp(-T * r3), e1 = exp(-T * r1), e2 = exp(-T2 * invT);
    const double Fc = (1.0 - a) * e3 + a * e1 + e2;
    const double dFc = -(1.0 - a) * r3 * e3 - a * r1 * e1 + T2 * invT * invT * e2;
    const double phi = log10(Fc);
    const double c = -0.4 - 0.67 * phi, nn = 0.75 - 1.27 * phi, d = 0.14;
    const double L = log10(Prd) + c;
    const double rden = 1.0 / (nn - d * L);
    const double f1 = L * rden;
    const double rq = 1.0 / (1.0 + f1 * f1);
    F = exp10(phi * rq);
    const double df1_dL = nn * rden * rden;
    glg = -phi * 2.0 * f1 * rq * rq * df1_dL;
    const double df1_dphi = (-0.67 * (nn - d * L) - L * (-1.27 + d * 0.67)) * rden * rden;
    const double dlgF_dphi = rq - phi * 2.0 * f1 * rq * rq * df1_dphi;
    const double dphi_dT = dFc / (Fc * 2.302585092994046);
    dFdT_atPr = F * 2.302585092994046 * dlgF_dphi * dphi_dT;
}

// The same blending in FP32 (the mixed mode): F, glg and dF/dT at fixed Pr to FP32 accuracy.
__device__ void troe_F_f32(const double *tp, float T, float invT, float Prd, float &F, float &glg, float &dFdT_atPr) {
    const float a = f64_to_f32_trunc(__ldg(tp)), r3 = f64_to_f32_trunc(__ldg(tp + 1));
    const float r1 = f64_to_f32_trunc(__ldg(tp + 2)), T2 = f64_to_f32_trunc(__ldg(tp + 3));
    const float e3 = expf(-T * r3), e1 = expf(-T * r1), e2 = expf(-T2 * invT);
    const float Fc = (1.0f - a) * e3 + a * e1 + e2;
    const float dFc = -(1.0f - a) * r3 * e3 - a * r1 * e1 + T2 * invT * invT * e2;
    const float phi = log10f(Fc);
    const float c = -0.4f - 0.67f * phi, nn = 0.75f - 1.27f * phi, d = 0.14f;
    const float L = log10f(Prd) + c;
    const float rden = 1.0f / (nn - d * L);
    const float f1 = L * rden;
    const float rq = 1.0f / (1.0f + f1 * f1);
    F = exp10f(phi * rq);
    const float df1_dL = nn * rden * rden;
    glg = -phi * 2.0f * f1 * rq * rq * df1_dL;
    const float df1_dphi = (-0.67f * (nn - d * L) - L * (-1.27f + d * 0.67f)) * rden * rden;
    const float dlgF_dphi = rq - phi * 2.0f * f1 * rq * rq * df1_dphi;
    const float dphi_dT = dFc / (Fc * 2.30258509f);
    dFdT_atPr = F * 2.30258509f * dlgF_dphi * dphi_dT;
}

// exp(x) for the mixed mode: the argument and the result cross between FP64 and FP32 on the
// integer pipe (truncation: relative error below 2^-23 of the argument), exp in FP32
__device__ __forceinline__ double exp_mx(double x) { return f32_to_f64_int(expf(f64_to_f32_trunc(x))); }

// f = f(y) for the warp's cell. With jac, also stores what build_matrix needs. MX (the mixed
// mode): the rate constants' exponentials and the fall-off blending in FP32, the rest FP64.
template <int W, bool MX>
__device__ EvalInfo eval_rhs(const DevMech &m, const Slice &sh, Team<W> tm, int lane, double p, const double y[2],
                             double f[2], bool jac) {
    const int N = m.N, R = m.R, n = N + 1;
    EvalInfo info;
    f[0] = 0.0;
    f[1] = 0.0;
    const double T = __shfl_sync(kFull, y[0], 0);
    const double invT = 1.0 / T;
    const double lnT = log(T);
    info.T = T;
    info.invT = invT;
    const int rng = (T >= m.T_mid) ? 1 : 0;
    tm.sync();                 // every warp of the team is done reading the previous evaluation
    // species pass: thermo and mixture sums (lane per species; in a team every warp
    // computes them and the first writes the shared copies)
    const bool wr = tm.lead();
    double S = 0.0, cp = 0.0, dcp = 0.0;
    double yw_s[2] = {0.0, 0.0};
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            const int k = c - 1;
            const double *a = m.f64.nasa_cp + (size_t)(rng * N + k) * 5;
            const double *b = m.f64.nasa_h + (size_t)(rng * N + k) * 6;
            const double *e = m.nasa_s + (size_t)(rng * N + k) * 6;
            const double a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3), a4 = __ldg(a + 4);
            const double cpR = a0 + T * (a1 + T * (a2 + T * (a3 + T * a4)));
            const double HRT = __ldg(b) + T * (__ldg(b + 1) + T * (__ldg(b + 2) + T * (__ldg(b + 3) + T * __ldg(b + 4))))
                               + __ldg(b + 5) * invT;
            const double SR = __ldg(e) * lnT + T * (__ldg(e + 1) + T * (__ldg(e + 2) + T * (__ldg(e + 3) + T * __ldg(e + 4))))
                              + __ldg(e + 5);
            const double yw = y[s] * __ldg(m.f64.invW + k);
            yw_s[s] = yw;
            S += yw;
            cp += yw * cpR;
            if (wr) {
                sh.HRT[k] = HRT;
                sh.SR[k] = SR;
                sh.cpR[k] = cpR;
            }
            if (jac) dcp += yw * (a1 + T * (2.0 * a2 + T * (3.0 * a3 + T * 4.0 * a4)));
        }
    }
    S = warp_sum(S);
    cp = warp_sum(cp) * kR;
    if (jac) dcp = warp_sum(dcp) * kR;
    const double Wbar = 1.0 / S;
    const double rho = p * invT * Wbar * (1.0 / kR);
    const double invrho = 1.0 / rho;
    info.rho = rho;
    info.invrho = invrho;
    info.cp = cp;
    info.dcpdT = dcp;
    info.Wbar = Wbar;
    // the mixed mode's FP32 concentrations for the third-body sums, in the space of V (written
    // only by the gather below, after the reaction pass has used them)
    float *Cf = reinterpret_cast<float *>(sh.V);
    if (wr)
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;
            if (c >= 1 && c < n) {
                sh.C[c - 1] = rho * yw_s[s];
                if (MX) Cf[c - 1] = f64_to_f32_trunc(rho * yw_s[s]);
            }
        }
    tm.sync();
    // reaction pass (thread per reaction over the team's lanes)
    const double lnPRT = m.lnPR - lnT;
    for (int j = tm.wt * 32 + lane; j < R; j += 32 * W) {
        const int *re = m.reac + 3 * j;
        const int *pr = m.prod + 3 * j;
        const int r0 = __ldg(re), r1 = __ldg(re + 1), r2 = __ldg(re + 2);
        const int p0 = __ldg(pr), p1 = __ldg(pr + 1), p2 = __ldg(pr + 2);
        const double beta = __ldg(m.beta + j), EaR = __ldg(m.EaR + j);
        const double lnkf = __ldg(m.lnA + j) + beta * lnT - EaR * invT;
        const double kf = MX ? exp_mx(lnkf) : exp(lnkf);
        double lnKp = 0.0, dH = 0.0;
        if (p0 >= 0) { lnKp += sh.SR[p0] - sh.HRT[p0]; dH += sh.HRT[p0]; }
        if (r0 >= 0) { lnKp -= sh.SR[r0] - sh.HRT[r0]; dH -= sh.HRT[r0]; }
        if (p1 >= 0) { lnKp += sh.SR[p1] - sh.HRT[p1]; dH += sh.HRT[p1]; }
        if (r1 >= 0) { lnKp -= sh.SR[r1] - sh.HRT[r1]; dH -= sh.HRT[r1]; }
        if (p2 >= 0) { lnKp += sh.SR[p2] - sh.HRT[p2]; dH += sh.HRT[p2]; }
        if (r2 >= 0) { lnKp -= sh.SR[r2] - sh.HRT[r2]; dH -= sh.HRT[r2]; }
        const double dnu = (double)__ldg(m.dnu + j);
        // k_r = k_f / K_c, ln K_c = ln K_p + dnu ln(P_std / RT)
        const double kr = MX ? exp_mx(lnkf - lnKp - dnu * lnPRT) : exp(lnkf - lnKp - dnu * lnPRT);
        double Pf = 1.0, Pr = 1.0;
        if (r0 >= 0) Pf *= sh.C[r0];
        if (r1 >= 0) Pf *= sh.C[r1];
        if (r2 >= 0) Pf *= sh.C[r2];
        if (p0 >= 0) Pr *= sh.C[p0];
        if (p1 >= 0) Pr *= sh.C[p1];
        if (p2 >= 0) Pr *= sh.C[p2];
        const int type = __ldg(m.rtype + j);
        const double dlnkf = (beta + EaR * invT) * invT;
        double F = 1.0, dFdC = 0.0, dFdT = 0.0;
        if (type != 0) {
            const double *e = m.eff + (size_t)__ldg(m.tb_row + j) * N;
            double M = 0.0;
            if (MX) {
                float Mf = 0.0f;
                for (int k = 0; k < N; ++k) Mf = fmaf(f64_to_f32_trunc(__ldg(e + k)), Cf[k], Mf);
                M = f32_to_f64_int(Mf);
            } else {
                for (int k = 0; k < N; ++k) M += __ldg(e + k) * sh.C[k];
            }
            if (type == 1) {
                F = M;
                dFdC = 1.0;
            } else {
                const double beta0 = __ldg(m.beta0 + j), Ea0R = __ldg(m.Ea0R + j);
                const double lr = __ldg(m.lnA0 + j) + beta0 * lnT - Ea0R * invT - lnkf;
                const double ratio = MX ? exp_mx(lr) : exp(lr);   // k0 / k_inf
                double Prd = M * ratio;
                if (Prd < 1e-300) Prd = 1e-300;
                double Ft, glg, dFtdT;
                if (MX) {
                    float Ff, gf, df;
                    troe_F_f32(m.troe_r + 4 * j, f64_to_f32_trunc(T), f64_to_f32_trunc(invT),
                               fmaxf(f64_to_f32_trunc(Prd), 1e-37f), Ff, gf, df);
                    Ft = f32_to_f64_int(Ff);
                    glg = f32_to_f64_int(gf);
                    dFtdT = f32_to_f64_int(df);
                } else {
                    troe_F(m.troe_r + 4 * j, T, invT, Prd, Ft, glg, dFtdT);
                }
                const double ip = 1.0 / (1.0 + Prd);
                const double blend = Prd * ip;
                const double dF_dPrd = Ft * ip * (ip + glg);
                F = blend * Ft;
                dFdC = dF_dPrd * ratio;
                const double dlnk0 = (beta0 + Ea0R * invT) * invT;
                dFdT = dF_dPrd * Prd * (dlnk0 - dlnkf) + blend * dFtdT;
            }
        }
        const double rop = kf * Pf - kr * Pr;
        sh.rq[j] = F * rop;
        if (jac) {
            const double dlnKc = (dH - dnu) * invT;
            const double dkfdT = kf * dlnkf;
            const double dkrdT = kr * (dlnkf - dlnKc);
            sh.rdqT[j] = F * (dkfdT * Pf - dkrdT * Pr) + rop * dFdT;
            sh.rc3[j] = (type != 0) ? rop * dFdC : 0.0;
            // d q / d C_l through the mass-action products, for the distinct species l
            for (int u = 0; u < 6; ++u) {
                const int l = __ldg(m.rsp + 6 * j + u);
                if (l < 0) break;
                double dPf = 0.0, dPr = 0.0;
                if (r0 == l) dPf += (r1 >= 0 ? sh.C[r1] : 1.0) * (r2 >= 0 ? sh.C[r2] : 1.0);
                if (r1 == l) dPf += (r0 >= 0 ? sh.C[r0] : 1.0) * (r2 >= 0 ? sh.C[r2] : 1.0);
                if (r2 == l) dPf += (r0 >= 0 ? sh.C[r0] : 1.0) * (r1 >= 0 ? sh.C[r1] : 1.0);
                if (p0 == l) dPr += (p1 >= 0 ? sh.C[p1] : 1.0) * (p2 >= 0 ? sh.C[p2] : 1.0);
                if (p1 == l) dPr += (p0 >= 0 ? sh.C[p0] : 1.0) * (p2 >= 0 ? sh.C[p2] : 1.0);
                if (p2 == l) dPr += (p0 >= 0 ? sh.C[p0] : 1.0) * (p1 >= 0 ? sh.C[p1] : 1.0);
                sh.rdq[6 * j + u] = F * (kf * dPf - kr * dPr);
            }
        }
    }
    tm.sync();
    // species gather: wdot_k = sum_j nu_kj q_j (reactions ascending)
    double Q = 0.0;
    const double RT = kR * T;
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            const int k = c - 1;
            double w = 0.0, wt = 0.0;
            const int b = __ldg(m.inc_ptr + k), e = __ldg(m.inc_ptr + k + 1);
            for (int t = b; t < e; ++t) {
                const int2 ent = __ldg(m.inc + t);
                w += (double)ent.y * sh.rq[ent.x];
                if (jac) wt += (double)ent.y * sh.rdqT[ent.x];
            }
            const double Wk = __ldg(m.W + k);
            if (jac && wr) {
                sh.wdot[k] = w;
                sh.wT[k] = wt;
                sh.U[k] = Wk * invrho;
                sh.V[k] = Wk * w * Wbar * invrho;
            }
            f[s] = Wk * w * invrho;
            Q += sh.HRT[k] * RT * w;
        }
    }
    Q = warp_sum(Q);
    info.Q = Q;
    if (lane == 0) f[0] = -Q / (rho * cp);
    return info;
}

// shared-memory FP64 value in the working type of the matrix assembly (FP32: by truncation on
// the integer pipe)
template <typename real>
__device__ __forceinline__ real rd(double x) {
    if constexpr (sizeof(real) == 4) return f64_to_f32_trunc(x);
    else return x;
}

// G = I/(h g) - J from the data of eval_rhs(..., jac = true), built by one warp into Gm (the FP64
// matrix sh.G, or in the mixed mode its FP32 counterpart in the same space: the Jacobian then
// carries FP32 rounding, about 1e-7 relative, which the mixed mode's loose tolerances absorb).
template <typename real>
__device__ void build_matrix_warp(const DevMech &m, const Slice &sh, real *G, int lane, const EvalInfo &in, double h) {
    const int N = m.N, n = N + 1;
    for (int s = 0; s < 2; ++s) {            // zero the species block (column owners)
        const int c = lane + 32 * s;
        if (c >= 1 && c < n)
            for (int r = 1; r < n; ++r) G[r * n + c] = 0;
    }
    __syncwarp();
    // sparse part of JC = d wdot / d C: row owners gather their reactions (ascending)
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            const int k = c - 1;
            real *row = G + (size_t)c * n + 1;
            const int b = __ldg(m.inc_ptr + k), e = __ldg(m.inc_ptr + k + 1);
            for (int t = b; t < e; ++t) {
                const int2 ent = __ldg(m.inc + t);
                const real nu = (real)ent.y;
                for (int u = 0; u < 6; ++u) {
                    const int l = __ldg(m.rsp + 6 * ent.x + u);
                    if (l < 0) break;
                    row[l] += nu * rd<real>(sh.rdq[6 * ent.x + u]);
                }
            }
        }
    }
    __syncwarp();
    // dense third-body part: rank-1 terms nu_j (rop dF/dM) eff_j (column owners)
    for (int t = 0; t < m.n_tb; ++t) {
        const int j = __ldg(m.tb_list + t);
        const real c3 = rd<real>(sh.rc3[j]);
        const double *e = m.eff + (size_t)__ldg(m.tb_row + j) * N;
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;
            if (c >= 1 && c < n) {
                const real v = c3 * rd<real>(__ldg(e + c - 1));
                for (int u = 0; u < 6; ++u) {
                    const int k = __ldg(m.rsp + 6 * j + u);
                    if (k < 0) break;
                    G[(1 + k) * n + c] += (real)__ldg(m.rnu + 6 * j + u) * v;
                }
            }
        }
    }
    __syncwarp();
    // JCC[k] = sum_l JC[k][l] C_l (row owners)
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            real acc = 0;
            for (int l = 0; l < N; ++l) acc += G[c * n + 1 + l] * rd<real>(sh.C[l]);
            sh.JCC[c - 1] = (double)acc;
        }
    }
    __syncwarp();
    // chain rule through C(T, Y) and rho(T, Y); then G = I/(h g) - J
    const real T = rd<real>(in.T), invT = rd<real>(in.invT), cp = rd<real>(in.cp), Wbar = rd<real>(in.Wbar);
    const real Q = rd<real>(in.Q), rho = rd<real>(in.rho), dcpdT = rd<real>(in.dcpdT);
    const real invrcp = (real)1 / (rho * cp);
    const real qq = Q * invrcp / cp;              // Q / (rho cp^2)
    const real Rr = (real)kR;
    const real RT = Rr * T;
    const real ghinv = rd<real>(1.0 / (h * kGam));
    real sT = 0;
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c < 1 || c >= n) continue;
        // species column c (column owner)
        const int mm = c - 1;
        const real iWm = rd<real>(__ldg(m.f64.invW + mm));
        const real a = rho * iWm, b = Wbar * iWm;
        real sTr = 0;
        for (int k = 0; k < N; ++k) {
            real *g = G + (size_t)(1 + k) * n + c;
            const real dw = *g * a - b * rd<real>(sh.JCC[k]);
            sTr += rd<real>(sh.HRT[k]) * RT * dw;
            const real J = rd<real>(sh.U[k]) * dw + rd<real>(sh.V[k]) * iWm;
            *g = (1 + k == c) ? ghinv - J : -J;
        }
        G[c] = sTr * invrcp + qq * (cp * Wbar - rd<real>(sh.cpR[mm]) * Rr) * iWm;   // -J[0][c]
        // temperature column entry of row c (row owner)
        const real dwdT = rd<real>(sh.wT[mm]) - rd<real>(sh.JCC[mm]) * invT;
        const real Um = rd<real>(sh.U[mm]), wm = rd<real>(sh.wdot[mm]);
        G[(size_t)c * n] = -(Um * dwdT + Um * wm * invT);
        sT += rd<real>(sh.cpR[mm]) * Rr * wm + rd<real>(sh.HRT[mm]) * RT * dwdT;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sT += __shfl_xor_sync(kFull, sT, o);
    if (lane == 0) G[0] = ghinv + sT * invrcp + qq * (cp * invT - dcpdT);
    __syncwarp();
}

template <int W, typename real>
__device__ void build_matrix(const DevMech &m, const Slice &sh, real *G, Team<W> tm, int lane, const EvalInfo &in,
                             double h) {
    if (tm.lead()) build_matrix_warp<real>(m, sh, G, lane, in, h);
    tm.sync();
}

// In-place LU with partial pivoting of G (FP64, or its FP32 copy in the mixed mode), the
// reciprocal pivots in invd and the pivot rows in sh.piv; false for a zero or non-finite pivot
// column. In a team every warp searches the pivot (same data, same choice), the first warp swaps
// and scales, and the trailing update splits the rows over the warps.
template <int W, typename real>
__device__ bool lu_factor(const Slice &sh, real *G, real *invd, Team<W> tm, int lane, int n) {
    for (int k = 0; k < n; ++k) {
        real best = -1;
        int bi = n;
        for (int s = 0; s < 2; ++s) {
            const int i = lane + 32 * s;
            if (i >= k && i < n) {
                const real v = fabs(G[i * n + k]);
                if (v > best || (v == best && i < bi)) { best = v; bi = i; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const real ob = __shfl_xor_sync(kFull, best, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0) || !(best < (real)INFINITY) || bi >= n) return false;
        if (tm.lead()) {
            if (lane == 0) sh.piv[k] = bi;
            if (bi != k) {
                for (int s = 0; s < 2; ++s) {
                    const int c = lane + 32 * s;
                    if (c < n) {
                        const real t = G[k * n + c];
                        G[k * n + c] = G[bi * n + c];
                        G[bi * n + c] = t;
                    }
                }
            }
        }
        tm.sync();
        const real rp = (real)1 / G[k * n + k];
        if (tm.lead()) {
            if (lane == 0) invd[k] = rp;
            for (int s = 0; s < 2; ++s) {
                const int i = lane + 32 * s;
                if (i > k && i < n) G[i * n + k] *= rp;
            }
        }
        tm.sync();
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;
            if (c > k && c < n) {
                const real akc = G[k * n + c];
                for (int i = k + 1 + tm.wt; i < n; i += W) G[i * n + c] -= G[i * n + k] * akc;
            }
        }
        tm.sync();
    }
    return true;
}

// b <- G^-1 b with the stored factors G, invd (FP64, or FP32 in the mixed mode); b is
// lane-distributed. bsw is this warp's own permutation buffer (every warp of a team solves on
// its own).
template <typename real>
__device__ void tri_solve(const Slice &sh, const real *G, const real *invd, real *bsw, int lane, int n, real b[2]) {
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c < n) bsw[c] = b[s];
    }
    __syncwarp();
    if (lane == 0) {
        for (int k = 0; k < n; ++k) {
            const int p = sh.piv[k];
            if (p != k) { const real t = bsw[k]; bsw[k] = bsw[p]; bsw[p] = t; }
        }
    }
    __syncwarp();
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        b[s] = (c < n) ? bsw[c] : (real)0;
    }
    for (int k = 0; k < n - 1; ++k) {
        const real bk = __shfl_sync(kFull, k >> 5 ? b[1] : b[0], k & 31);
        for (int s = 0; s < 2; ++s) {
            const int i = lane + 32 * s;
            if (i > k && i < n) b[s] -= G[i * n + k] * bk;
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        if ((k & 31) == lane) {
            if (k >> 5) b[1] *= invd[k];
            else b[0] *= invd[k];
        }
        const real bk = __shfl_sync(kFull, k >> 5 ? b[1] : b[0], k & 31);
        for (int s = 0; s < 2; ++s) {
            const int i = lane + 32 * s;
            if (i < k) b[s] -= G[i * n + k] * bk;
        }
    }
    __syncwarp();
}

// b <- G^-1 b with the FP64 factors (the default, FP64 mode)
__device__ __forceinline__ void lu_solve(const Slice &sh, double *bsw, int lane, int n, double b[2]) {
    tri_solve<double>(sh, sh.G, sh.invd, bsw, lane, n, b);
}

// The mixed mode's stage solve with the FP32 matrix Gc and its FP32 LU factors Gf (both in the
// space of the FP64 matrix: n^2 floats each): x = Gf^-1 b, then one step of iterative refinement,
// r = b - Gc x in FP64 arithmetic and x += Gf^-1 r. The correction solves the residual to FP32's
// relative accuracy, so the refined x carries about cond(G) 2^-24 times that error. The
// conversions between FP64 and FP32 run on the integer pipe (truncation; magnitudes below
// 2^-126 become 0).
__device__ void lu_solve_mixed(const Slice &sh, const float *Gf, const float *invdf, const float *Gc, double *bsw,
                               int lane, int n, double b[2]) {
    float v[2] = {f64_to_f32_trunc(b[0]), f64_to_f32_trunc(b[1])};
    tri_solve<float>(sh, Gf, invdf, reinterpret_cast<float *>(bsw), lane, n, v);
    const double x[2] = {f32_to_f64_int(v[0]), f32_to_f64_int(v[1])};
    __syncwarp();
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c < n) bsw[c] = x[s];
    }
    __syncwarp();
    double r[2] = {0.0, 0.0};
    for (int s = 0; s < 2; ++s) {
        const int c = lane + 32 * s;
        if (c < n) {
            const float *row = Gc + (size_t)c * n;
            double acc = b[s];
            for (int j = 0; j < n; ++j) acc = fma(-f32_to_f64_int(row[j]), bsw[j], acc);
            r[s] = acc;
        }
    }
    __syncwarp();
    float w[2] = {f64_to_f32_trunc(r[0]), f64_to_f32_trunc(r[1])};
    tri_solve<float>(sh, Gf, invdf, reinterpret_cast<float *>(bsw), lane, n, w);
    for (int s = 0; s < 2; ++s) b[s] = x[s] + f32_to_f64_int(w[s]);
}

// Integrates cells popped from the work queue until it is exhausted; W warps per cell. MX: the
// mixed mode (FP32 rate exponentials and fall-off blending; FP32 LU with one FP64 refinement).
template <int W, bool MX>
__device__ void integrate_cells(const DevMech &m, char *smem, int *blk_pos, int64_t limit, int64_t ld, double dt,
                                const chem_ode_opts &o, double *__restrict__ Tg, const double *__restrict__ pg,
                                double *__restrict__ Yg, int32_t *__restrict__ status,
                                int32_t *__restrict__ nsteps_out, unsigned int *__restrict__ queue,
                                const int32_t *__restrict__ list, int ok_status) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int N = m.N, n = N + 1;
    const size_t sb = slice_bytes(N, m.R);
    Team<W> tm{W == 1 ? 0 : warp};
    // the team's shared data live in its first warp's slice; every warp keeps its own permutation buffer
    Slice sh = make_slice(smem + (size_t)(W == 1 ? warp : 0) * sb, N, m.R);
    double *bsw = make_slice(smem + (size_t)warp * sb, N, m.R).bsw;
    for (;;) {
        unsigned int pos = 0;
        if (W == 1) {
            if (lane == 0) pos = atomicAdd(queue, 1u);
            pos = __shfl_sync(kFull, pos, 0);
        } else {
            if (tm.lead() && lane == 0) *blk_pos = (int)atomicAdd(queue, 1u);
            tm.sync();
            pos = (unsigned int)*blk_pos;
            // the next write of *blk_pos comes after this cell's evaluations, whose barriers
            // order it after every warp's read above
        }
        if ((int64_t)pos >= limit) break;
        const int64_t cell = list ? (int64_t)list[pos] : (int64_t)pos;
        double y[2], yn[2], f0[2], K1[2], K2[2], K3[2], K4[2], ys[2], fs[2];
        for (int s = 0; s < 2; ++s) {
            int c = lane + 32 * s;
            y[s] = (c == 0) ? Tg[cell] : (c < n ? Yg[(int64_t)(c - 1) * ld + cell] : 0.0);
        }
        const double p = pg[cell];
        double t = 0.0, h = (o.h0 < dt) ? o.h0 : dt;
        int nst = 0, rejected_last = 0, stat = CHEM_CELL_OK;
        while (t < dt) {
            if (nst >= o.max_steps) { stat = CHEM_CELL_MAXSTEPS; break; }
            if (h < 1e-20 * dt) { stat = CHEM_CELL_UNDERFLOW; break; }
            const double rem = dt - t;
            bool last = false;
            if (h >= rem) { h = rem; last = true; }
            EvalInfo info = eval_rhs<W, MX>(m, sh, tm, lane, p, y, f0, true);
            bool bad = false;
            for (int s = 0; s < 2; ++s)
                if (lane + 32 * s < n && !isfinite(f0[s])) bad = true;
            if (__any_sync(kFull, bad)) { stat = CHEM_CELL_NONFINITE; break; }
            // the mixed mode assembles an FP32 matrix Gc and factors its copy Gf, both in the space
            // of the FP64 matrix
            float *Gc = reinterpret_cast<float *>(sh.G);
            float *Gf = Gc + n * n;
            float *invdf = reinterpret_cast<float *>(sh.invd);
            bool factored;
            if (MX) {
                build_matrix<W, float>(m, sh, Gc, tm, lane, info, h);
                ++nst;
                if (tm.lead()) {
                    for (int s = 0; s < 2; ++s) {
                        const int c = lane + 32 * s;
                        if (c < n)
                            for (int r = 0; r < n; ++r) Gf[r * n + c] = Gc[r * n + c];
                    }
                }
                tm.sync();
                factored = lu_factor<W, float>(sh, Gf, invdf, tm, lane, n);
            } else {
                build_matrix<W, double>(m, sh, sh.G, tm, lane, info, h);
                ++nst;
                factored = lu_factor<W, double>(sh, sh.G, sh.invd, tm, lane, n);
            }
            if (!factored) { h *= 0.2; rejected_last = 1; continue; }
            auto solve = [&](double b[2]) {
                if (MX) lu_solve_mixed(sh, Gf, invdf, Gc, bsw, lane, n, b);
                else lu_solve(sh, bsw, lane, n, b);
            };
            const double ih = 1.0 / h;
            // stage 1
            for (int s = 0; s < 2; ++s) K1[s] = f0[s];
            solve(K1);
            // stage 2: the stage point is y itself (a21 = 0)
            for (int s = 0; s < 2; ++s) K2[s] = f0[s] + (kC21 * ih) * K1[s];
            solve(K2);
            // stage 3: y + 2 K1
            for (int s = 0; s < 2; ++s) ys[s] = y[s] + kA31 * K1[s];
            eval_rhs<W, MX>(m, sh, tm, lane, p, ys, fs, false);
            for (int s = 0; s < 2; ++s) {
                double v = fs[s];
                v += (kC31 * ih) * K1[s];
                v += (kC32 * ih) * K2[s];
                K3[s] = v;
            }
            solve(K3);
            // stage 4: y + 2 K1 + K3
            for (int s = 0; s < 2; ++s) ys[s] = y[s] + kA41 * K1[s] + kA43 * K3[s];
            eval_rhs<W, MX>(m, sh, tm, lane, p, ys, fs, false);
            for (int s = 0; s < 2; ++s) {
                double v = fs[s];
                v += (kC41 * ih) * K1[s];
                v += (kC42 * ih) * K2[s];
                v += (kC43 * ih) * K3[s];
                K4[s] = v;
            }
            solve(K4);
            // y_new = y + 2 K1 + K3 + K4, error = K4
            double acc = 0.0;
            bool nonfinite = false;
            for (int s = 0; s < 2; ++s) {
                int c = lane + 32 * s;
                if (c < n) {
                    double v = y[s];
                    v += 2.0 * K1[s];
                    v += K3[s];
                    v += K4[s];
                    yn[s] = v;
                    double e = K4[s];
                    double ay = fabs(y[s]), ayn = fabs(v);
                    double sc = ((c == 0) ? o.atol_T : o.atol_Y) + o.rtol * (ay > ayn ? ay : ayn);
                    double r = e / sc;
                    acc += r * r;
                    if (!isfinite(v) || !isfinite(e)) nonfinite = true;
                } else {
                    yn[s] = 0.0;
                }
            }
            acc = warp_sum(acc);
            nonfinite = __any_sync(kFull, nonfinite);
            double err = sqrt(acc / (double)n);
            double fac;
            if (nonfinite || !isfinite(err)) {
                fac = 0.2;
                err = 2.0;
            } else {
                fac = (err > 0.0) ? 0.9 * pow(err, -1.0 / 3.0) : 5.0;
                fac = fmin(5.0, fmax(0.2, fac));
            }
            if (err <= 1.0) {
                t = last ? dt : t + h;
                y[0] = yn[0];
                y[1] = yn[1];
                if (rejected_last && fac > 1.0) fac = 1.0;
                h *= fac;
                rejected_last = 0;
            } else {
                h *= fac;
                rejected_last = 1;
            }
        }
        if (tm.lead()) {
            for (int s = 0; s < 2; ++s) {
                int c = lane + 32 * s;
                if (c == 0) Tg[cell] = y[s];
                else if (c < n) Yg[(int64_t)(c - 1) * ld + cell] = y[s];
            }
            if (lane == 0) {
                status[cell] = (stat == CHEM_CELL_OK) ? ok_status : stat;
                if (nsteps_out) nsteps_out[cell] = nst;
            }
        }
    }
}

// Blocks that take a cell each in team mode: one per SM (the first blocks of a
// grid are spread over the SMs), at most the grid.
inline int team_blocks(int sms, int blocks) { return sms < blocks ? sms : blocks; }

// Cells 0..ncells-1, or (list != null) the *list_count cells list[0..) of a
// device-built queue; status of a successful cell = ok_status. When the cells
// number at most team_blocks, the first team_blocks blocks integrate them with
// all kWarps warps per cell and the other blocks return at once; otherwise
// every warp takes cells of its own.
__global__ void __launch_bounds__(kWarps * 32) stiff_kernel(DevMech m, int64_t ncells, int64_t ld, double dt,
                                                             chem_ode_opts o, double *__restrict__ Tg,
                                                             const double *__restrict__ pg, double *__restrict__ Yg,
                                                             int32_t *__restrict__ status,
                                                             int32_t *__restrict__ nsteps_out,
                                                             unsigned int *__restrict__ queue,
                                                             const int32_t *__restrict__ list,
                                                             const unsigned int *__restrict__ list_count,
                                                             int ok_status, int team_blocks) {
    extern __shared__ __align__(16) char smem_raw[];
    int *blk_pos = reinterpret_cast<int *>(smem_raw);
    char *smem = smem_raw + kSmemHeader;
    const int64_t limit = list ? (int64_t)(*list_count < (unsigned int)ncells ? *list_count : (unsigned int)ncells)
                               : ncells;
    // the mixed mode takes tolerances no tighter than kMixedMinRtol (its FP32 rates carry about
    // 1e-6 relative noise)
    const bool mx = o.mode == CHEM_ODE_MIXED && o.rtol >= kMixedMinRtol;
    if (limit <= (int64_t)team_blocks) {
        if ((int)blockIdx.x >= team_blocks) return;
        if (mx)
            integrate_cells<kWarps, true>(m, smem, blk_pos, limit, ld, dt, o, Tg, pg, Yg, status, nsteps_out, queue,
                                          list, ok_status);
        else
            integrate_cells<kWarps, false>(m, smem, blk_pos, limit, ld, dt, o, Tg, pg, Yg, status, nsteps_out, queue,
                                           list, ok_status);
    } else if (mx) {
        integrate_cells<1, true>(m, smem, blk_pos, limit, ld, dt, o, Tg, pg, Yg, status, nsteps_out, queue, list,
                                 ok_status);
    } else {
        integrate_cells<1, false>(m, smem, blk_pos, limit, ld, dt, o, Tg, pg, Yg, status, nsteps_out, queue, list,
                                  ok_status);
    }
}

// PaSR scaling (Sec. 4.1), one warp per cell. The species times Y_k / |dY_k/dt| come from the
// reactor right-hand side at the state before the step (the same FP64 evaluation as the
// integrator's); tau_c is the largest over the species with Y_k >= y_min and a non-zero rate
// (the slowest formation rate), +inf when none qualifies; tau_mix = sqrt(tau_T tau_K);
// kappa = tau_c / (tau_c + tau_mix), 1 for an infinite tau_c. With T, Y given (the chemistry
// step's result), they become T0 + kappa (T - T0), Y0 + kappa (Y - Y0).
__global__ void __launch_bounds__(kWarps * 32) pasr_kernel(DevMech m, int64_t ncells, int64_t ld, double y_min,
                                                            const double *__restrict__ T0,
                                                            const double *__restrict__ pg,
                                                            const double *__restrict__ Y0,
                                                            const double *__restrict__ tau_t,
                                                            const double *__restrict__ tau_k, double *__restrict__ T,
                                                            double *__restrict__ Y, double *__restrict__ tau_c_out,
                                                            double *__restrict__ kappa_out) {
    extern __shared__ __align__(16) char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = m.N, n = N + 1;
    const Slice sh = make_slice(smem_raw + (size_t)warp * slice_bytes(N, m.R), N, m.R);
    const Team<1> tm{0};
    for (int64_t cell = (int64_t)blockIdx.x * kWarps + warp; cell < ncells; cell += (int64_t)gridDim.x * kWarps) {
        double y[2], f[2];
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;
            y[s] = (c == 0) ? T0[cell] : (c < n ? Y0[(int64_t)(c - 1) * ld + cell] : 0.0);
        }
        eval_rhs<1, false>(m, sh, tm, lane, pg[cell], y, f, false);
        double tmax = -1.0;                       // species times are >= 0: -1 marks none
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;
            if (c >= 1 && c < n) {
                const double r = fabs(f[s]);
                if (y[s] >= y_min && r > 0.0) tmax = fmax(tmax, y[s] / r);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = fmax(tmax, __shfl_xor_sync(kFull, tmax, o));
        const double tau_c = (tmax >= 0.0) ? tmax : CUDART_INF;
        const double tau_mix = sqrt(tau_t[cell] * tau_k[cell]);
        const double kap = (tmax >= 0.0) ? tau_c / (tau_c + tau_mix) : 1.0;
        if (lane == 0) {
            if (tau_c_out) tau_c_out[cell] = tau_c;
            if (kappa_out) kappa_out[cell] = kap;
        }
        if (T && Y)
            for (int s = 0; s < 2; ++s) {
                const int c = lane + 32 * s;
                if (c == 0) T[cell] = y[s] + kap * (T[cell] - y[s]);
                else if (c < n) {
                    const int64_t q = (int64_t)(c - 1) * ld + cell;
                    Y[q] = y[s] + kap * (Y[q] - y[s]);
                }
            }
    }
}

}  // namespace
}  // namespace chemgb

using namespace chemgb;

extern "C" int chem_pasr(const chem_mech *m, int64_t ncells, int64_t ld, double y_min, const double *T0,
                         const double *p, const double *Y0, const double *tau_taylor, const double *tau_kolmogorov,
                         double *T, double *Y, double *tau_c, double *kappa, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_pasr: null mechanism");
    if (ncells < 0 || ld < ncells || (ld & 3) != 0 || ncells > (int64_t)0x7fffffff)
        return set_error(CHEM_EINVAL, "chem_pasr: need 0 <= ncells <= ld < 2^31, ld a multiple of 4");
    if (!(y_min > 0.0)) return set_error(CHEM_EINVAL, "chem_pasr: y_min must be positive");
    if (m->N > 63) return set_error(CHEM_EUNSUPPORTED, "chem_pasr: at most 63 species");
    if (ncells == 0) return CHEM_OK;
    if (!T0 || !p || !Y0 || !tau_taylor || !tau_kolmogorov) return set_error(CHEM_EINVAL, "chem_pasr: null input");
    if ((T == nullptr) != (Y == nullptr)) return set_error(CHEM_EINVAL, "chem_pasr: give both T and Y or neither");
    const void *ptrs[] = {T0, p, Y0, tau_taylor, tau_kolmogorov, T, Y, tau_c, kappa};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return set_error(CHEM_EINVAL, "chem_pasr: arrays must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_pasr: " + why);
    const size_t smem = slice_bytes(m->N, m->R) * kWarps;
    if (smem > 227 * 1024) return set_error(CHEM_EUNSUPPORTED, "chem_pasr: mechanism too large for shared memory");
    static size_t configured = 0;
    if (smem > configured) {
        int rc = check_cuda(cudaFuncSetAttribute(pasr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "chem_pasr: smem attribute");
        if (rc) return rc;
        configured = smem;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pasr_kernel, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t need = (ncells + kWarps - 1) / kWarps;
    const int blocks = (int)((int64_t)sms * per_sm < need ? (int64_t)sms * per_sm : need);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *pb = prof_begin(st);
    pasr_kernel<<<blocks, kWarps * 32, smem, st>>>(m->dev, ncells, ld, y_min, T0, p, Y0, tau_taylor, tau_kolmogorov,
                                                   T, Y, tau_c, kappa);
    prof_end(pb, st, "pasr_kernel", 0.0, (double)ncells * ((m->N + 2) * 8 + 2 * 8 + (T ? 2 * (m->N + 1) * 8 : 0)));
    return check_cuda(cudaGetLastError(), "chem_pasr launch");
}

extern "C" int chem_step_stiff(const chem_mech *m, int64_t ncells, int64_t ld, double dt, const chem_ode_opts *opts,
                               double *T, const double *p, double *Y, int32_t *status, int32_t *nsteps,
                               chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_step_stiff: null mechanism");
    if (ncells < 0 || ld < ncells || (ld & 3) != 0 || ncells > (int64_t)0x7fffffff)
        return set_error(CHEM_EINVAL, "chem_step_stiff: need 0 <= ncells <= ld < 2^31, ld a multiple of 4");
    if (!(dt > 0.0)) return set_error(CHEM_EINVAL, "chem_step_stiff: dt must be positive");
    if (m->N > 63) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff: at most 63 species");
    if (ncells == 0) return CHEM_OK;
    if (!T || !p || !Y || !status) return set_error(CHEM_EINVAL, "chem_step_stiff: null array");
    const void *ptrs[] = {T, p, Y, status, nsteps};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return set_error(CHEM_EINVAL, "chem_step_stiff: arrays must be 16-byte aligned");
    chem_ode_opts o;
    chem_ode_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || !(o.atol_Y > 0.0) || !(o.atol_T > 0.0) || !(o.h0 > 0.0) || o.max_steps < 1)
        return set_error(CHEM_EINVAL, "chem_step_stiff: tolerances, h0 and max_steps must be positive");
    if (o.mode != CHEM_ODE_FP64 && o.mode != CHEM_ODE_MIXED)
        return set_error(CHEM_EINVAL, "chem_step_stiff: mode must be CHEM_ODE_FP64 or CHEM_ODE_MIXED");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff: " + why);
    size_t per_warp = slice_bytes(m->N, m->R);
    size_t smem = kSmemHeader + per_warp * kWarps;
    if (smem > 227 * 1024) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff: mechanism too large for shared memory");
    static size_t configured = 0;
    if (smem > configured) {
        int rc = check_cuda(cudaFuncSetAttribute(stiff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "chem_step_stiff: smem attribute");
        if (rc) return rc;
        configured = smem;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stiff_kernel, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t need = (ncells + kWarps - 1) / kWarps;
    int blocks = (int)((int64_t)sms * per_sm < need ? (int64_t)sms * per_sm : need);
    if (ncells <= sms) blocks = (int)ncells;      // one block (a team of warps) per cell
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned int *queue = m->dev.counters;
    int rc = check_cuda(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st), "chem_step_stiff: queue reset");
    if (rc) return rc;
    void *pb = prof_begin(st);
    stiff_kernel<<<blocks, kWarps * 32, smem, st>>>(m->dev, ncells, ld, dt, o, T, p, Y, status, nsteps, queue, nullptr,
                                                    nullptr, CHEM_CELL_OK, team_blocks(sms, blocks));
    prof_end(pb, st, "stiff_kernel", 0.0, 0.0);
    return check_cuda(cudaGetLastError(), "chem_step_stiff launch");
}

namespace chemgb {
// Stiff integration of the cells a device queue lists (the fallback of the
// learned step): list[0..*count) with count <= capacity, status ok_status on
// success. Uses the mechanism's second work-queue counter.
int launch_stiff_list(const chem_mech *m, int64_t capacity, int64_t ld, double dt, const chem_ode_opts &o, double *T,
                      const double *p, double *Y, int32_t *status, const int32_t *list, const unsigned int *count,
                      int ok_status, cudaStream_t st) {
    if (m->N > 63) return set_error(CHEM_EUNSUPPORTED, "fallback: at most 63 species");
    size_t smem = kSmemHeader + slice_bytes(m->N, m->R) * kWarps;
    if (smem > 227 * 1024) return set_error(CHEM_EUNSUPPORTED, "fallback: mechanism too large for shared memory");
    int rc = check_cuda(cudaFuncSetAttribute(stiff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "fallback: smem attribute");
    if (rc) return rc;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stiff_kernel, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t need = (capacity + kWarps - 1) / kWarps;
    int blocks = (int)((int64_t)sms * per_sm < need ? (int64_t)sms * per_sm : need);
    if (blocks < 1) blocks = 1;
    unsigned int *queue = m->dev.counters + 1;
    rc = check_cuda(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st), "fallback: queue reset");
    if (rc) return rc;
    stiff_kernel<<<blocks, kWarps * 32, smem, st>>>(m->dev, capacity, ld, dt, o, T, p, Y, status, nullptr, queue, list,
                                                    count, ok_status, team_blocks(sms, blocks));
    return check_cuda(cudaGetLastError(), "fallback launch");
}
}  // namespace chemgb

// ---------------------------------------------------------------------------
// Allocation-free variant of chem_step_stiff.
//
// The regular entry point keeps its only global scratch (the work-queue
// counter) inside the mechanism handle. This variant keeps it in the
// file-scope array below instead, so a call neither allocates device memory
// nor writes into the handle. The array is 256 bytes (64 32-bit words) and
// every GPU that loads the library holds it until the process exits. A call
// uses word 0 as its queue counter and clears it first on its stream; calls
// that overlap on the GPU share that word and race.
// ---------------------------------------------------------------------------
namespace chemgb {
namespace {

constexpr int kNoAllocWords = 64;
// Largest ncells one call accepts: every resident warp takes one ticket past
// the last cell, so the 32-bit counter needs headroom below 2^32.
constexpr int64_t kNoAllocMaxCells = (int64_t)1 << 30;

static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocWords];

// Device address of g_noalloc_scratch for the current device, looked up once
// per device (with that device current). In host code the array's name is only
// a host-side stand-in, so kernels must be given this address.
int noalloc_scratch(unsigned int **out) {
    static std::mutex mu;
    static unsigned int *addr[64] = {nullptr};
    int dev = -1;
    int rc = check_cuda(cudaGetDevice(&dev), "chem_step_stiff_noalloc: cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= 64) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "chem_step_stiff_noalloc: cudaGetSymbolAddress");
        if (rc) return rc;
        addr[dev] = static_cast<unsigned int *>(p);
    }
    *out = addr[dev];
    return CHEM_OK;
}

}  // namespace
}  // namespace chemgb

extern "C" int chem_step_stiff_noalloc(const chem_mech *m, int64_t ncells, int64_t ld, double dt,
                                       const chem_ode_opts *opts, double *T, const double *p, double *Y,
                                       int32_t *status, int32_t *nsteps, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: null mechanism");
    if (ncells < 0 || ld < ncells || (ld & 3) != 0)
        return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: need 0 <= ncells <= ld, ld a multiple of 4");
    if (ncells > kNoAllocMaxCells)
        return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: ncells exceeds the 2^30-cell limit of its static "
                                      "work-queue scratch");
    if (!(dt > 0.0)) return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: dt must be positive");
    if (m->N > 63) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff_noalloc: at most 63 species");
    if (ncells == 0) return CHEM_OK;
    if (!T || !p || !Y || !status) return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: null array");
    const void *ptrs[] = {T, p, Y, status, nsteps};
    for (const void *q : ptrs)
        if (q && !aligned16(q))
            return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: arrays must be 16-byte aligned");
    chem_ode_opts o;
    chem_ode_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.rtol > 0.0) || !(o.atol_Y > 0.0) || !(o.atol_T > 0.0) || !(o.h0 > 0.0) || o.max_steps < 1)
        return set_error(CHEM_EINVAL, "chem_step_stiff_noalloc: tolerances, h0 and max_steps must be positive");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff_noalloc: " + why);
    unsigned int *queue = nullptr;
    int rc = noalloc_scratch(&queue);
    if (rc) return rc;
    size_t smem = kSmemHeader + slice_bytes(m->N, m->R) * kWarps;
    if (smem > 227 * 1024)
        return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff_noalloc: mechanism too large for shared memory");
    rc = check_cuda(cudaFuncSetAttribute(stiff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "chem_step_stiff_noalloc: smem attribute");
    if (rc) return rc;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stiff_kernel, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t need = (ncells + kWarps - 1) / kWarps;
    int blocks = (int)((int64_t)sms * per_sm < need ? (int64_t)sms * per_sm : need);
    if (ncells <= sms) blocks = (int)ncells;      // one block (a team of warps) per cell
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rc = check_cuda(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st), "chem_step_stiff_noalloc: clear queue");
    if (rc) return rc;
    stiff_kernel<<<blocks, kWarps * 32, smem, st>>>(m->dev, ncells, ld, dt, o, T, p, Y, status, nsteps, queue, nullptr,
                                                    nullptr, CHEM_CELL_OK, team_blocks(sms, blocks));
    return check_cuda(cudaGetLastError(), "chem_step_stiff_noalloc launch");
}
