// stiff.cu -- chem_step_stiff: FP64 constant-pressure reactor integration over
// dt for every cell (Sec. 3.1: the compositions are integrated over dt = 1 us;
// Sec. 4.2: direct integration, "CPU-DI", is the plain method the network
// replaces).
//
// Design for sm_103a:
//  - One warp per cell. Cells are popped from a device work queue (one atomic
//    per cell), so cells with very different step counts balance across the
//    persistent grid (one block of kWarps warps per resident slot).
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
#include <cmath>

#include "internal.cuh"

namespace chemgb {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;

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

struct Slice {                 // one warp's shared-memory slice
    double *G;                 // [n][n] Jacobian / LU
    double *bsw;               // [n] permutation buffer
    double *C, *HRT, *SR, *cpR, *dcpR, *wdot, *wT, *JCC;   // [N]
    double *rF, *rkf, *rkr, *rrop, *rdFdC, *rq, *rdqT;      // [R]
    int *piv;                  // [n]
};

__host__ __device__ inline size_t slice_doubles(int N, int R) {
    int n = N + 1;
    return (size_t)n * n + n + 8 * (size_t)N + 7 * (size_t)R;
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
    s.C = d; d += N; s.HRT = d; d += N; s.SR = d; d += N; s.cpR = d; d += N;
    s.dcpR = d; d += N; s.wdot = d; d += N; s.wT = d; d += N; s.JCC = d; d += N;
    s.rF = d; d += R; s.rkf = d; d += R; s.rkr = d; d += R; s.rrop = d; d += R;
    s.rdFdC = d; d += R; s.rq = d; d += R; s.rdqT = d; d += R;
    s.piv = reinterpret_cast<int *>(d);
    return s;
}

// values of the last right-hand-side evaluation needed by the Jacobian
struct EvalInfo {
    double T, rho, cp, dcpdT, Wbar, Q;
};

__device__ __forceinline__ double sel(const double v[2], int slot) { return slot ? v[1] : v[0]; }

// Troe blending function with the derivatives used by the Jacobian
__device__ void troe_F(const double *tp, double T, double Prd, double &F, double &glg, double &dFdT_atPr) {
    double a = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
    double e3 = exp(-T / T3), e1 = exp(-T / T1), e2 = exp(-T2 / T);
    double Fc = (1.0 - a) * e3 + a * e1 + e2;
    double dFc = -(1.0 - a) / T3 * e3 - a / T1 * e1 + T2 / (T * T) * e2;
    double phi = log10(Fc);
    double c = -0.4 - 0.67 * phi, nn = 0.75 - 1.27 * phi, d = 0.14;
    double L = log10(Prd) + c;
    double den = nn - d * L;
    double f1 = L / den;
    double q = 1.0 + f1 * f1;
    double lgF = phi / q;
    F = exp10(lgF);
    double df1_dL = nn / (den * den);
    glg = -phi * 2.0 * f1 / (q * q) * df1_dL;
    double df1_dphi = (-0.67 * den - L * (-1.27 - d * -0.67)) / (den * den);
    double dlgF_dphi = 1.0 / q - phi * 2.0 * f1 / (q * q) * df1_dphi;
    double dphi_dT = dFc / (Fc * 2.302585092994046);
    dFdT_atPr = F * 2.302585092994046 * dlgF_dphi * dphi_dT;
}

// f = f(y) for the warp's cell; with jac, also stores what the Jacobian needs.
__device__ EvalInfo eval_rhs(const DevMech &m, const Slice &sh, int lane, double p, const double y[2], double f[2],
                             bool jac) {
    const int N = m.N, R = m.R, n = N + 1;
    EvalInfo info;
    f[0] = 0.0;
    f[1] = 0.0;
    const double T = __shfl_sync(kFull, y[0], 0);
    info.T = T;
    const int rng = (T >= m.T_mid) ? 1 : 0;
    const double lnT = log(T);
    __syncwarp();
    // species pass: thermo, mixture sums
    double S = 0.0, cp = 0.0, dcp = 0.0;
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            int k = c - 1;
            const double *a = m.nasa + (size_t)(rng * N + k) * 7;
            double a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3), a4 = __ldg(a + 4),
                   a5 = __ldg(a + 5), a6 = __ldg(a + 6);
            double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
            double cpR = a0 + a1 * T + a2 * T2 + a3 * T3 + a4 * T4;
            double HRT = a0 + a1 * T / 2.0 + a2 * T2 / 3.0 + a3 * T3 / 4.0 + a4 * T4 / 5.0 + a5 / T;
            double SR = a0 * lnT + a1 * T + a2 * T2 / 2.0 + a3 * T3 / 3.0 + a4 * T4 / 4.0 + a6;
            double Yk = y[s];
            double W = __ldg(m.W + k);
            S += Yk / W;
            cp += Yk * cpR * kR / W;
            sh.HRT[k] = HRT;
            sh.SR[k] = SR;
            sh.cpR[k] = cpR;
            if (jac) {
                double dcpR = a1 + 2.0 * a2 * T + 3.0 * a3 * T2 + 4.0 * a4 * T3;
                sh.dcpR[k] = dcpR;
                dcp += Yk * dcpR * kR / W;
            }
        }
    }
    S = warp_sum(S);
    cp = warp_sum(cp);
    if (jac) dcp = warp_sum(dcp);
    const double rho = p / (kR * T * S);
    info.rho = rho;
    info.cp = cp;
    info.dcpdT = dcp;
    info.Wbar = 1.0 / S;
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= 1 && c < n) sh.C[c - 1] = rho * y[s] / __ldg(m.W + c - 1);
    }
    __syncwarp();
    // reaction pass: lane per reaction
    const double RT = kR * T;
    const double PRT = m.P_std / RT;
    for (int j = lane; j < R; j += 32) {
        const int *re = m.reac + 3 * j;
        const int *pr = m.prod + 3 * j;
        int r0 = __ldg(re), r1 = __ldg(re + 1), r2 = __ldg(re + 2);
        int p0 = __ldg(pr), p1 = __ldg(pr + 1), p2 = __ldg(pr + 2);
        double kf = exp(__ldg(m.lnA + j) + __ldg(m.beta + j) * lnT - __ldg(m.EaR + j) / T);
        double lnKp = 0.0, dH = 0.0;
        int dnu = 0;
        if (p0 >= 0) { lnKp += sh.SR[p0] - sh.HRT[p0]; dH += sh.HRT[p0] / T; ++dnu; }
        if (r0 >= 0) { lnKp -= sh.SR[r0] - sh.HRT[r0]; dH -= sh.HRT[r0] / T; --dnu; }
        if (p1 >= 0) { lnKp += sh.SR[p1] - sh.HRT[p1]; dH += sh.HRT[p1] / T; ++dnu; }
        if (r1 >= 0) { lnKp -= sh.SR[r1] - sh.HRT[r1]; dH -= sh.HRT[r1] / T; --dnu; }
        if (p2 >= 0) { lnKp += sh.SR[p2] - sh.HRT[p2]; dH += sh.HRT[p2] / T; ++dnu; }
        if (r2 >= 0) { lnKp -= sh.SR[r2] - sh.HRT[r2]; dH -= sh.HRT[r2] / T; --dnu; }
        double pw = (dnu == 0) ? 1.0 : (dnu == 1 ? PRT : (dnu == -1 ? 1.0 / PRT : pow(PRT, (double)dnu)));
        double Kc = exp(lnKp) * pw;
        double kr = kf / Kc;
        double Pf = 1.0, Pr = 1.0;
        if (r0 >= 0) Pf *= sh.C[r0];
        if (r1 >= 0) Pf *= sh.C[r1];
        if (r2 >= 0) Pf *= sh.C[r2];
        if (p0 >= 0) Pr *= sh.C[p0];
        if (p1 >= 0) Pr *= sh.C[p1];
        if (p2 >= 0) Pr *= sh.C[p2];
        const int type = __ldg(m.rtype + j);
        double F = 1.0, dFdC = 0.0, dFdT = 0.0;
        double dlnkf = __ldg(m.beta + j) / T + __ldg(m.EaR + j) / (T * T);
        if (type != 0) {
            const double *e = m.eff + (size_t)__ldg(m.tb_row + j) * N;
            double M = 0.0;
            for (int k = 0; k < N; ++k) M += __ldg(e + k) * sh.C[k];
            if (type == 1) {
                F = M; dFdC = 1.0;
            } else {
                double k0 = exp(__ldg(m.lnA0 + j) + __ldg(m.beta0 + j) * lnT - __ldg(m.Ea0R + j) / T);
                double dlnk0 = __ldg(m.beta0 + j) / T + __ldg(m.Ea0R + j) / (T * T);
                double Prd = k0 * M / kf;
                if (Prd < 1e-300) Prd = 1e-300;
                double Ft, glg, dFtdT;
                troe_F(m.troe + 4 * j, T, Prd, Ft, glg, dFtdT);
                double blend = Prd / (1.0 + Prd);
                double dF_dPrd = Ft / ((1.0 + Prd) * (1.0 + Prd)) + blend * Ft * glg / Prd;
                F = blend * Ft;
                dFdC = dF_dPrd * k0 / kf;
                dFdT = dF_dPrd * Prd * (dlnk0 - dlnkf) + blend * dFtdT;
            }
        }
        double rop = kf * Pf - kr * Pr;
        sh.rq[j] = F * rop;
        if (jac) {
            double dlnKc = dH - (double)dnu / T;
            double dkfdT = kf * dlnkf;
            double dkrdT = kr * (dlnkf - dlnKc);
            sh.rF[j] = F;
            sh.rkf[j] = kf;
            sh.rkr[j] = kr;
            sh.rrop[j] = rop;
            sh.rdFdC[j] = dFdC;
            sh.rdqT[j] = F * (dkfdT * Pf - dkrdT * Pr) + rop * dFdT;
        }
    }
    __syncwarp();
    // species gather: wdot_k = sum_j nu_kj q_j (reactions ascending)
    double Q = 0.0;
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            int k = c - 1;
            double w = 0.0, wt = 0.0;
            int b = __ldg(m.inc_ptr + k), e = __ldg(m.inc_ptr + k + 1);
            for (int t = b; t < e; ++t) {
                int2 ent = __ldg(m.inc + t);
                w += (double)ent.y * sh.rq[ent.x];
                if (jac) wt += (double)ent.y * sh.rdqT[ent.x];
            }
            if (jac) { sh.wdot[k] = w; sh.wT[k] = wt; }
            double W = __ldg(m.W + k);
            f[s] = W * w / rho;
            Q += sh.HRT[k] * RT * w;
        }
    }
    Q = warp_sum(Q);
    info.Q = Q;
    if (lane == 0) f[0] = -Q / (rho * cp);
    return info;
}

// Builds G = I/(h g) - J in the slice from the data of eval_rhs(..., jac = true).
__device__ void build_matrix(const DevMech &m, const Slice &sh, int lane, const EvalInfo &in, double h) {
    const int N = m.N, R = m.R, n = N + 1;
    double *G = sh.G;
    // zero the species block (lane owns the columns c = lane + 32 s throughout)
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= 1 && c < n)
            for (int r = 1; r < n; ++r) G[r * n + c] = 0.0;
    }
    __syncwarp();
    // JC[k][l] = d wdot_k / d C_l, reaction by reaction (ascending), column-parallel
    for (int j = 0; j < R; ++j) {
        const int type = __ldg(m.rtype + j);
        int rs[3], ps[3];
        for (int i = 0; i < 3; ++i) { rs[i] = __ldg(m.reac + 3 * j + i); ps[i] = __ldg(m.prod + 3 * j + i); }
        const double F = sh.rF[j], kf = sh.rkf[j], kr = sh.rkr[j], rop = sh.rrop[j], dFdC = sh.rdFdC[j];
        const double *e = (type != 0) ? m.eff + (size_t)__ldg(m.tb_row + j) * N : nullptr;
        for (int s = 0; s < 2; ++s) {
            const int c = lane + 32 * s;   // matrix column c = species l + 1
            if (c < 1 || c >= n) continue;
            const int l = c - 1;
            bool part = (type != 0);
            for (int i = 0; i < 3; ++i) part |= (rs[i] == l) || (ps[i] == l);
            if (!part) continue;
            double dPf = 0.0, dPr = 0.0;
            for (int i = 0; i < 3; ++i) {
                if (rs[i] == l) {
                    double t = 1.0;
                    for (int i2 = 0; i2 < 3; ++i2)
                        if (i2 != i && rs[i2] >= 0) t *= sh.C[rs[i2]];
                    dPf += t;
                }
                if (ps[i] == l) {
                    double t = 1.0;
                    for (int i2 = 0; i2 < 3; ++i2)
                        if (i2 != i && ps[i2] >= 0) t *= sh.C[ps[i2]];
                    dPr += t;
                }
            }
            double dFl = (type == 0) ? 0.0 : dFdC * __ldg(e + l);
            double dq = F * (kf * dPf - kr * dPr) + rop * dFl;
            for (int i = 0; i < 3; ++i) {
                if (rs[i] >= 0) G[(1 + rs[i]) * n + 1 + l] -= dq;
                if (ps[i] >= 0) G[(1 + ps[i]) * n + 1 + l] += dq;
            }
        }
    }
    __syncwarp();
    // JCC[k] = sum_l JC[k][l] C_l (lane per row)
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= 1 && c < n) {
            double acc = 0.0;
            for (int l = 0; l < N; ++l) acc += G[c * n + 1 + l] * sh.C[l];
            sh.JCC[c - 1] = acc;
        }
    }
    __syncwarp();
    const double T = in.T, rho = in.rho, cp = in.cp, Wbar = in.Wbar, Q = in.Q;
    const double rcp = rho * cp;
    const double ghinv = 1.0 / (h * kGam);
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c >= n) continue;
        if (c == 0) {
            // temperature column and J[0][0]
            double sT = 0.0;
            for (int k = 0; k < N; ++k) {
                double Wk = __ldg(m.W + k);
                double dwdT = sh.wT[k] - sh.JCC[k] / T;
                sT += sh.cpR[k] * kR * sh.wdot[k] + sh.HRT[k] * kR * T * dwdT;
                double J = Wk / rho * dwdT + Wk * sh.wdot[k] / (rho * T);
                G[(1 + k) * n] = -J;
            }
            double J00 = -sT / rcp - Q * (cp / T - in.dcpdT) / (rho * cp * cp);
            G[0] = ghinv - J00;
        } else {
            int mm = c - 1;
            double Wm = __ldg(m.W + mm);
            double sTr = 0.0;
            for (int k = 0; k < N; ++k) {
                double Wk = __ldg(m.W + k);
                double dw = G[(1 + k) * n + c] * rho / Wm - Wbar / Wm * sh.JCC[k];
                sTr += sh.HRT[k] * kR * T * dw;
                double J = Wk / rho * dw + Wk * sh.wdot[k] * Wbar / (rho * Wm);
                G[(1 + k) * n + c] = (1 + k == c) ? ghinv - J : -J;
            }
            double J0 = -sTr / rcp - Q * (cp * Wbar - sh.cpR[mm] * kR) / (rho * cp * cp * Wm);
            G[c] = -J0;
        }
    }
    __syncwarp();
}

// In-place LU with partial pivoting; returns false for an exactly singular matrix.
__device__ bool lu_factor(const Slice &sh, int lane, int n) {
    double *G = sh.G;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = n;
        for (int s = 0; s < 2; ++s) {
            int i = lane + 32 * s;
            if (i >= k && i < n) {
                double v = fabs(G[i * n + k]);
                if (v > best || (v == best && i < bi)) { best = v; bi = i; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(kFull, best, o);
            int oi = __shfl_xor_sync(kFull, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0) || bi >= n) return false;   // zero or non-finite column
        if (lane == 0) sh.piv[k] = bi;
        if (bi != k) {
            for (int s = 0; s < 2; ++s) {
                int c = lane + 32 * s;
                if (c < n) {
                    double t = G[k * n + c];
                    G[k * n + c] = G[bi * n + c];
                    G[bi * n + c] = t;
                }
            }
        }
        __syncwarp();
        const double pivot = G[k * n + k];
        for (int s = 0; s < 2; ++s) {
            int i = lane + 32 * s;
            if (i > k && i < n) G[i * n + k] = G[i * n + k] / pivot;
        }
        __syncwarp();
        for (int s = 0; s < 2; ++s) {
            int c = lane + 32 * s;
            if (c > k && c < n) {
                const double akc = G[k * n + c];
                for (int i = k + 1; i < n; ++i) G[i * n + c] -= G[i * n + k] * akc;
            }
        }
        __syncwarp();
    }
    return true;
}

// b <- G^-1 b with the stored factors; b is lane-distributed.
__device__ void lu_solve(const Slice &sh, int lane, int n, double b[2]) {
    const double *G = sh.G;
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        if (c < n) sh.bsw[c] = b[s];
    }
    __syncwarp();
    if (lane == 0) {
        for (int k = 0; k < n; ++k) {
            int p = sh.piv[k];
            if (p != k) { double t = sh.bsw[k]; sh.bsw[k] = sh.bsw[p]; sh.bsw[p] = t; }
        }
    }
    __syncwarp();
    for (int s = 0; s < 2; ++s) {
        int c = lane + 32 * s;
        b[s] = (c < n) ? sh.bsw[c] : 0.0;
    }
    for (int k = 0; k < n - 1; ++k) {
        double bk = __shfl_sync(kFull, sel(b, k >> 5), k & 31);
        for (int s = 0; s < 2; ++s) {
            int i = lane + 32 * s;
            if (i > k && i < n) b[s] -= G[i * n + k] * bk;
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        if ((k & 31) == lane) {
            if (k >> 5) b[1] = b[1] / G[k * n + k];
            else b[0] = b[0] / G[k * n + k];
        }
        double bk = __shfl_sync(kFull, sel(b, k >> 5), k & 31);
        for (int s = 0; s < 2; ++s) {
            int i = lane + 32 * s;
            if (i < k) b[s] -= G[i * n + k] * bk;
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kWarps * 32) stiff_kernel(DevMech m, int64_t ncells, int64_t ld, double dt,
                                                             chem_ode_opts o, double *__restrict__ Tg,
                                                             const double *__restrict__ pg, double *__restrict__ Yg,
                                                             int32_t *__restrict__ status,
                                                             int32_t *__restrict__ nsteps_out,
                                                             unsigned int *__restrict__ queue) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int N = m.N, n = N + 1;
    Slice sh = make_slice(smem + (size_t)warp * slice_bytes(N, m.R), N, m.R);
    for (;;) {
        unsigned int cell_u = 0;
        if (lane == 0) cell_u = atomicAdd(queue, 1u);
        cell_u = __shfl_sync(kFull, cell_u, 0);
        const int64_t cell = (int64_t)cell_u;
        if (cell >= ncells) break;
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
            EvalInfo info = eval_rhs(m, sh, lane, p, y, f0, true);
            bool bad = false;
            for (int s = 0; s < 2; ++s)
                if (lane + 32 * s < n && !isfinite(f0[s])) bad = true;
            if (__any_sync(kFull, bad)) { stat = CHEM_CELL_NONFINITE; break; }
            build_matrix(m, sh, lane, info, h);
            ++nst;
            if (!lu_factor(sh, lane, n)) { h *= 0.2; rejected_last = 1; continue; }
            const double ih = 1.0 / h;
            // stage 1
            for (int s = 0; s < 2; ++s) K1[s] = f0[s];
            lu_solve(sh, lane, n, K1);
            // stage 2: the stage point is y itself (a21 = 0)
            for (int s = 0; s < 2; ++s) K2[s] = f0[s] + (kC21 * ih) * K1[s];
            lu_solve(sh, lane, n, K2);
            // stage 3: y + 2 K1
            for (int s = 0; s < 2; ++s) ys[s] = y[s] + kA31 * K1[s];
            eval_rhs(m, sh, lane, p, ys, fs, false);
            for (int s = 0; s < 2; ++s) {
                double v = fs[s];
                v += (kC31 * ih) * K1[s];
                v += (kC32 * ih) * K2[s];
                K3[s] = v;
            }
            lu_solve(sh, lane, n, K3);
            // stage 4: y + 2 K1 + K3
            for (int s = 0; s < 2; ++s) ys[s] = y[s] + kA41 * K1[s] + kA43 * K3[s];
            eval_rhs(m, sh, lane, p, ys, fs, false);
            for (int s = 0; s < 2; ++s) {
                double v = fs[s];
                v += (kC41 * ih) * K1[s];
                v += (kC42 * ih) * K2[s];
                v += (kC43 * ih) * K3[s];
                K4[s] = v;
            }
            lu_solve(sh, lane, n, K4);
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
        for (int s = 0; s < 2; ++s) {
            int c = lane + 32 * s;
            if (c == 0) Tg[cell] = y[s];
            else if (c < n) Yg[(int64_t)(c - 1) * ld + cell] = y[s];
        }
        if (lane == 0) {
            status[cell] = stat;
            if (nsteps_out) nsteps_out[cell] = nst;
        }
    }
}

}  // namespace
}  // namespace chemgb

using namespace chemgb;

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
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_step_stiff: " + why);
    size_t per_warp = slice_bytes(m->N, m->R);
    size_t smem = per_warp * kWarps;
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
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned int *queue = m->dev.counters;
    int rc = check_cuda(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st), "chem_step_stiff: queue reset");
    if (rc) return rc;
    stiff_kernel<<<blocks, kWarps * 32, smem, st>>>(m->dev, ncells, ld, dt, o, T, p, Y, status, nsteps, queue);
    return check_cuda(cudaGetLastError(), "chem_step_stiff launch");
}
