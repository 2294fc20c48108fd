/*
 * chem_oracle.c -- plain, slow FP64 CPU oracle of the per-cell chemistry and
 * properties step (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py may load this library. The product path never calls it, and it
 * shares no code, header or table with the CUDA library.
 *
 * What it computes (the paper names the models, Sec. 2 and Sec. 3.1, but prints
 * no formulas; the formulas below are the textbook definitions):
 *   - NASA-7 species thermodynamics and mixture cp, h         (Sec. 2: thermal properties on the GPU)
 *   - mixture-averaged transport: Wilke viscosity, Wilke-form
 *     conductivity with Eucken species conductivities, and
 *     Hirschfelder-Curtiss mixture diffusion coefficients      (Sec. 2; Sec. 3.1 names Hirschfelder-Curtiss)
 *   - mass-action kinetics with reverse rates from the NASA
 *     Gibbs energies, three-body and Troe fall-off reactions    (Sec. 3.1: the chemistry the ODEs describe)
 *   - the constant-pressure adiabatic reactor dy/dt = f(y),
 *     y = (T, Y_1..Y_N), and its analytic Jacobian              (Sec. 3.1: ODE integration over dt = 1 us)
 *   - an embedded L-stable Rosenbrock method, Rodas3 of Sandu et
 *     al. (1997), 4 stages, order 3(2), with adaptive steps     (Sec. 3.1 uses CVODE; Sec. 4.2 "CPU-DI")
 * Every loop runs in the plain order of the definitions; cells are independent
 * and are split across OpenMP threads with no other reordering.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OM_R 8.314462618
#define OM_MAXN 64

typedef struct {
    int N, R, E, bath;
    double P_std, T_lo, T_mid, T_hi;
    const double *W;        /* [N] kg/mol */
    const double *nasa_lo;  /* [N][7] */
    const double *nasa_hi;  /* [N][7] */
    const double *visc_fit; /* [N][5]: ln mu_k = sum c_n x^n, x = ln(T/1000) */
    const double *diff_fit; /* [N][N][5]: g_jk = p T^-1.5 / D_jk = sum c_n x^n */
    const int *rtype;       /* [R]: 0 elementary, 1 three-body, 2 Troe */
    const int *reac;        /* [R][3], -1 pad, repeated species for nu = 2 */
    const int *prod;        /* [R][3] */
    const double *A, *beta, *Ea, *A0, *beta0, *Ea0;
    const double *troe;     /* [R][4]: a, T***, T*, T** */
    const double *eff;      /* [R][N] */
} om_mech;

typedef struct {
    double rtol, atol_Y, atol_T, h0;
    int max_steps;
} om_ode_opts;

/* ------------------------------------------------------------------------- */
/* NASA-7 thermodynamics                                                      */
/* ------------------------------------------------------------------------- */

static const double *nasa_coef(const om_mech *m, int k, double T) {
    /* T >= T_mid uses the high range; outside [T_lo, T_hi] the end polynomial
       is extrapolated (no clamp). */
    return (T >= m->T_mid) ? m->nasa_hi + 7 * k : m->nasa_lo + 7 * k;
}

/* cp/R, H/(RT), S/R and d(cp/R)/dT of species k */
void om_species_thermo(const om_mech *m, int k, double T, double *cp_R, double *H_RT, double *S_R,
                       double *dcp_RdT) {
    const double *a = nasa_coef(m, k, T);
    double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    if (cp_R) *cp_R = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    if (H_RT) *H_RT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    if (S_R) *S_R = a[0] * log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
    if (dcp_RdT) *dcp_RdT = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T2 + 4.0 * a[4] * T3;
}

/* mixture cp (J/kg/K) and h (J/kg) of one cell */
static void mix_thermo(const om_mech *m, double T, const double *Y, double *cp, double *h) {
    double c = 0.0, hh = 0.0;
    for (int k = 0; k < m->N; ++k) {
        double cpR, HRT;
        om_species_thermo(m, k, T, &cpR, &HRT, NULL, NULL);
        c += Y[k] * cpR * OM_R / m->W[k];
        hh += Y[k] * HRT * OM_R * T / m->W[k];
    }
    *cp = c;
    *h = hh;
}

/* ------------------------------------------------------------------------- */
/* Mixture-averaged transport                                                 */
/* ------------------------------------------------------------------------- */

static double poly5(const double *c, double x) {
    return c[0] + c[1] * x + c[2] * x * x + c[3] * x * x * x + c[4] * x * x * x * x;
}

/* One cell. Y has unit stride here; Dk receives N values. */
static void cell_props(const om_mech *m, double T, double p, const double *Y, double *cp, double *h,
                       double *mu, double *lam, double *Dk) {
    int N = m->N;
    double muk[OM_MAXN], lamk[OM_MAXN], X[OM_MAXN];
    double x = log(T / 1000.0);
    mix_thermo(m, T, Y, cp, h);
    double S = 0.0;
    for (int k = 0; k < N; ++k) S += Y[k] / m->W[k];
    double Wbar = 1.0 / S;
    for (int k = 0; k < N; ++k) {
        double cpR;
        om_species_thermo(m, k, T, &cpR, NULL, NULL, NULL);
        X[k] = Y[k] * Wbar / m->W[k];
        muk[k] = exp(poly5(m->visc_fit + 5 * k, x));
        /* Eucken: lambda_k = mu_k (cp_k + 5R/4) / W_k, cp_k molar */
        lamk[k] = muk[k] * (cpR * OM_R + 1.25 * OM_R) / m->W[k];
    }
    /* Wilke: mu = sum_k X_k mu_k / sum_j X_j Phi_kj; the conductivity uses the same Phi */
    double mus = 0.0, lams = 0.0;
    for (int k = 0; k < N; ++k) {
        double den = 0.0;
        for (int j = 0; j < N; ++j) {
            double t = 1.0 + sqrt(muk[k] / muk[j]) * pow(m->W[j] / m->W[k], 0.25);
            double phi = t * t / sqrt(8.0 * (1.0 + m->W[k] / m->W[j]));
            den += X[j] * phi;
        }
        mus += X[k] * muk[k] / den;
        lams += X[k] * lamk[k] / den;
    }
    *mu = mus;
    *lam = lams;
    /* Hirschfelder-Curtiss: D_km = (1 - Y_k) / sum_{j != k} X_j / D_jk, D_jk = T^1.5 / (p g_jk) */
    double T15 = T * sqrt(T);
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int j = 0; j < N; ++j)
            if (j != k) s += X[j] * poly5(m->diff_fit + 5 * (j * N + k), x);
        if (1.0 - X[k] < 1e-12) {
            /* pure species k: the limit is not defined by the formula; use the mean resistance */
            double g = 0.0;
            for (int j = 0; j < N; ++j)
                if (j != k) g += poly5(m->diff_fit + 5 * (j * N + k), x);
            Dk[k] = T15 / (p * g / (double)(N - 1));
        } else {
            Dk[k] = (1.0 - Y[k]) * T15 / (p * s);
        }
    }
}

/* props over ncells SoA cells: Y[k*ld + i], Dk[k*ld + i] */
void om_props(const om_mech *m, long ncells, long ld, const double *T, const double *p, const double *Y,
              double *cp, double *h, double *mu, double *lam, double *Dk) {
    int N = m->N;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < ncells; ++i) {
        double y[OM_MAXN], d[OM_MAXN];
        for (int k = 0; k < N; ++k) y[k] = Y[(long)k * ld + i];
        cell_props(m, T[i], p[i], y, &cp[i], &h[i], &mu[i], &lam[i], d);
        for (int k = 0; k < N; ++k) Dk[(long)k * ld + i] = d[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Kinetics                                                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    /* per-reaction values at (T, C) needed by the RHS and the Jacobian */
    double kf, kr, Pf, Pr, F, dFdC, dFdT, dkfdT, dkrdT;
} rxn_state;

/* Troe blending F(T, Pr) with d(log10 F)/dL and d(log10 F)/d(log10 Fcent), plus dFcent/dT */
static void troe_F(const double *tp, double T, double Prd, double *F, double *dlgF_dlgPr, double *dF_dT_atPr) {
    double a = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
    double Fc = (1.0 - a) * exp(-T / T3) + a * exp(-T / T1) + exp(-T2 / T);
    double dFc = -(1.0 - a) / T3 * exp(-T / T3) - a / T1 * exp(-T / T1) + T2 / (T * T) * exp(-T2 / T);
    double phi = log10(Fc);
    double c = -0.4 - 0.67 * phi, n = 0.75 - 1.27 * phi, d = 0.14;
    double L = log10(Prd) + c;
    double den = n - d * L;
    double f1 = L / den;
    double q = 1.0 + f1 * f1;
    double lgF = phi / q;
    *F = pow(10.0, lgF);
    /* d lgF / dL at fixed phi */
    double df1_dL = n / (den * den);
    *dlgF_dlgPr = -phi * 2.0 * f1 / (q * q) * df1_dL;
    /* d lgF / dphi at fixed Prd */
    double dL_dphi = -0.67, dn_dphi = -1.27;
    double df1_dphi = (dL_dphi * den - L * (dn_dphi - d * dL_dphi)) / (den * den);
    double dlgF_dphi = 1.0 / q - phi * 2.0 * f1 / (q * q) * df1_dphi;
    double dphi_dT = dFc / (Fc * log(10.0));
    *dF_dT_atPr = (*F) * log(10.0) * dlgF_dphi * dphi_dT;
}

/* per-reaction rate data at temperature T and concentrations C (mol/m^3) */
static void reaction_states(const om_mech *m, double T, const double *C, const double *H_RT, const double *S_R,
                            const double *cpR_unused, rxn_state *rs) {
    (void)cpR_unused;
    int N = m->N;
    double RT = OM_R * T;
    for (int j = 0; j < m->R; ++j) {
        rxn_state *r = &rs[j];
        const int *re = m->reac + 3 * j, *pr = m->prod + 3 * j;
        double kf = m->A[j] * pow(T, m->beta[j]) * exp(-m->Ea[j] / RT);
        double dlnkf = m->beta[j] / T + m->Ea[j] / (RT * T);
        /* Gibbs: ln Kp = sum nu (S/R - H/RT); Kc = Kp (P_std/RT)^sum(nu) */
        double lnKp = 0.0, dH_RT2 = 0.0;
        int dnu = 0;
        for (int i = 0; i < 3; ++i) {
            if (pr[i] >= 0) { lnKp += S_R[pr[i]] - H_RT[pr[i]]; dH_RT2 += H_RT[pr[i]] / T; dnu += 1; }
            if (re[i] >= 0) { lnKp -= S_R[re[i]] - H_RT[re[i]]; dH_RT2 -= H_RT[re[i]] / T; dnu -= 1; }
        }
        double Kc = exp(lnKp) * pow(m->P_std / RT, (double)dnu);
        double dlnKc = dH_RT2 - (double)dnu / T;
        double kr = kf / Kc;
        double Pf = 1.0, Pr = 1.0;
        for (int i = 0; i < 3; ++i) {
            if (re[i] >= 0) Pf *= C[re[i]];
            if (pr[i] >= 0) Pr *= C[pr[i]];
        }
        r->kf = kf; r->kr = kr; r->Pf = Pf; r->Pr = Pr;
        r->dkfdT = kf * dlnkf;
        r->dkrdT = kr * (dlnkf - dlnKc);
        if (m->rtype[j] == 0) {
            r->F = 1.0; r->dFdC = 0.0; r->dFdT = 0.0;
        } else {
            double M = 0.0;
            for (int k = 0; k < N; ++k) M += m->eff[(long)j * N + k] * C[k];
            if (m->rtype[j] == 1) {
                r->F = M; r->dFdC = 1.0; r->dFdT = 0.0;   /* dF/dC_k = eff_jk * dFdC */
            } else {
                double k0 = m->A0[j] * pow(T, m->beta0[j]) * exp(-m->Ea0[j] / RT);
                double dlnk0 = m->beta0[j] / T + m->Ea0[j] / (RT * T);
                double Prd = k0 * M / kf;
                if (Prd < 1e-300) Prd = 1e-300;
                double Ft, glg, dFtdT;
                troe_F(m->troe + 4 * j, T, Prd, &Ft, &glg, &dFtdT);
                double blend = Prd / (1.0 + Prd);
                /* dF/dPrd with F = blend * Ft, dFt/dPrd = Ft * glg / Prd */
                double dF_dPrd = Ft / ((1.0 + Prd) * (1.0 + Prd)) + blend * Ft * glg / Prd;
                r->F = blend * Ft;
                r->dFdC = dF_dPrd * k0 / kf;           /* times eff_jk */
                r->dFdT = dF_dPrd * Prd * (dlnk0 - dlnkf) + blend * dFtdT;
            }
        }
    }
}

/* net production rates wdot (mol/m^3/s) and rates of progress q at (T, p, Y) */
void om_rates(const om_mech *m, double T, double p, const double *Y, double *wdot, double *q) {
    int N = m->N;
    double H_RT[OM_MAXN], S_R[OM_MAXN], C[OM_MAXN];
    double S = 0.0;
    for (int k = 0; k < N; ++k) S += Y[k] / m->W[k];
    double rho = p / (OM_R * T * S);
    for (int k = 0; k < N; ++k) {
        om_species_thermo(m, k, T, NULL, &H_RT[k], &S_R[k], NULL);
        C[k] = rho * Y[k] / m->W[k];
        wdot[k] = 0.0;
    }
    rxn_state *rs = (rxn_state *)malloc(sizeof(rxn_state) * (size_t)m->R);
    reaction_states(m, T, C, H_RT, S_R, NULL, rs);
    for (int j = 0; j < m->R; ++j) {
        double qj = rs[j].F * (rs[j].kf * rs[j].Pf - rs[j].kr * rs[j].Pr);
        if (q) q[j] = qj;
        for (int i = 0; i < 3; ++i) {
            if (m->reac[3 * j + i] >= 0) wdot[m->reac[3 * j + i]] -= qj;
            if (m->prod[3 * j + i] >= 0) wdot[m->prod[3 * j + i]] += qj;
        }
    }
    free(rs);
}

/* forward and reverse rate constants (for the detailed-balance pin) */
void om_rate_constants(const om_mech *m, double T, double p, const double *Y, double *kf, double *kr) {
    int N = m->N;
    double H_RT[OM_MAXN], S_R[OM_MAXN], C[OM_MAXN];
    double S = 0.0;
    for (int k = 0; k < N; ++k) S += Y[k] / m->W[k];
    double rho = p / (OM_R * T * S);
    for (int k = 0; k < N; ++k) {
        om_species_thermo(m, k, T, NULL, &H_RT[k], &S_R[k], NULL);
        C[k] = rho * Y[k] / m->W[k];
    }
    rxn_state *rs = (rxn_state *)malloc(sizeof(rxn_state) * (size_t)m->R);
    reaction_states(m, T, C, H_RT, S_R, NULL, rs);
    for (int j = 0; j < m->R; ++j) { kf[j] = rs[j].kf * rs[j].F; kr[j] = rs[j].kr * rs[j].F; }
    free(rs);
}

/* Reactor right-hand side f(y), y = (T, Y_1..Y_N), at constant p:
   dY_k/dt = W_k wdot_k / rho,  dT/dt = -sum_k H_k wdot_k / (rho cp). */
void om_rhs(const om_mech *m, double p, const double *y, double *f) {
    int N = m->N;
    double T = y[0];
    const double *Y = y + 1;
    double wdot[OM_MAXN];
    om_rates(m, T, p, Y, wdot, NULL);
    double S = 0.0, cp = 0.0, Q = 0.0;
    for (int k = 0; k < N; ++k) S += Y[k] / m->W[k];
    double rho = p / (OM_R * T * S);
    for (int k = 0; k < N; ++k) {
        double cpR, HRT;
        om_species_thermo(m, k, T, &cpR, &HRT, NULL, NULL);
        cp += Y[k] * cpR * OM_R / m->W[k];
        Q += HRT * OM_R * T * wdot[k];
        f[1 + k] = m->W[k] * wdot[k] / rho;
    }
    f[0] = -Q / (rho * cp);
}

/* Analytic Jacobian J[a*n + b] = d f_a / d y_b, n = N + 1; rho depends on (T, Y). */
void om_jac(const om_mech *m, double p, const double *y, double *J) {
    int N = m->N, n = N + 1;
    double T = y[0];
    const double *Y = y + 1;
    double H_RT[OM_MAXN], S_R[OM_MAXN], cpR[OM_MAXN], dcpR[OM_MAXN], C[OM_MAXN], wdot[OM_MAXN];
    double S = 0.0;
    for (int k = 0; k < N; ++k) S += Y[k] / m->W[k];
    double Wbar = 1.0 / S;
    double rho = p / (OM_R * T * S);
    double cp = 0.0, dcpdT = 0.0, Q = 0.0;
    for (int k = 0; k < N; ++k) {
        om_species_thermo(m, k, T, &cpR[k], &H_RT[k], &S_R[k], &dcpR[k]);
        C[k] = rho * Y[k] / m->W[k];
        cp += Y[k] * cpR[k] * OM_R / m->W[k];
        dcpdT += Y[k] * dcpR[k] * OM_R / m->W[k];
        wdot[k] = 0.0;
    }
    rxn_state *rs = (rxn_state *)malloc(sizeof(rxn_state) * (size_t)m->R);
    reaction_states(m, T, C, H_RT, S_R, NULL, rs);
    /* JC[k][l] = d wdot_k / d C_l ; wT[k] = d wdot_k / dT at fixed C */
    double *JC = (double *)calloc((size_t)N * N, sizeof(double));
    double wT[OM_MAXN];
    for (int k = 0; k < N; ++k) wT[k] = 0.0;
    double dq[OM_MAXN];
    for (int j = 0; j < m->R; ++j) {
        const rxn_state *r = &rs[j];
        const int *re = m->reac + 3 * j, *pr = m->prod + 3 * j;
        double rop = r->kf * r->Pf - r->kr * r->Pr;
        double qj = r->F * rop;
        for (int l = 0; l < N; ++l) {
            /* d Pf / d C_l and d Pr / d C_l by the product rule over the reactant / product slots */
            double dPf = 0.0, dPr = 0.0;
            for (int i = 0; i < 3; ++i) {
                if (re[i] == l) {
                    double t = 1.0;
                    for (int i2 = 0; i2 < 3; ++i2) if (i2 != i && re[i2] >= 0) t *= C[re[i2]];
                    dPf += t;
                }
                if (pr[i] == l) {
                    double t = 1.0;
                    for (int i2 = 0; i2 < 3; ++i2) if (i2 != i && pr[i2] >= 0) t *= C[pr[i2]];
                    dPr += t;
                }
            }
            double dFl = (m->rtype[j] == 0) ? 0.0 : r->dFdC * m->eff[(long)j * N + l];
            dq[l] = r->F * (r->kf * dPf - r->kr * dPr) + rop * dFl;
        }
        double dqT = r->F * (r->dkfdT * r->Pf - r->dkrdT * r->Pr) + rop * r->dFdT;
        for (int i = 0; i < 3; ++i) {
            int s;
            if ((s = re[i]) >= 0) {
                for (int l = 0; l < N; ++l) JC[s * N + l] -= dq[l];
                wT[s] -= dqT;
                wdot[s] -= qj;
            }
            if ((s = pr[i]) >= 0) {
                for (int l = 0; l < N; ++l) JC[s * N + l] += dq[l];
                wT[s] += dqT;
                wdot[s] += qj;
            }
        }
    }
    free(rs);
    for (int k = 0; k < N; ++k) Q += H_RT[k] * OM_R * T * wdot[k];
    /* chain rule through C_l(T, Y): dC_l/dY_m = rho/W_l delta_lm - C_l Wbar / W_m ; dC_l/dT = -C_l / T */
    double JCC[OM_MAXN];
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int l = 0; l < N; ++l) s += JC[k * N + l] * C[l];
        JCC[k] = s;
    }
    double rcp = rho * cp;
    /* T row */
    {
        double sT = 0.0;
        for (int k = 0; k < N; ++k) {
            double dwdT = wT[k] - JCC[k] / T;
            sT += cpR[k] * OM_R * wdot[k] + H_RT[k] * OM_R * T * dwdT;
        }
        J[0] = -sT / rcp - Q * (cp / T - dcpdT) / (rho * cp * cp);
        for (int mm = 0; mm < N; ++mm) {
            double s = 0.0;
            for (int k = 0; k < N; ++k) {
                double dw = JC[k * N + mm] * rho / m->W[mm] - Wbar / m->W[mm] * JCC[k];
                s += H_RT[k] * OM_R * T * dw;
            }
            J[1 + mm] = -s / rcp - Q * (cp * Wbar - cpR[mm] * OM_R) / (rho * cp * cp * m->W[mm]);
        }
    }
    /* Y rows */
    for (int k = 0; k < N; ++k) {
        double dwdT = wT[k] - JCC[k] / T;
        J[(1 + k) * n + 0] = m->W[k] / rho * dwdT + m->W[k] * wdot[k] / (rho * T);
        for (int mm = 0; mm < N; ++mm) {
            double dw = JC[k * N + mm] * rho / m->W[mm] - Wbar / m->W[mm] * JCC[k];
            J[(1 + k) * n + 1 + mm] = m->W[k] / rho * dw + m->W[k] * wdot[k] * Wbar / (rho * m->W[mm]);
        }
    }
    free(JC);
}

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (row-major n x n)                           */
/* ------------------------------------------------------------------------- */

static int lu_factor(double *A, int n, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(const double *A, int n, const int *piv, double *b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 1; i < n; ++i) {
        double s = b[i];
        for (int j = 0; j < i; ++j) s -= A[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
}

/* ------------------------------------------------------------------------- */
/* Rodas3 (Sandu et al. 1997) in the transformed Rosenbrock form              */
/*   (I/(h g) - J) K_i = f(y + sum_j a_ij K_j) + sum_j (c_ij / h) K_j          */
/*   y_new = y + sum m_i K_i ; error estimate = sum e_i K_i                     */
/* ------------------------------------------------------------------------- */

static const double RO_G = 0.5;
static const double RO_A[4][3] = {{0, 0, 0}, {0.0, 0, 0}, {2.0, 0.0, 0}, {2.0, 0.0, 1.0}};
static const double RO_C[4][3] = {{0, 0, 0}, {4.0, 0, 0}, {1.0, -1.0, 0}, {1.0, -1.0, -8.0 / 3.0}};
static const double RO_M[4] = {2.0, 0.0, 1.0, 1.0};
static const double RO_E[4] = {0.0, 0.0, 0.0, 1.0};

enum { OM_OK = 0, OM_MAXSTEPS = 2, OM_UNDERFLOW = 3, OM_NONFINITE = 4 };

/* Integrate one cell over [0, dt]; y (n = N+1) is updated in place. */
int om_integrate_cell(const om_mech *m, double p, double dt, const om_ode_opts *o, double *y, int *nsteps_out) {
    int N = m->N, n = N + 1;
    double *G = (double *)malloc(sizeof(double) * (size_t)n * n);
    double K[4][OM_MAXN + 1], f0[OM_MAXN + 1], ys[OM_MAXN + 1], fs[OM_MAXN + 1], yn[OM_MAXN + 1];
    int piv[OM_MAXN + 1];
    double t = 0.0, h = (o->h0 < dt) ? o->h0 : dt;
    int nsteps = 0, rejected_last = 0, status = OM_OK;
    while (t < dt) {
        if (nsteps >= o->max_steps) { status = OM_MAXSTEPS; break; }
        if (h < 1e-20 * dt) { status = OM_UNDERFLOW; break; }
        double rem = dt - t;
        int last = 0;
        if (h >= rem) { h = rem; last = 1; }
        om_rhs(m, p, y, f0);
        int bad = 0;
        for (int i = 0; i < n; ++i) if (!isfinite(f0[i])) bad = 1;
        if (bad) { status = OM_NONFINITE; break; }
        om_jac(m, p, y, G);
        double ghinv = 1.0 / (h * RO_G);
        for (int i = 0; i < n * n; ++i) G[i] = -G[i];
        for (int i = 0; i < n; ++i) G[i * n + i] += ghinv;
        ++nsteps;
        if (lu_factor(G, n, piv)) { h *= 0.2; rejected_last = 1; continue; }
        for (int s = 0; s < 4; ++s) {
            const double *fx;
            int need_f = 0;
            for (int j = 0; j < s; ++j) if (RO_A[s][j] != 0.0) need_f = 1;
            if (need_f) {
                for (int i = 0; i < n; ++i) {
                    double v = y[i];
                    for (int j = 0; j < s; ++j) v += RO_A[s][j] * K[j][i];
                    ys[i] = v;
                }
                om_rhs(m, p, ys, fs);
                fx = fs;
            } else {
                fx = f0;   /* the stage point is y itself */
            }
            for (int i = 0; i < n; ++i) {
                double v = fx[i];
                for (int j = 0; j < s; ++j) v += (RO_C[s][j] / h) * K[j][i];
                K[s][i] = v;
            }
            lu_solve(G, n, piv, K[s]);
        }
        double acc = 0.0;
        int nonfinite = 0;
        for (int i = 0; i < n; ++i) {
            double v = y[i], e = 0.0;
            for (int s = 0; s < 4; ++s) { v += RO_M[s] * K[s][i]; e += RO_E[s] * K[s][i]; }
            yn[i] = v;
            double ay = fabs(y[i]), ayn = fabs(v);
            double sc = ((i == 0) ? o->atol_T : o->atol_Y) + o->rtol * (ay > ayn ? ay : ayn);
            double r = e / sc;
            acc += r * r;
            if (!isfinite(v) || !isfinite(e)) nonfinite = 1;
        }
        double err = sqrt(acc / (double)n);
        double fac;
        if (nonfinite || !isfinite(err)) {
            fac = 0.2;
            err = 2.0;
        } else {
            fac = (err > 0.0) ? 0.9 * pow(err, -1.0 / 3.0) : 5.0;
            if (fac > 5.0) fac = 5.0;
            if (fac < 0.2) fac = 0.2;
        }
        if (err <= 1.0) {
            t = last ? dt : t + h;
            for (int i = 0; i < n; ++i) y[i] = yn[i];
            if (rejected_last && fac > 1.0) fac = 1.0;
            h *= fac;
            rejected_last = 0;
        } else {
            h *= fac;
            rejected_last = 1;
        }
    }
    free(G);
    if (nsteps_out) *nsteps_out = nsteps;
    return status;
}

/* Stiff step over ncells SoA cells (T and Y updated in place). */
void om_step_stiff(const om_mech *m, long ncells, long ld, double dt, const om_ode_opts *o, double *T,
                   const double *p, double *Y, int *status, int *nsteps) {
    int N = m->N;
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < ncells; ++i) {
        double y[OM_MAXN + 1];
        y[0] = T[i];
        for (int k = 0; k < N; ++k) y[1 + k] = Y[(long)k * ld + i];
        int ns = 0;
        int st = om_integrate_cell(m, p[i], dt, o, y, &ns);
        T[i] = y[0];
        for (int k = 0; k < N; ++k) Y[(long)k * ld + i] = y[1 + k];
        if (status) status[i] = st;
        if (nsteps) nsteps[i] = ns;
    }
}

/* Rodas3 with nsub equal steps and no error control (used to observe the order
   of the method on problems with a closed-form solution). */
void om_rodas3_fixed(const om_mech *m, double p, double dt, int nsub, double *y) {
    int N = m->N, n = N + 1;
    double *G = (double *)malloc(sizeof(double) * (size_t)n * n);
    double K[4][OM_MAXN + 1], f0[OM_MAXN + 1], ys[OM_MAXN + 1], fs[OM_MAXN + 1];
    int piv[OM_MAXN + 1];
    double h = dt / (double)nsub;
    for (int st = 0; st < nsub; ++st) {
        om_rhs(m, p, y, f0);
        om_jac(m, p, y, G);
        for (int i = 0; i < n * n; ++i) G[i] = -G[i];
        for (int i = 0; i < n; ++i) G[i * n + i] += 1.0 / (h * RO_G);
        lu_factor(G, n, piv);
        for (int s = 0; s < 4; ++s) {
            for (int i = 0; i < n; ++i) {
                double v = y[i];
                for (int j = 0; j < s; ++j) v += RO_A[s][j] * K[j][i];
                ys[i] = v;
            }
            om_rhs(m, p, ys, fs);
            for (int i = 0; i < n; ++i) {
                double v = fs[i];
                for (int j = 0; j < s; ++j) v += (RO_C[s][j] / h) * K[j][i];
                K[s][i] = v;
            }
            lu_solve(G, n, piv, K[s]);
        }
        for (int i = 0; i < n; ++i)
            for (int s = 0; s < 4; ++s) y[i] += RO_M[s] * K[s][i];
    }
    free(G);
}

int om_max_species(void) { return OM_MAXN; }
