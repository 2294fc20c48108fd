/*
 * chemgb.h -- C ABI of the GB300 (sm_103a) per-cell chemistry and properties
 * library (libchemgb.so).
 *
 * The operation behind every entry point is the per-cell step of the paper's
 * GPU-ANN LES method (Zhang et al., arXiv 2312.05800): given the thermochemical
 * state (T, p, Y) of every cell, evaluate the thermal and transport properties
 * (Sec. 2) and advance the composition over one flow step dt (Sec. 3.1: the
 * reaction ODEs integrated over dt = 1 us; Sec. 3.2: the network maps
 * x(t) = {T, p, F(Y)} to u*(t) = Y(t + dt) - Y(t)).
 *
 * Conventions shared by all entry points
 *  - Cell data are structure-of-arrays with a leading dimension ld >= ncells:
 *    T[i], p[i] for cell i and Y[k * ld + i] for species k. ld must be a
 *    multiple of 4 (16-byte rows for FP32, 32-byte for FP64) and every array
 *    pointer 16-byte aligned; otherwise the call returns CHEM_EINVAL.
 *  - Unless an argument says "host", array pointers are DEVICE pointers owned
 *    by the caller; the library never frees them. Mechanism and network
 *    handles are owned by the library (create / free pairs).
 *  - Calls are asynchronous on the given CUDA stream (0 = legacy default
 *    stream). Results are valid once the stream reaches that point.
 *  - Units are SI: K, Pa, kg, m, s, mol, J.
 *  - Return codes: CHEM_OK (0) on success; a negative code otherwise, with a
 *    message available from chem_last_error() on the calling thread. Errors
 *    that belong to one cell (a step limit hit, a non-finite state) never fail
 *    the call: they are reported in the per-cell status array.
 *  - No host fallback exists: on a machine without an sm_103 device every
 *    compute call returns CHEM_EUNSUPPORTED.
 */
#ifndef CHEMGB_H
#define CHEMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *chem_stream_t; /* a cudaStream_t */

enum {
    CHEM_OK = 0,
    CHEM_EINVAL = -1,      /* null pointer, bad size, misalignment, mismatched handles */
    CHEM_ECUDA = -2,       /* a CUDA runtime error (launch, allocation at load time) */
    CHEM_EUNSUPPORTED = -3,/* no sm_103 device, or a feature not built */
    CHEM_EIO = -4          /* a file could not be read or has a bad format */
};

/* per-cell status codes written by the stepping entry points */
enum {
    CHEM_CELL_OK = 0,          /* integrated (stiff) or predicted (ANN) */
    CHEM_CELL_FALLBACK = 1,    /* ANN step: routed to the stiff integrator, which succeeded */
    CHEM_CELL_MAXSTEPS = 2,    /* stiff: step limit reached before dt */
    CHEM_CELL_UNDERFLOW = 3,   /* stiff: step size fell below 1e-20 dt */
    CHEM_CELL_NONFINITE = 4    /* a non-finite state or right-hand side */
};

enum {
    CHEM_F32 = 0,        /* float inputs, float arithmetic, float outputs */
    CHEM_F64 = 1,        /* double inputs, double arithmetic, double outputs */
    CHEM_F64_IN_F32 = 2  /* double inputs (the stepped FP64 state), float arithmetic, float outputs */
};

/* ---------------------------------------------------------------------------
 * Mechanism
 * ---------------------------------------------------------------------------
 * A reaction mechanism with NASA-7 thermodynamics, transport fits and reaction
 * data (the paper's chemistry, Sec. 3.1; its own mechanism is DRM19, which any
 * file in this format can stand in for).
 *
 * File format (little-endian, packed, in this order):
 *   char magic[8] = "CHMECH01"
 *   int32 N, R, E, bath                     species, reactions, elements, bath index
 *   float64 P_std, T_lo, T_mid, T_hi        standard pressure (Pa), NASA ranges (K)
 *   float64 W[N]                            molar masses, kg/mol
 *   float64 nasa_lo[N][7], nasa_hi[N][7]    NASA-7 rows; T >= T_mid uses nasa_hi
 *   int32   elem[N][E]                      atom counts
 *   float64 sigma[N], eps_k[N]              Lennard-Jones data (informational)
 *   float64 visc_fit[N][5]                  ln(mu_k / Pa s) = sum_n c_n x^n, x = ln(T / 1000 K)
 *   float64 diff_fit[N][N][5]               g_jk = p T^-1.5 / D_jk = sum_n c_n x^n (g_kk = 0)
 *   int32   rtype[R]                        0 elementary, 1 three-body, 2 Troe fall-off
 *   int32   reac[R][3], prod[R][3]          species indices, -1 padded, repeated for nu = 2
 *   float64 A[R], beta[R], Ea[R]            k = A T^beta exp(-Ea / RT) (k_inf for fall-off), SI
 *   float64 A0[R], beta0[R], Ea0[R]         low-pressure limit (fall-off only)
 *   float64 troe[R][4]                      a, T***, T*, T**
 *   float64 eff[R][N]                       third-body efficiencies
 * Limits: 1 <= N <= 64, 1 <= R <= 4096.
 */
typedef struct chem_mech chem_mech;

/* Reads a mechanism file (host path) and uploads its tables to the current
 * device. *out receives a library-owned handle. Returns CHEM_EIO on a bad
 * file, CHEM_EINVAL on a null argument or out-of-range sizes. */
int chem_mech_load(const char *path, chem_mech **out);
/* Same from an in-memory image of the file format above (host bytes). */
int chem_mech_load_bytes(const void *data, size_t nbytes, chem_mech **out);
/* Frees the handle and its device tables (synchronises the device). */
int chem_mech_free(chem_mech *mech);
/* Number of species / reactions of a loaded mechanism (-1 on a null handle). */
int chem_mech_nspecies(const chem_mech *mech);
int chem_mech_nreactions(const chem_mech *mech);

/* ---------------------------------------------------------------------------
 * props_eval -- thermal and transport properties of every cell
 * ---------------------------------------------------------------------------
 * Sec. 2: thermal and transport properties are computed on the GPU each step;
 * Sec. 3.1 names the Hirschfelder-Curtiss mixture-averaged transport model.
 * Per cell: NASA-7 mixture cp (J/kg/K) and h (J/kg); Wilke mixture viscosity
 * mu (Pa s); the conductivity lambda (W/m/K) with Eucken species values and
 * the same Wilke weights; and the mixture-averaged diffusion coefficients
 * D_k = (1 - Y_k) / sum_{j != k} X_j / D_jk (m^2/s), D_jk from the fits.
 *
 * dtype = CHEM_F32 (float arrays) or CHEM_F64 (double arrays) for all of
 * T, p, Y (inputs, [ld], [ld], [N][ld]) and cp, h, mu, lambda ([ld]) and
 * Dk ([N][ld]) (outputs); CHEM_F64_IN_F32 reads double inputs (the FP64
 * state the stepping calls update) and computes and writes in float. Any of the outputs may be NULL to skip it (mu,
 * lambda and Dk together select the transport part). ncells == 0 is a no-op.
 * Every array is 16-byte aligned and ld a multiple of 4 (else CHEM_EINVAL):
 * without transport outputs, in float arithmetic, the state is streamed by
 * 16-byte bulk copies that may read up to 3 cells past ncells (inside ld). If
 * one of those copies never lands (a bounded wait runs out), the affected
 * cells' cp and h are NaN.
 */
int props_eval(const chem_mech *mech, int64_t ncells, int64_t ld, int dtype,
               const void *T, const void *p, const void *Y,
               void *cp, void *h, void *mu, void *lambda, void *Dk, chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * chem_step_stiff -- the plain method: stiff reactor integration over dt
 * ---------------------------------------------------------------------------
 * Sec. 3.1 integrates every composition over dt = 1 us with CVODE; Sec. 4.2
 * calls this direct integration "CPU-DI". Here each cell is an adiabatic
 * constant-pressure reactor, dY_k/dt = W_k wdot_k / rho and
 * dT/dt = -sum_k H_k wdot_k / (rho cp), integrated in FP64 by the embedded
 * L-stable Rosenbrock method Rodas3 (Sandu et al. 1997, 4 stages, order 3(2))
 * with an analytic dense Jacobian, LU with partial pivoting, and the
 * step-size control described by chem_ode_opts.
 *
 * T [ld] and Y [N][ld] (double, device) are updated in place; p [ld] is read.
 * status [ld] (int32, device) receives a CHEM_CELL_* code and nsteps [ld]
 * (int32, device, may be NULL) the number of attempted steps. opts is a host
 * pointer (NULL = defaults below).
 *
 * Scratch: a work-queue counter inside the mechanism handle; two calls with
 * the same handle must not overlap on the device (stream-order them).
 */
typedef struct {
    double rtol;      /* relative tolerance (default 1e-6) */
    double atol_Y;    /* absolute tolerance on mass fractions (default 1e-12) */
    double atol_T;    /* absolute tolerance on temperature, K (default 1e-6) */
    double h0;        /* first trial step, s (default 1e-9; clipped to dt) */
    int32_t max_steps;/* attempted-step limit per cell (default 10000) */
    int32_t mode;     /* CHEM_ODE_FP64 (default) or CHEM_ODE_MIXED */
} chem_ode_opts;

/* Arithmetic of the integrator. CHEM_ODE_FP64: everything in FP64 (the parity
 * setting). CHEM_ODE_MIXED, for loose tolerances (the learned step's fallback
 * and the plain method's throughput setting, rtol 1e-2): the exponentials of
 * the rate constants and the Troe blending are evaluated in FP32 (relative
 * error about 1e-6 on the rates, far below rtol); the matrix I/(h gamma) - J is
 * assembled and LU-factored in FP32 (a Jacobian with FP32 rounding, about 1e-7
 * relative), and each stage solve takes one step of iterative refinement with
 * an FP64 residual r = b - G x, x += G^-1 r, which solves that system to
 * FP64-grade accuracy. The right-hand side's sums, the state update, the error
 * norm and the step-size control stay FP64. It takes rtol >= 1e-5 (the FP32
 * rates' relative noise of about 1e-6 would stall the step control of tighter
 * tolerances); a tighter rtol integrates in FP64. */
enum { CHEM_ODE_FP64 = 0, CHEM_ODE_MIXED = 1 };

/* Fills *o with the defaults listed above. */
void chem_ode_opts_default(chem_ode_opts *o);

int chem_step_stiff(const chem_mech *mech, int64_t ncells, int64_t ld, double dt, const chem_ode_opts *opts,
                    double *T, const double *p, double *Y, int32_t *status, int32_t *nsteps,
                    chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * chem_step_stiff_noalloc -- chem_step_stiff without any device allocation
 * ---------------------------------------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory, or write into library-owned memory, while they
 * step. Examples are a host code that hands out its whole device budget from
 * its own pool and forbids other allocations, and a caller that runs the step
 * in a region where cudaMalloc is not allowed or would synchronise the device.
 * It computes exactly what chem_step_stiff computes, with the same arguments
 * and results. Its only scratch, the work-queue counter, lives in a static
 * 256-byte device array inside the library instead of the mechanism handle;
 * every GPU that loads the library holds that array until the process exits.
 *  - The call allocates nothing and leaves the mechanism handle untouched
 *    (its tables are only read).
 *  - ncells is limited to 2^30 by the 32-bit counter; larger values return
 *    CHEM_EINVAL.
 *  - All calls share the array. Each call clears the counter on its own stream
 *    first, so calls that overlap on the GPU (different streams, or different
 *    host threads on one device) race and must be ordered by the caller.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on the device.
 *  - That address is kept per device index for the life of the process: after
 *    a cudaDeviceReset in the same process it is stale, so do not call this
 *    entry point after resetting the device.
 */
int chem_step_stiff_noalloc(const chem_mech *mech, int64_t ncells, int64_t ld, double dt, const chem_ode_opts *opts,
                            double *T, const double *p, double *Y, int32_t *status, int32_t *nsteps,
                            chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * chem_pasr -- partially stirred reactor scaling of one chemistry step
 * ---------------------------------------------------------------------------
 * Sec. 4.1: the turbulence-chemistry interaction is the PaSR model, in which a
 * cell's reaction rate is scaled by kappa = tau_c / (tau_c + tau_mix); the
 * chemical time tau_c comes from the slowest formation rate of the species and
 * the mixing time tau_mix is the geometric mean of the Taylor and Kolmogorov
 * time scales. Per cell i < ncells (SoA, leading dimension ld):
 *   dY_k/dt  the reactor right-hand side (Sec. 3.1) at (T0, p, Y0), in FP64;
 *   tau_c    max over species k with Y0_k >= y_min and dY_k/dt != 0 of
 *            Y0_k / |dY_k/dt|, or +inf when no species qualifies;
 *   tau_mix  sqrt(tau_taylor * tau_kolmogorov);
 *   kappa    tau_c / (tau_c + tau_mix), or 1 when tau_c is infinite.
 * T0, p, Y0 [N][ld]: the state before the chemistry step (device, read only).
 * tau_taylor, tau_kolmogorov [ncells] (s, device, read only).
 * T, Y (device, may both be NULL): on entry the chemistry step's result at
 * t + dt (chem_step_stiff or chem_step_ann), on exit T0 + kappa (T - T0) and
 * Y0 + kappa (Y - Y0). They must not alias T0, Y0.
 * tau_c, kappa [ncells] (device, FP64, may be NULL): outputs.
 * y_min > 0 (e.g. 1e-6). Errors: CHEM_EINVAL for null inputs, only one of T
 * and Y, misaligned arrays or ncells > ld; CHEM_EUNSUPPORTED for more than 63
 * species or a non-sm_103 device. Asynchronous on stream; allocates nothing.
 */
int chem_pasr(const chem_mech *mech, int64_t ncells, int64_t ld, double y_min, const double *T0, const double *p,
              const double *Y0, const double *tau_taylor, const double *tau_kolmogorov, double *T, double *Y,
              double *tau_c, double *kappa, chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * Random training-data generation (Sec. 3.1, Eq. 1-4 and Table 1)
 * ---------------------------------------------------------------------------
 * The paper widens its flamelet dataset by random perturbations of every base
 * composition and keeps those whose element ratios stay physical (Table 1).
 * chem_hfrd_perturb computes, per state i < n (SoA, leading dimension ld), with
 * the caller's uniform random numbers c in [-1, 1] (device, [3 + N][ld]: rows
 * c_T, c_p, c_bath, then one row per species, the bath's row unused):
 *   T'    = T + alpha c_T (T_max - T_min)                 (Eq. 1)
 *   p'    = p + beta  c_p (p_max - p_min)                 (Eq. 2)
 *   Y'_b  = Y_b + alpha c_bath (Yb_max - Yb_min)          (Eq. 3; b = the bath, N2)
 *   Y'_j  = max(Y_j, 0)^(1 + gamma c_j), j != b           (Eq. 4)
 * and scales the other species to sum to 1 - Y'_b. keep[i] (uint8, device) is
 * 1 when the state is admissible (0 <= Y'_b < 1, T' > 0, p' > 0, some other
 * species left) and H/C, O/N and phi = (2 n_C + n_H / 2) / n_O, from the
 * element moles n_e = sum_k a_ek Y'_k / W_k, lie in the closed Table 1 ranges.
 * T2, p2 [ld] and Y2 [N][ld] (device) receive the perturbed state (for a
 * rejected inadmissible state, Y2 holds the unscaled Eq. 4 values and 0 for
 * the bath). chon (host int32 [4][N]): the atoms of C, H, O and N in each
 * species. Every operation is FP64, rounded as written (no fused multiply-add).
 * Errors: CHEM_EINVAL for null or misaligned arrays or bad sizes.
 *
 * chem_hfrd_blend: the lean-mixing states of Sec. 3.1, linear in T and every
 * Y between endpoint a (s = 0) and endpoint b (s = 1):
 *   T = (1 - s) Ta + s Tb,  Y_k = (1 - s) Ya_k + s Yb_k
 * for s [n] (device), endpoints Ya, Yb [N] (host), outputs T [ld], Y [N][ld].
 */
typedef struct {
    double alpha, beta, gamma;            /* amplitudes of Eq. 1-4 (Sec. 3.1: 0.125, 10, 0.1) */
    double T_min, T_max, p_min, p_max;    /* ranges over the base dataset */
    double Yb_min, Yb_max;                /* bath mass-fraction range over the base dataset */
    double hc_lo, hc_hi, on_lo, on_hi, phi_lo, phi_hi;   /* Table 1: 2.65-4.67, 0.254-0.32, 0.20-1.15 */
} chem_hfrd_params;

/* The paper's alpha, beta, gamma and Table 1; the dataset ranges set to 0. */
void chem_hfrd_params_default(chem_hfrd_params *params);
int chem_hfrd_perturb(const chem_mech *mech, const chem_hfrd_params *params, const int32_t *chon, int64_t n,
                      int64_t ld, const double *T, const double *p, const double *Y, const double *c, double *T2,
                      double *p2, double *Y2, uint8_t *keep, chem_stream_t stream);
int chem_hfrd_blend(int N, int64_t n, int64_t ld, const double *s, double Ta, const double *Ya, double Tb,
                    const double *Yb, double *T, double *Y, chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * chem_dense_bf16 -- one dense layer of the network on the tensor cores
 * ---------------------------------------------------------------------------
 * Sec. 3.2: each hidden layer applies GELU to an affine map of the layer below.
 * Computes, for i < M and n < N,
 *     acc[i][n] = sum_k x[i][k] W[n][k]      (BF16 operands, FP32 accumulation)
 *     act = 0:  y[i][n] = acc + b[n]         (float y)
 *     act = 1:  y[i][n] = GELU(acc + b[n])   (BF16 y; GELU(z) = z Phi(z) to 4e-6 (1 + |z|))
 * x: [M][ldx] BF16, W: [N][ldw] BF16 (row n = output n), b: [N] float or NULL,
 * y: [M][ldy]. ldx and ldw must make rows a multiple of 16 bytes and the bases
 * 16-byte aligned. tile_n selects the output tile width (32, 64, 128, 160, 208
 * or 256; 0 = automatic). err (device int, may be NULL) receives a non-zero
 * code if a pipeline wait timed out (the call then returns without a result).
 */
int chem_dense_bf16(int64_t M, int N, int K, const void *x, int64_t ldx, const void *W, int64_t ldw,
                    const float *b, int act, void *y, int64_t ldy, int tile_n, int *err, chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * Learned chemistry (Sec. 3.2)
 * ---------------------------------------------------------------------------
 * The network maps the input x(t) = {T, p, F(Y_1..Y_N)}, F(Y) = (Y^0.1 - 1)/0.1
 * (the Box-Cox map; negative Y clamp to 0), Z-score normalised with training
 * statistics, through three GELU hidden layers (1600, 800, 400 in the paper)
 * to the Z-scored change u*(t) = Y(t + dt) - Y(t) of the N - 1 species other
 * than the bath species (ascending species index). Two forms:
 *  - one multi-output network (ensemble = 0), the default;
 *  - the paper's form (ensemble = 1): one network per output species, each
 *    with the three hidden layers and a single output unit, trained on its own
 *    output (Sec. 3.2, "individual training and prediction ... for each
 *    species"). The G = N - 1 networks run side by side: the first layers as
 *    one GEMM over their stacked weights, the hidden-to-hidden layers as
 *    grouped GEMMs (one launch per layer), the output units as per-network
 *    dot products. Its parameter layout stacks the networks per layer: W of
 *    layer l is [G * out_l][in_l] (network g's rows after network g - 1's), b
 *    is [G * out_l]; with out_3 = 1 the last layer is [G][h3], [G].
 * Layers run on the tensor cores in BF16 with FP32 accumulation; parameters
 * are kept in FP32. The first layer carries its input and its weights as two
 * BF16 terms each (hi = bf16(v), lo = bf16(v - hi)) and multiplies
 * z_hi W_hi + z_lo W_hi + z_hi W_lo, so the state and the first layer's
 * weights enter at about 16 significant bits. The bath species is closed by
 * mass conservation (dY_bath = -sum dY_k).
 */
typedef struct chem_mlp chem_mlp;

typedef struct {
    int32_t n_hidden[3]; /* hidden widths, multiples of 8 (Sec. 3.2: 1600, 800, 400) */
    int32_t chunk;       /* cells per inference chunk (0 = 262144; 65536 for an ensemble): sets the
                            activation workspace (an ensemble keeps G x (h1 + h2 + h3) BF16 per cell) */
    int32_t max_batch;   /* largest training batch (0 = 4096) */
    int32_t ensemble;    /* 0: one multi-output network; 1: one network per output species */
    double dt;           /* the flow step the network predicts, s (Sec. 3.1: 1e-6) */
} chem_mlp_desc;

enum { CHEM_PREC_BF16 = 0, CHEM_PREC_FP8 = 1 };

/* Creates a network for the mechanism's species (inputs N + 2, outputs N - 1)
 * with seeded U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and unit statistics.
 * Allocates all device memory it will use (parameters, Adam moments,
 * inference and training workspaces). */
int chem_mlp_create(const chem_mech *mech, const chem_mlp_desc *desc, uint64_t seed, chem_mlp **out);
int chem_mlp_free(chem_mlp *mlp);
/* widths[5] = {N + 2, h1, h2, h3, N - 1} (per network for an ensemble) */
int chem_mlp_dims(const chem_mlp *mlp, int32_t *widths);
/* Number of networks: 1, or N - 1 for an ensemble; negative on a null handle. */
int chem_mlp_groups(const chem_mlp *mlp);
/* Number of parameters: sum over the 4 layers of out * in + out. */
int64_t chem_mlp_nparams(const chem_mlp *mlp);
/* Host float arrays of chem_mlp_nparams values, layer by layer: W[out][in]
 * row-major then b[out]. set_params also resets the Adam state. get_grads
 * returns the gradients of the last mlp_train_step in the same layout. */
int chem_mlp_set_params(chem_mlp *mlp, const float *host);
int chem_mlp_get_params(const chem_mlp *mlp, float *host);
int chem_mlp_get_grads(const chem_mlp *mlp, float *host);
/* Z-score statistics, host doubles: mu_x, sd_x [N + 2] of the inputs and
 * mu_u, sd_u [N - 1] of the outputs (sd below 1e-12 is replaced by 1). */
int chem_mlp_set_norm(chem_mlp *mlp, const double *mu_x, const double *sd_x, const double *mu_u, const double *sd_u);
int chem_mlp_get_norm(const chem_mlp *mlp, double *mu_x, double *sd_x, double *mu_u, double *sd_u);
/* Computes and sets the statistics (FP64, population standard deviation) of n
 * training pairs: inputs from (T, p, Y) and outputs from u* = Y1 - Y, where Y1
 * [N][ld] is the state after dt (device, SoA). Synchronises the stream. */
int chem_mlp_fit_norm(chem_mlp *mlp, int64_t n, int64_t ld, const double *T, const double *p, const double *Y,
                      const double *Y1, chem_stream_t stream);
/* Normalised network outputs u [ncells][ldu] (float, device) for SoA states. */
int chem_mlp_forward(const chem_mlp *mlp, int64_t ncells, int64_t ld, const double *T, const double *p,
                     const double *Y, float *u, int64_t ldu, chem_stream_t stream);
/* The same at precision prec: CHEM_PREC_BF16 as chem_mlp_forward, or
 * CHEM_PREC_FP8 (below). CHEM_EINVAL for FP8 without current E4M3 scales. */
int chem_mlp_forward_prec(const chem_mlp *mlp, int prec, int64_t ncells, int64_t ld, const double *T,
                          const double *p, const double *Y, float *u, int64_t ldu, chem_stream_t stream);

/* Reduced-precision inference (no counterpart in the paper, which states no
 * precision). With CHEM_PREC_FP8 the two hidden-to-hidden layers (h1 -> h2,
 * h2 -> h3: about 94 % of the multiply-adds of a 1600/800/400 network) run on
 * FP8-E4M3 operands with FP32 accumulation; the first layer (whose inputs are
 * the state) and the output layer stay BF16. For hidden-to-hidden layer l:
 *   sw_l[n]  = max_k |W_l[n][k]| / 448   (per output row; 1 for a zero row)
 *   Wq_l     = E4M3(W_l[n][k] / sw_l[n]),  h_q = E4M3(h / s_h)
 *   z_l[n]   = (sum_k h_q[k] Wq_l[n][k]) * (sw_l[n] * s_h) + b_l[n]
 * with E4M3 rounding to nearest even, saturating at +-448, and s_h the
 * per-tensor scale of the layer's input activation (s_1 for h1, s_2 for h2).
 * The E4M3 weights are made from the FP32 parameters when scales are set and
 * become stale (FP8 calls fail with CHEM_EINVAL) after set_params, set_norm,
 * fit_norm or a training step; checkpoints do not hold them.
 *
 * chem_mlp_set_fp8_scales: act_scale[2] = {s_1, s_2} (host, positive, finite);
 * quantises the weights; synchronises the device.
 * chem_mlp_calibrate_fp8: s_i = max |h_i| / 448 over the BF16 forward of n
 * cells (device SoA, e.g. the training states), then as set_fp8_scales.
 * chem_mlp_get_fp8_scales: the current {s_1, s_2} (CHEM_EINVAL if none).
 * chem_mlp_get_fp8_weights: layer 1 or 2; Wq [out][in] (host bytes, E4M3
 * codes) and sw [out] (host floats). */
int chem_mlp_set_fp8_scales(chem_mlp *mlp, const float *act_scale);
int chem_mlp_calibrate_fp8(chem_mlp *mlp, int64_t n, int64_t ld, const double *T, const double *p, const double *Y,
                           chem_stream_t stream);
int chem_mlp_get_fp8_scales(const chem_mlp *mlp, float *act_scale);
int chem_mlp_get_fp8_weights(const chem_mlp *mlp, int layer, uint8_t *Wq, float *sw);
/* Checkpoint (host path): statistics, FP32 parameters, Adam moments and step
 * count, with a version header and an FNV-1a checksum. Training resumed from a
 * checkpoint continues bit for bit (training is deterministic). load checks
 * the species against the mechanism and returns CHEM_EIO on a damaged file. */
int chem_mlp_save(const chem_mlp *mlp, const char *path);
int chem_mlp_load(const chem_mech *mech, const char *path, chem_mlp **out);
/* Autotuner (no counterpart in the paper): for each layer, times every
 * compiled output-tile width of the tensor-core GEMM on `rows` rows of the
 * inference workspace (CUDA events, the first launch discarded) and keeps the
 * fastest for chem_step_ann / chem_mlp_forward. tiles_out[4] (host, may be
 * NULL) receives the choice.
 * Synchronises the stream; results are bitwise
 * the same for every tile width. */
int chem_mlp_autotune(chem_mlp *mlp, int64_t rows, int32_t *tiles_out, chem_stream_t stream);
/* Layer fusion of the BF16 forward (no counterpart in the paper). mask is 0
 * or CHEM_FUSE_34 (the default): the last hidden layer and the output layer
 * run as one launch in which h3 is made on chip and multiplied at once by the
 * output weights. It applies to a last hidden layer of 400 units and at most
 * 32 outputs; the results are bitwise those of the two separate layers. Where
 * it does not apply, and for E4M3, training and the per-species ensemble, the
 * layers run one by one. chem_mlp_autotune times the fused launch against its
 * two layers and keeps the faster. chem_mlp_get_fusion returns the mask the
 * forward uses. */
enum { CHEM_FUSE_34 = 2 };
int chem_mlp_set_fusion(chem_mlp *mlp, int mask);
int chem_mlp_get_fusion(const chem_mlp *mlp);
/* Sticky error word of the network's pipeline waits (0 = none); synchronises the device.
 * Codes: 1 a k-block's operands did not arrive, 2 a pipeline stage was not
 * released, 3 an accumulator was not completed, 4 an accumulator was not
 * released (the tensor-core GEMM's producer, MMA and epilogue roles), 5 a
 * closing drain did not finish. After a non-zero code the network's results
 * are undefined; the word stays set for the life of the handle. */
int chem_mlp_error(const chem_mlp *mlp, int *host_err);
/* Bounded waits (no counterpart in the paper; a failure-detection aid). Every
 * wait of the network's tensor-core pipeline is a loop of at most `tries`
 * mbarrier try_wait operations (0 = the default, 2^22, seconds in total);
 * one that runs out records its code in the error word and the kernel
 * unwinds: it waits (always with the default limit) for the copies and
 * tensor-core operations it has issued, frees its tensor memory and returns.
 * A small limit makes waits run out on purpose, to test that path. */
int chem_mlp_set_wait_limit(chem_mlp *mlp, uint32_t tries);

/* ---------------------------------------------------------------------------
 * Out-of-distribution test and stiff fallback of the learned step
 * ---------------------------------------------------------------------------
 * The paper has no such guard: it applies its networks to every cell. Here the
 * network is trusted only where it was trained; other cells go to the plain
 * method (chem_step_stiff's integrator), which is both the fallback and the
 * reference for the network's error.
 * chem_mlp_fit_ood builds, from n training states (T, p, Y; device, SoA), an
 * nbins^3 occupancy grid over the per-cell features
 *     (T, h/R = sum_k (Y_k / W_k) H_k/R, Y_species)        (FP32, NASA-7)
 * spanning the training range plus 5 % on each side. A cell is in the
 * distribution iff its bin lies inside the grid and the 3 x 3 x 3 block of
 * bins around it holds at least min_count training states. The call enables
 * the test (nbins <= 64; synchronises the stream).
 * With the test enabled, chem_step_ann applies the network only to cells in
 * the distribution; the others keep their state and are integrated by the
 * stiff method with the `fallback` options (defaults when NULL), status
 * CHEM_CELL_FALLBACK on success or the stiff error code.
 */
int chem_mlp_fit_ood(chem_mlp *mlp, const chem_mech *mech, int64_t n, int64_t ld, const double *T, const double *p,
                     const double *Y, int32_t species, int32_t nbins, int32_t min_count, chem_stream_t stream);
/* The same test with ngrids (1 or 2) grids, one per feature species
 * species[0..ngrids): a cell stays with the network only if every grid holds
 * it, which catches off-manifold cells that one feature species alone
 * misses. chem_mlp_fit_ood is this call with one grid. */
int chem_mlp_fit_ood_multi(chem_mlp *mlp, const chem_mech *mech, int64_t n, int64_t ld, const double *T,
                           const double *p, const double *Y, const int32_t *species, int32_t ngrids, int32_t nbins,
                           int32_t min_count, chem_stream_t stream);
/* Turns the test on or off (on requires a fitted grid). */
int chem_mlp_set_ood(chem_mlp *mlp, int enable);
/* flags[i] (uint8, device) = 1 when cell i is outside the training distribution. */
int chem_mlp_ood_flags(const chem_mlp *mlp, const chem_mech *mech, int64_t ncells, int64_t ld, const double *T,
                       const double *p, const double *Y, uint8_t *flags, chem_stream_t stream);
/* The first fitted grid's feature ranges lo3[3], hi3[3] (host floats) and settings. */
int chem_mlp_get_ood(const chem_mlp *mlp, float *lo3, float *hi3, int32_t *nbins, int32_t *species,
                     int32_t *min_count);
/* Feature ranges and species of fitted grid `grid` (0 or 1). */
int chem_mlp_get_ood_grid(const chem_mlp *mlp, int32_t grid, float *lo3, float *hi3, int32_t *species);

/* ---------------------------------------------------------------------------
 * chem_step_ann -- the learned method: advance every cell by the network
 * ---------------------------------------------------------------------------
 * Sec. 3.2: the network predicts u*(t) = Y(t + dt) - Y(t) from (T, p, Y). Per
 * cell: dY = sigma_u u + mu_u for the output species, dY_bath = -sum dY,
 * Y' = max(Y + dY, 0) renormalised to sum 1, and T' solves h(T', Y') = h(T, Y)
 * (adiabatic, constant pressure) by Newton iteration on the NASA-7 enthalpy.
 * T [ld], Y [N][ld] (double, device) are updated in place; p [ld] is read.
 * dt must equal the dt the network was created for (CHEM_EINVAL otherwise).
 * prec: CHEM_PREC_BF16, or CHEM_PREC_FP8 after chem_mlp_calibrate_fp8 /
 * chem_mlp_set_fp8_scales. status [ld] (int32, device, may be NULL) receives
 * CHEM_CELL_OK, or for cells outside the network's training distribution (when
 * the test of chem_mlp_fit_ood is enabled) the stiff fallback's code. A cell
 * whose prediction is not finite goes to the fallback too when the test is
 * enabled; without it, the cell keeps its state with CHEM_CELL_NONFINITE.
 * fallback: stiff options for those cells (NULL = defaults).
 */
int chem_step_ann(const chem_mech *mech, const chem_mlp *mlp, int64_t ncells, int64_t ld, double dt, int prec,
                  const chem_ode_opts *fallback, double *T, const double *p, double *Y, int32_t *status,
                  chem_stream_t stream);

/* chem_step_ann followed by the properties of the advanced state (Sec. 2: the
 * per-cell thermal and transport properties the flow solver needs next), with
 * the same results as chem_step_ann then props_eval(CHEM_F64_IN_F32): cp, h,
 * mu, lambda [ld] and Dk [N][ld] (float, device, each may be NULL; 16-byte
 * aligned), in one call on the caller's stream. Errors as chem_step_ann and
 * props_eval. */
int chem_step_ann_props(const chem_mech *mech, const chem_mlp *mlp, int64_t ncells, int64_t ld, double dt, int prec,
                        const chem_ode_opts *fallback, double *T, const double *p, double *Y, int32_t *status,
                        float *cp, float *h, float *mu, float *lambda, float *Dk, chem_stream_t stream);

/* ---------------------------------------------------------------------------
 * mlp_train_step -- one Adam step on the L1 loss of Eq. 5
 * ---------------------------------------------------------------------------
 * L = (1/B) sum_i |u*_i - u_i|_1 on normalised outputs (Sec. 3.2, Eq. 5),
 * gradients by back-propagation through the same tensor-core layers, then
 * Adam (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on the FP32
 * parameters. The batch is rows idx[0..batch) (int32, device) of a training
 * set of SoA pairs with leading dimension ld: the state (T, p, Y) at t and the
 * mass fractions Y1 at t + dt, so the target is u* = Y1 - Y; idx == NULL takes
 * rows 0..batch-1. batch: a multiple of 8, at most max_batch. loss_dev
 * (float, device, may be NULL) receives L. Deterministic: no atomics.
 */
int mlp_train_step(chem_mlp *mlp, int64_t batch, const int32_t *idx, int64_t ld, const double *T, const double *p,
                   const double *Y, const double *Y1, float lr, float *loss_dev, chem_stream_t stream);

/* mlp_train_step in two halves, for data-parallel training (each rank a shard
 * of the batch, one gradient all-reduce per step between them):
 *  - mlp_train_grads: the forward, the loss and the back-propagation of
 *    mlp_train_step (same arguments but lr), leaving dL/dW and dL/db of this
 *    batch in the handle's gradient buffers;
 *  - chem_mlp_grad_buffers: device pointers to those buffers for layer 0..3
 *    (gW: nW floats, the layer's W layout [out][in padded to a multiple of 8];
 *    gb: nb floats), owned by the handle and valid until it is destroyed, so
 *    that a collective can reduce them in place. Padding entries are zero;
 *  - mlp_adam_step: the Adam update of mlp_train_step from the buffers'
 *    current contents.
 * mlp_train_grads then mlp_adam_step on one stream is bitwise mlp_train_step.
 * With the L1 loss of Eq. 5 averaged over the batch, the mean over R ranks of
 * the gradients of R equal shards is the gradient of the whole batch (up to
 * the FP32 order of the sums). */
int mlp_train_grads(chem_mlp *mlp, int64_t batch, const int32_t *idx, int64_t ld, const double *T, const double *p,
                    const double *Y, const double *Y1, float *loss_dev, chem_stream_t stream);
int chem_mlp_grad_buffers(const chem_mlp *mlp, int layer, float **gW, int64_t *nW, float **gb, int64_t *nb);
int mlp_adam_step(chem_mlp *mlp, float lr, chem_stream_t stream);

/* Physics terms of the training loss (Sec. 3.2 adds the principles of
 * mass-fraction unity, energy conservation and heat release to Eq. 5, with no
 * formula or weight; the forms below are this library's reading). For sample
 * i, with r_j = u_j - u*_j on normalised outputs, sd_j the output scales and
 * c_ij = h_k(T_i) - h_bath(T_i) (J/kg; species k of output j; the bath closes
 * sum dY = 0, so its change is folded in):
 *   r_m,i = sum_j sd_j r_j            error of the implied bath change (unity)
 *   r_q,i = -sum_j c_ij sd_j r_j      error of the heat release at T_i,
 *                                     q = -sum_k h_k(T) dY_k (energy and heat release)
 *   L = Eq. 5 + (1/B) sum_i (lam_m |r_m,i| / s_m + lam_q |r_q,i| / s_q)
 * and mlp_train_step descends this L (subgradient sign(0) = 0). Enthalpies are
 * the mechanism's NASA-7 rows in FP32. lam_m = lam_q = 0 (the default) is
 * Eq. 5 alone. Weights >= 0, scales > 0 (CHEM_EINVAL otherwise); non-zero
 * weights on a per-species ensemble return CHEM_EUNSUPPORTED.
 * chem_mlp_fit_physics_scales: s_m = mean_i sum_j |dY*_ij| (the typical
 * composition change; the mean bath change is no scale, since an inert bath
 * such as N2 changes by exactly zero) and s_q = mean_i |sum_j c_ij dY*_ij|
 * over n training pairs (dY* = Y1 - Y of the output species; device SoA), in
 * FP64 with a fixed summation order; host outputs; synchronises the stream. */
int chem_mlp_set_physics_loss(chem_mlp *mlp, double lam_m, double lam_q, double s_m, double s_q);
int chem_mlp_fit_physics_scales(chem_mlp *mlp, int64_t n, int64_t ld, const double *T, const double *Y,
                                const double *Y1, double *s_m, double *s_q, chem_stream_t stream);

/* Opt-in kernel timing (no counterpart in the paper; a measurement aid).
 * chem_prof_enable(1) clears the counters and starts recording CUDA events on
 * the launch stream around the library's kernels (tensor-core GEMMs, the
 * network's prologue and epilogue, props and the stiff integrator);
 * chem_prof_read writes one line per kernel tag:
 * "tag\tlaunches\tmilliseconds\tflops\tbytes\n" (algorithmic flops and bytes
 * where defined: 2 M N K for a GEMM), synchronising on the recorded events.
 * Off by default; timing adds two event records per launch. */
int chem_prof_enable(int on);
int chem_prof_read(char *buf, int64_t buflen);

/* Last error message of the calling thread ("" if none). */
const char *chem_last_error(void);

/* Library build string (compiler, target architecture). */
const char *chem_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CHEMGB_H */
