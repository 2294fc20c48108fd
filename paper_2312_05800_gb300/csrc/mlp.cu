// mlp.cu -- the learned chemistry of Sec. 3.2 on the GPU: the network handle,
// the per-cell prologue (Box-Cox + Z-score -> BF16 rows), the tensor-core
// layers (gemm_*.cu), the per-cell epilogue (de-normalised dY, bath closure,
// clamp + renormalise, T from the conserved enthalpy), and training (L1 loss
// of Eq. 5, backward through the same GEMM kernel, Adam).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gemm_launch.cuh"

namespace chemgb {
int launch_stiff_list(const chem_mech *m, int64_t capacity, int64_t ld, double dt, const chem_ode_opts &o, double *T,
                      const double *p, double *Y, int32_t *status, const int32_t *list, const unsigned int *count,
                      int ok_status, cudaStream_t st);
int props_f64_in_f32(const chem_mech *m, int64_t ncells, int64_t ld, const double *T, const double *p,
                     const double *Y, float *cp, float *h, float *mu, float *lam, float *Dk, cudaStream_t st);
}

namespace chemgb {
namespace {

constexpr int kLayers = 4;
// The first layer's input rows carry three BF16 terms, [z_hi | z_lo | z_hi], against the weight
// rows [W_hi | W_hi | W_lo] (hi = bf16(v), lo = bf16(v - hi)): z W^T to about 2^-16 relative in
// both factors (the z_lo W_lo term, ~2^-18, is dropped). Measured on trained networks, rounding
// the first layer's weights to one BF16 term moved dY by up to 5e-4 relative, the largest single
// rounding point of the forward.
constexpr int kXTerms = 3;
constexpr int kOodMaxBins = 64;
constexpr int kOodMaxGrids = 2;     // grids of the out-of-distribution test (a cell must pass all)
constexpr int kOodBlocks = 512;
constexpr int64_t kFallbackQueue = 8388608;   // cells queued for the stiff fallback before a flush
constexpr float kLambdaBC = 0.1f;     // Box-Cox lambda (Sec. 3.2)
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;
constexpr float kE4M3Max = 448.0f;    // largest finite E4M3 value

inline int64_t pad8(int64_t x) { return (x + 7) & ~int64_t(7); }
inline int64_t pad16(int64_t x) { return (x + 15) & ~int64_t(15); }
// the layers whose operands are E4M3 in the reduced-precision forward: the two
// hidden-to-hidden layers (their inputs are GELU activations, not the state)
inline bool fp8_layer(int l) { return l == 1 || l == 2; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct Layer {
    int in, out;          // logical widths (an ensemble: in per network, out over all networks)
    int gout;             // output width of one network (out / G)
    int kin;              // padded input width (row length of W, multiple of 8)
    int kx;               // forward GEMM K and row length of Wb: kXTerms kin for the first layer
                          // (input and weights as hi + lo BF16 terms), else kin
    int outp;             // padded output width (multiple of 8)
    float *W, *b;         // FP32 master [out][kin], [outp]
    __nv_bfloat16 *Wb;    // BF16 [out][kx] (the first layer: [W_hi | W_hi | W_lo], see kXTerms)
    __nv_bfloat16 *Wt;    // BF16 transposed [in][outp]
    float *mW, *vW, *mb, *vb;   // Adam moments
    float *gW, *gb;       // gradients of the last training step
    int tile;             // forward tile width
    int kin8;             // input width padded to 16 (row length of Wq)
    uint8_t *Wq;          // E4M3 [out][kin8] (hidden-to-hidden layers only)
    float *sw, *cs;       // per-output weight scale; sw x the input activation scale [outp padded to 16]
};

}  // namespace chemgb

struct chem_mlp {
    int N, bath, n_in, n_in_pad, n_out, n_out_pad;
    int ens, G;                             // one network per output (G = n_out networks) or one (G = 1)
    int widths[5];
    int out_species[64];
    double dt;
    int64_t chunk, max_batch;
    chemgb::Layer L[chemgb::kLayers];
    float *mu_x, *isd_x, *mu_u, *sd_u;     // device FP32 Z-score statistics
    int *out_sp_dev;                        // [n_out] species of each output
    double h_mu_x[66], h_sd_x[66], h_mu_u[64], h_sd_u[64];
    // inference workspace
    __nv_bfloat16 *a0, *h[3];
    float *out;
    // training workspace
    __nv_bfloat16 *tx0, *th[3], *tdout, *tdz[3], *tT0, *tT1;
    float *tz[3], *tout, *loss_part;
    int *err;
    // out-of-distribution grid over (T, h/R, Y_s) and the fallback queue
    uint32_t *ood_counts[chemgb::kOodMaxGrids];    // [64^3] each
    uint8_t *ood_mask[chemgb::kOodMaxGrids];       // [64^3] each
    float *ood_range_dev;                          // per grid: lo[3], inv_width[3]
    float ood_lo[chemgb::kOodMaxGrids][3], ood_hi[chemgb::kOodMaxGrids][3];
    int ood_species[chemgb::kOodMaxGrids];
    int ood_nb, ood_kmin, ood_ngrids, ood_fitted, ood_enabled;
    int32_t *fb_queue;                      // [chunk]
    unsigned int *fb_count;
    int32_t *fb_status;                     // [chunk] when the caller passes no status array
    float *ood_part;                        // per-block feature extrema
    int64_t adam_t;
    // reduced-precision forward: E4M3 scales of the activations h1 and h2 (the
    // inputs of the E4M3 layers) and whether the quantised weights are current
    float act_scale[2];
    int fp8_ready;
    unsigned int *amax;                     // [2] calibration maxima (float bits)
    void *blob;
    size_t blob_bytes;
    int device;
    uint64_t seed;
    uint32_t wait_limit;                    // tries of each GEMM pipeline wait (chem_mlp_set_wait_limit)
    int fuse34;                             // layers 3 and 4 of the BF16 forward in one launch (where supported)
    // physics terms of the training loss (chem_mlp_set_physics_loss): weights and scales, and the
    // mechanism's FP32 NASA-7 enthalpy rows [2][N][6] and 1/W [N] for the heat release
    double lam_m, lam_q, s_m, s_q;
    float *nasa_h, *invW;
    float T_mid;
};

namespace chemgb {
namespace {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Rows z = (x - mu) / sigma, x = (T, p, F(Y_1..Y_N)), F(Y) = (max(Y,0)^0.1 - 1)/0.1, each value as
// two BF16 terms z = hi + lo (hi = bf16(z), lo = bf16(z - hi): 16 significant bits, so the state
// reaches the first layer at about 2^-17 relative instead of BF16's 2^-9). Row layout (kXTerms):
// [hi(0 .. n_in_pad) | lo(0 .. n_in_pad) | hi(0 .. n_in_pad)]; padding columns are 0.
__global__ void prologue_kernel(int64_t n, int64_t ld, const double *__restrict__ T, const double *__restrict__ p,
                                const double *__restrict__ Y, const int32_t *__restrict__ idx, int N, int n_in_pad,
                                const float *__restrict__ mu, const float *__restrict__ isd,
                                __nv_bfloat16 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c = idx ? (int64_t)idx[i] : i;
    __nv_bfloat16 *row = out + i * kXTerms * n_in_pad;
    for (int j0 = 0; j0 < n_in_pad; j0 += 8) {
        __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = j0 + u;
            float x;
            if (j == 0) x = (float)T[c];
            else if (j == 1) x = (float)p[c];
            else if (j < N + 2) {
                const float y = fmaxf((float)Y[(int64_t)(j - 2) * ld + c], 0.0f);
                x = (powf(y, kLambdaBC) - 1.0f) * (1.0f / kLambdaBC);
            } else {
                x = 0.0f;
            }
            const float z = (j < N + 2) ? (x - __ldg(mu + j)) * __ldg(isd + j) : 0.0f;
            hi[u] = __float2bfloat16_rn(z);
            lo[u] = __float2bfloat16_rn(z - __bfloat162float(hi[u]));
        }
        *reinterpret_cast<uint4 *>(row + j0) = *reinterpret_cast<const uint4 *>(hi);
        *reinterpret_cast<uint4 *>(row + n_in_pad + j0) = *reinterpret_cast<const uint4 *>(lo);
        *reinterpret_cast<uint4 *>(row + 2 * n_in_pad + j0) = *reinterpret_cast<const uint4 *>(hi);
    }
}

// Out-of-distribution features of one cell (FP32): T, h/R = sum_k (Y_k / W_k) H_k/R, Y_s.
__device__ __forceinline__ void ood_features(const PropTables<float> &tb, int N, float T_mid, int64_t ld, int64_t i,
                                             const double *T, const double *Y, int s, float f[3]) {
    const float t = (float)T[i];
    const int rg = (t >= T_mid) ? 1 : 0;
    float h = 0.0f;
    for (int k = 0; k < N; ++k) {
        const float *b = tb.nasa_h + (rg * N + k) * 6;
        float hh = fmaf(fmaf(fmaf(fmaf(__ldg(b + 4), t, __ldg(b + 3)), t, __ldg(b + 2)), t, __ldg(b + 1)), t, __ldg(b));
        hh = hh * t + __ldg(b + 5);
        h = fmaf((float)Y[(int64_t)k * ld + i] * __ldg(tb.invW + k), hh, h);
    }
    f[0] = t;
    f[1] = h;
    f[2] = (float)Y[(int64_t)s * ld + i];
}

// Bin of a feature vector, or -1 outside the grid range.
__device__ __forceinline__ int ood_bin(const float f[3], const float *range, int nb) {
    int idx = 0;
    for (int d = 0; d < 3; ++d) {
        const float u = (f[d] - range[d]) * range[3 + d];
        if (!(u >= 0.0f) || u >= (float)nb) return -1;
        idx = idx * nb + (int)u;
    }
    return idx;
}

// Per cell: dY_k = sigma_k u_k + mu_k (output species), dY_bath = -sum dY_k,
// Y' = max(Y + dY, 0) renormalised, T' from h(T', Y') = h(T, Y) by Newton.
// dY and the provisional Y' live in FP32 registers (species loops unrolled to
// the compile-time bound NMAX) for the enthalpy Newton iteration; the final
// clamp and renormalisation are FP64 so that sum Y' = 1 to FP64 round-off.
struct OodRoute {
    const float *range;      // per grid lo[3], inv_width[3]; null: no test
    const uint8_t *mask[kOodMaxGrids];
    int species[kOodMaxGrids];
    int ngrids, nb;
    int32_t *queue;          // absolute cell indices (the call's first cell is 0)
    unsigned int *count;
    int64_t base;            // index of this chunk's first cell within the call
};

// true when a cell with features (T, h/R) and the state Y is outside any grid's distribution
__device__ __forceinline__ bool ood_outside(const OodRoute &ood, float T, float h, const double *Y, int64_t ld,
                                            int64_t i) {
    for (int g = 0; g < ood.ngrids; ++g) {
        const float f[3] = {T, h, f64_to_f32_trunc(Y[(int64_t)ood.species[g] * ld + i])};
        const int b = ood_bin(f, ood.range + 6 * g, ood.nb);
        if (b < 0 || ood.mask[g][b] == 0) return true;
    }
    return false;
}

template <int NMAX>
__global__ void __launch_bounds__(128, (NMAX <= 32 ? 8 : 4)) epilogue_kernel(int64_t n, int64_t ld, const float *__restrict__ u, int ldu,
                                                       int N, int bath, const float *__restrict__ mu_u,
                                                       const float *__restrict__ sd_u, PropTables<float> tb,
                                                       float T_mid, double *__restrict__ T, double *__restrict__ Y,
                                                       int32_t *__restrict__ status, OodRoute ood) {
    // per species and range: cp/R coefficients (5), H/R coefficients (6), 1/W -> 3 float4
    __shared__ float4 tab[2 * NMAX * 3];
    // dY per species and thread (column per thread: conflict-free), so that only the provisional
    // Y' stays in registers and the kernel keeps more warps resident
    __shared__ float dyS[NMAX][128];
    for (int e = threadIdx.x; e < 2 * N; e += blockDim.x) {
        const int rg = e / N, k = e % N;
        const float *a = tb.nasa_cp + (rg * N + k) * 5;
        const float *b = tb.nasa_h + (rg * N + k) * 6;
        float4 *o = tab + (rg * NMAX + k) * 3;
        o[0] = make_float4(a[0], a[1], a[2], a[3]);
        o[1] = make_float4(a[4], b[0], b[1], b[2]);
        o[2] = make_float4(b[3], b[4], b[5], tb.invW[k]);
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = threadIdx.x;
    const float *ur = u + i * ldu;
    const float T0 = (float)T[i];
    const int r0 = (T0 >= T_mid) ? 1 : 0;
    float sum = 0.0f, h0 = 0.0f;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        if (k < N) {
            const float y = f64_to_f32_trunc(Y[(int64_t)k * ld + i]);
            float d = 0.0f;
            if (k != bath) {
                const int j = (k < bath) ? k : k - 1;   // outputs: the non-bath species, ascending
                d = fmaf(__ldg(sd_u + j), ur[j], __ldg(mu_u + j));
                sum += d;
            }
            dyS[k][t] = d;
            const float4 *q = tab + (r0 * NMAX + k) * 3;
            const float4 q1 = q[1], q2 = q[2];
            float hh = fmaf(fmaf(fmaf(fmaf(q2.y, T0, q2.x), T0, q1.w), T0, q1.z), T0, q1.y);
            hh = hh * T0 + q2.z;                       // H_k / R
            h0 = fmaf(y * q2.w, hh, h0);
        }
    }
    // a non-finite prediction (non-finite weights or statistics, an overflow) never reaches the
    // state: the sum of the outputs' dY is non-finite exactly when one of them is or they overflow
    const bool bad = !isfinite(sum);
    if (ood.range) {
        // a cell outside the training distribution, or with a non-finite prediction, keeps its
        // state and goes to the stiff integrator
        if (bad || ood_outside(ood, T0, h0, Y, ld, i)) {
            const unsigned int q = atomicAdd(ood.count, 1u);
            ood.queue[q] = (int32_t)(ood.base + i);
            return;
        }
    } else if (bad) {
        if (status) status[i] = CHEM_CELL_NONFINITE;     // without the guard: the state is kept
        return;
    }
    dyS[bath][t] = -sum;
    // Newton on h(T', Y') = h0 with Y' = max(Y + dY, 0) / sum. The mixture's cp/R and H/R are
    // polynomials in T whose coefficients are sum_k (Y'_k / W_k) a_k: formed once per cell for the
    // range in use (again, from the state and dY, only if T' crosses T_mid), so that an iteration
    // is two polynomial evaluations instead of a pass over the species' NASA rows. The provisional
    // Y' is not kept: the state is re-read from cache.
    float mc[5], mh[6];
    auto mix = [&](int rg) {
#pragma unroll
        for (int j = 0; j < 5; ++j) mc[j] = 0.0f;
#pragma unroll
        for (int j = 0; j < 6; ++j) mh[j] = 0.0f;
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k < N) {
                const float y = fmaxf(f64_to_f32_trunc(Y[(int64_t)k * ld + i]) + dyS[k][t], 0.0f);
                s += y;
                const float4 *q = tab + (rg * NMAX + k) * 3;
                const float4 q0 = q[0], q1 = q[1], q2 = q[2];
                const float yw = y * q2.w;
                mc[0] = fmaf(yw, q0.x, mc[0]);
                mc[1] = fmaf(yw, q0.y, mc[1]);
                mc[2] = fmaf(yw, q0.z, mc[2]);
                mc[3] = fmaf(yw, q0.w, mc[3]);
                mc[4] = fmaf(yw, q1.x, mc[4]);
                mh[0] = fmaf(yw, q1.y, mh[0]);
                mh[1] = fmaf(yw, q1.z, mh[1]);
                mh[2] = fmaf(yw, q1.w, mh[2]);
                mh[3] = fmaf(yw, q2.x, mh[3]);
                mh[4] = fmaf(yw, q2.y, mh[4]);
                mh[5] = fmaf(yw, q2.z, mh[5]);
            }
        }
        const float invs = 1.0f / s;
#pragma unroll
        for (int j = 0; j < 5; ++j) mc[j] *= invs;
#pragma unroll
        for (int j = 0; j < 6; ++j) mh[j] *= invs;
    };
    float Tn = T0;
    int rc = -1;
    for (int it = 0; it < 30; ++it) {
        const int rg = (Tn >= T_mid) ? 1 : 0;
        if (rg != rc) {
            mix(rg);
            rc = rg;
        }
        const float c1 = fmaf(fmaf(fmaf(fmaf(mc[4], Tn, mc[3]), Tn, mc[2]), Tn, mc[1]), Tn, mc[0]);
        float h1 = fmaf(fmaf(fmaf(fmaf(mh[4], Tn, mh[3]), Tn, mh[2]), Tn, mh[1]), Tn, mh[0]);
        h1 = fmaf(h1, Tn, mh[5]);
        const float d = (h1 - h0) / c1;        // both in units of R
        Tn -= d;
        if (fabsf(d) < 1e-4f) break;
    }
    // FP64 update, clamp and renormalisation in two passes over the species (the state is
    // re-read from cache): the widening of dY and the clamp test of the sign bit run on the
    // integer pipe, leaving four FP64-pipe instructions per species
    double s64 = 0.0;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        if (k < N) {
            double y = Y[(int64_t)k * ld + i] + f32_to_f64_int(dyS[k][t]);
            if (__double_as_longlong(y) < 0) y = 0.0;
            s64 += y;
        }
    }
    const double inv = 1.0 / s64;
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        if (k < N) {
            double *q = Y + (int64_t)k * ld + i;
            double y = *q + f32_to_f64_int(dyS[k][t]);
            if (__double_as_longlong(y) < 0) y = 0.0;
            *q = y * inv;
        }
    }
    T[i] = (double)Tn;
    if (status) status[i] = CHEM_CELL_OK;
}

// per-block minima and maxima of the three features (fixed-order tree reduction)
__global__ void ood_extrema_kernel(int64_t n, int64_t ld, const double *T, const double *Y, PropTables<float> tb,
                                   int N, float T_mid, int s, float *part) {
    __shared__ float smin[3][256], smax[3][256];
    float mn[3] = {3.4e38f, 3.4e38f, 3.4e38f}, mx[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f[3];
        ood_features(tb, N, T_mid, ld, i, T, Y, s, f);
        for (int d = 0; d < 3; ++d) { mn[d] = fminf(mn[d], f[d]); mx[d] = fmaxf(mx[d], f[d]); }
    }
    for (int d = 0; d < 3; ++d) { smin[d][threadIdx.x] = mn[d]; smax[d][threadIdx.x] = mx[d]; }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int d = 0; d < 3; ++d) {
                smin[d][threadIdx.x] = fminf(smin[d][threadIdx.x], smin[d][threadIdx.x + w]);
                smax[d][threadIdx.x] = fmaxf(smax[d][threadIdx.x], smax[d][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) { part[blockIdx.x * 6 + d] = smin[d][0]; part[blockIdx.x * 6 + 3 + d] = smax[d][0]; }
}

__global__ void ood_hist_kernel(int64_t n, int64_t ld, const double *T, const double *Y, PropTables<float> tb, int N,
                                float T_mid, int s, const float *range, int nb, uint32_t *counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f[3];
        ood_features(tb, N, T_mid, ld, i, T, Y, s, f);
        const int b = ood_bin(f, range, nb);
        if (b >= 0) atomicAdd(counts + b, 1u);
    }
}

// in-distribution mask: the 3 x 3 x 3 neighbourhood of a bin holds >= kmin samples
__global__ void ood_mask_kernel(int nb, int kmin, const uint32_t *counts, uint8_t *mask) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb * nb * nb) return;
    const int i = b / (nb * nb), j = (b / nb) % nb, k = b % nb;
    uint32_t c = 0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
            for (int dk = -1; dk <= 1; ++dk) {
                const int a = i + di, bb = j + dj, cc = k + dk;
                if (a >= 0 && a < nb && bb >= 0 && bb < nb && cc >= 0 && cc < nb) c += counts[(a * nb + bb) * nb + cc];
            }
    mask[b] = (c >= (uint32_t)kmin) ? 1 : 0;
}

__global__ void ood_flags_kernel(int64_t n, int64_t ld, const double *T, const double *Y, PropTables<float> tb, int N,
                                 float T_mid, OodRoute ood, uint8_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[3];
    ood_features(tb, N, T_mid, ld, i, T, Y, ood.species[0], f);
    out[i] = ood_outside(ood, f[0], f[1], Y, ld, i) ? 1 : 0;
}

// Physics terms of the training loss (Sec. 3.2 names mass-fraction unity, energy and heat
// release; the forms are readings): with r_j = u_j - u*_j on normalised outputs, sd_j the output
// scales and c_j = h_k(T) - h_bath(T) (J/kg, species k of output j, the bath closure folded in),
//   r_m = sum_j sd_j r_j              the error of the implied bath change (sum dY = 0)
//   r_q = -sum_j c_j sd_j r_j         the error of the heat release q = -sum_k h_k(T) dY_k
// and the loss adds lam_m |r_m| / s_m + lam_q |r_q| / s_q per sample (then / B).
struct PhysLoss {
    float wm, wq;                 // lam_m / s_m and lam_q / s_q (0: Eq. 5 alone)
    const float *nasa_h;          // [2][N][6] H/RT rows
    const float *invW;            // [N]
    float T_mid;
    int N, bath;
};

// H_k(T) / R (K) from the FP32 NASA-7 row of H/RT coefficients (a1, a2/2, a3/3, a4/4, a5/5, a6)
__device__ __forceinline__ float h_over_R(const float *b, float T) {
    float hh = fmaf(fmaf(fmaf(fmaf(__ldg(b + 4), T, __ldg(b + 3)), T, __ldg(b + 2)), T, __ldg(b + 1)), T, __ldg(b));
    return hh * T + __ldg(b + 5);
}

// L1 loss of Eq. 5 on normalised outputs, dL/du = sign(u - u*)/B, plus the physics terms above
// when their weights are non-zero; dL/du written as BF16, the per-sample loss to part.
__global__ void l1_loss_kernel(int64_t B, const float *__restrict__ u, int ldu, const int32_t *__restrict__ idx,
                               int64_t ld, const double *__restrict__ Y0, const double *__restrict__ Y1, int n_out,
                               const int *__restrict__ out_sp, const float *__restrict__ mu_u,
                               const float *__restrict__ sd_u, __nv_bfloat16 *__restrict__ dout, int lddo,
                               float *__restrict__ part, const double *__restrict__ Tc, PhysLoss ph) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const int64_t c = idx ? (int64_t)idx[i] : i;
    const float invB = 1.0f / (float)B;
    const bool phys = ph.wm != 0.0f || ph.wq != 0.0f;
    float acc = 0.0f, rm = 0.0f, rq = 0.0f, T = 0.0f, hb = 0.0f;
    const float *rows = nullptr;
    if (phys) {
        T = (float)Tc[c];
        rows = ph.nasa_h + (size_t)((T >= ph.T_mid) ? 1 : 0) * ph.N * 6;
        hb = h_over_R(rows + ph.bath * 6, T) * __ldg(ph.invW + ph.bath);
    }
    for (int j = 0; j < n_out; ++j) {
        const int64_t q = (int64_t)out_sp[j] * ld + c;
        const float target = ((float)(Y1[q] - Y0[q]) - __ldg(mu_u + j)) / __ldg(sd_u + j);
        const float d = u[i * ldu + j] - target;
        acc += fabsf(d);
        if (phys) {
            const int k = out_sp[j];
            const float cj = h_over_R(rows + k * 6, T) * __ldg(ph.invW + k) - hb;   // (h_k - h_bath) / R
            rm = fmaf(__ldg(sd_u + j), d, rm);
            rq = fmaf(-cj * __ldg(sd_u + j), d, rq);
        }
    }
    // r_q in J/kg: the enthalpy differences above are in units of R (K mol/kg)
    constexpr float kRf = 8.314462618f;
    rq *= kRf;
    const float sm = (rm > 0.0f) ? 1.0f : ((rm < 0.0f) ? -1.0f : 0.0f);
    const float sq = (rq > 0.0f) ? 1.0f : ((rq < 0.0f) ? -1.0f : 0.0f);
    if (phys) acc += ph.wm * fabsf(rm) + ph.wq * fabsf(rq);
    for (int j = 0; j < lddo; ++j) {
        float g = 0.0f;
        if (j < n_out) {
            const int64_t q = (int64_t)out_sp[j] * ld + c;
            const float target = ((float)(Y1[q] - Y0[q]) - __ldg(mu_u + j)) / __ldg(sd_u + j);
            const float d = u[i * ldu + j] - target;
            g = (d > 0.0f) ? invB : ((d < 0.0f) ? -invB : 0.0f);
            if (phys) {
                const int k = out_sp[j];
                const float cj = (h_over_R(rows + k * 6, T) * __ldg(ph.invW + k) - hb) * kRf;
                g += invB * __ldg(sd_u + j) * (ph.wm * sm - ph.wq * sq * cj);
            }
        }
        dout[i * lddo + j] = __float2bfloat16_rn(g);
    }
    part[i] = acc;
}

// Scales of the physics terms over n training pairs, FP64: per-block sums of sum_j |dY*_j| and
// |sum_j (h_k - h_bath)(T) dY*_j| (dY* = Y1 - Y of the output species), fixed order within a
// block (grid-stride, then a tree), written to part[2 blockIdx.x + {0, 1}].
__global__ void phys_scales_kernel(int64_t n, int64_t ld, const double *__restrict__ T, const double *__restrict__ Y,
                                   const double *__restrict__ Y1, int n_out, const int *__restrict__ out_sp,
                                   PhysLoss ph, double *__restrict__ part) {
    __shared__ double sm[256], sq[256];
    double am = 0.0, aq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float t = (float)T[i];
        const float *rows = ph.nasa_h + (size_t)((t >= ph.T_mid) ? 1 : 0) * ph.N * 6;
        const double hb = (double)(h_over_R(rows + ph.bath * 6, t) * __ldg(ph.invW + ph.bath));
        double m = 0.0, q = 0.0;
        for (int j = 0; j < n_out; ++j) {
            const int k = out_sp[j];
            const double d = Y1[(int64_t)k * ld + i] - Y[(int64_t)k * ld + i];
            m += fabs(d);
            q += ((double)(h_over_R(rows + k * 6, t) * __ldg(ph.invW + k)) - hb) * d;
        }
        am += m;
        aq += fabs(q) * 8.314462618;
    }
    sm[threadIdx.x] = am;
    sq[threadIdx.x] = aq;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sm[threadIdx.x] += sm[threadIdx.x + w];
            sq[threadIdx.x] += sq[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sm[0];
        part[2 * blockIdx.x + 1] = sq[0];
    }
}

// the block partials of phys_scales_kernel summed in block order, divided by n
__global__ void phys_scales_reduce_kernel(int nblocks, int64_t n, const double *__restrict__ part,
                                          double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = 0.0, q = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        m += part[2 * b];
        q += part[2 * b + 1];
    }
    out[0] = m / (double)n;
    out[1] = q / (double)n;
}

// Deterministic sum of the per-sample partials (one block, fixed order), then / B.
__global__ void loss_reduce_kernel(int64_t B, const float *__restrict__ part, float *__restrict__ loss) {
    __shared__ float sh[256];
    float a = 0.0f;
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = sh[0] / (float)B;
}

// Column sums of a BF16 [B][ld] matrix (bias gradients) in a fixed order: block (32 columns x
// kColsumRows row groups); thread (x, y) sums rows y, y + kColsumRows, ... of its column, then
// thread y = 0 adds the groups' partial sums in ascending y. Deterministic, and every thread has
// many independent loads in flight.
constexpr int kColsumRows = 16;
__global__ void __launch_bounds__(32 * kColsumRows) colsum_kernel(int64_t B, int ncol, const __nv_bfloat16 *__restrict__ g,
                                                                  int ldg, float *__restrict__ out) {
    __shared__ float part[kColsumRows][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (j < ncol) {
#pragma unroll 8
        for (int64_t i = threadIdx.y; i < B; i += kColsumRows) s += __bfloat162float(g[i * ldg + j]);
    }
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && j < ncol) {
        float t = 0.0f;
        for (int y = 0; y < kColsumRows; ++y) t += part[y][threadIdx.x];
        out[j] = t;
    }
}

// out[c][r] = in[r][c] for a BF16 [rows][cols] matrix (row strides ldi, ldo), 32x32 tiles.
__global__ void transpose_kernel(int rows, int cols, const __nv_bfloat16 *__restrict__ in, int64_t ldi,
                                 __nv_bfloat16 *__restrict__ out, int64_t ldo) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < rows && c < cols) ? in[(int64_t)r * ldi + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(int64_t)c * ldo + r] = t[threadIdx.x][k];
    }
}

// Adam (Kingma and Ba 2015) on one layer; refreshes the BF16 and transposed BF16 copies.
__global__ void adam_kernel(int out, int in, int kin, int kx, int outp, float *__restrict__ W, float *__restrict__ b,
                            const float *__restrict__ gW, const float *__restrict__ gb, float *__restrict__ mW,
                            float *__restrict__ vW, float *__restrict__ mb, float *__restrict__ vb,
                            __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Wt, float lr, float bc1,
                            float bc2) {
    const int64_t nW = (int64_t)out * in;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nW) {
        const int o = (int)(t / in), k = (int)(t % in);
        const int64_t q = (int64_t)o * kin + k;
        const float g = gW[q];
        const float m = kAdamB1 * mW[q] + (1.0f - kAdamB1) * g;
        const float v = kAdamB2 * vW[q] + (1.0f - kAdamB2) * g * g;
        mW[q] = m;
        vW[q] = v;
        const float w = W[q] - lr * (m / bc1) / (sqrtf(v / bc2) + kAdamEps);
        W[q] = w;
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        Wb[(int64_t)o * kx + k] = wb;
        if (kx != kin) {                                      // the first layer: [W_hi | W_hi | W_lo]
            Wb[(int64_t)o * kx + kin + k] = wb;
            Wb[(int64_t)o * kx + 2 * kin + k] = __float2bfloat16_rn(w - __bfloat162float(wb));
        }
        Wt[(int64_t)k * outp + o] = wb;
    } else if (t < nW + out) {
        const int o = (int)(t - nW);
        const float g = gb[o];
        const float m = kAdamB1 * mb[o] + (1.0f - kAdamB1) * g;
        const float v = kAdamB2 * vb[o] + (1.0f - kAdamB2) * g * g;
        mb[o] = m;
        vb[o] = v;
        b[o] = b[o] - lr * (m / bc1) / (sqrtf(v / bc2) + kAdamEps);
    }
}

// FP32 master -> BF16 copies (after set_params).
__global__ void refresh_bf16_kernel(int out, int in, int kin, int kx, int outp, const float *__restrict__ W,
                                    __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Wt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)out * kin) return;
    const int o = (int)(t / kin), k = (int)(t % kin);
    const float w = k < in ? W[t] : 0.0f;
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    Wb[(int64_t)o * kx + k] = wb;
    if (kx != kin) {                                          // the first layer: [W_hi | W_hi | W_lo]
        Wb[(int64_t)o * kx + kin + k] = wb;
        Wb[(int64_t)o * kx + 2 * kin + k] = __float2bfloat16_rn(w - __bfloat162float(wb));
    }
    if (k < in) Wt[(int64_t)k * outp + o] = wb;
}

// Mean and population standard deviation of feature f over n samples, FP64,
// two passes, one block per feature (fixed reduction order).
__global__ void norm_stats_kernel(int64_t n, int64_t ld, const double *__restrict__ T, const double *__restrict__ p,
                                  const double *__restrict__ Y, const double *__restrict__ Y1, int N, int n_in,
                                  const int *__restrict__ out_sp, double *__restrict__ mean, double *__restrict__ sd) {
    __shared__ double sh[256];
    const int f = blockIdx.x;
    auto feat = [&](int64_t i) -> double {
        if (f == 0) return T[i];
        if (f == 1) return p[i];
        if (f < n_in) {
            const double y = fmax(Y[(int64_t)(f - 2) * ld + i], 0.0);
            return (pow(y, 0.1) - 1.0) / 0.1;
        }
        const int64_t q = (int64_t)out_sp[f - n_in] * ld + i;
        return Y1[q] - Y[q];
    };
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += feat(i);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double m = sh[0] / (double)n;
    __syncthreads();
    a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = feat(i) - m;
        a += d * d;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[f] = m;
        sd[f] = sqrt(sh[0] / (double)n);
    }
}

// ---------------------------------------------------------------------------
// E4M3 weights of a hidden-to-hidden layer, one block per output row n:
// sw[n] = max_k |W[n][k]| / 448 (1 for an all-zero row), Wq[n][k] = E4M3(W[n][k] / sw[n])
// rounded to nearest even with saturation, zero padding up to kin8, cs[n] = sw[n] * s_in.
__global__ void quant_rows_kernel(int in, int kin, int kin8, const float *__restrict__ W, uint8_t *__restrict__ Wq,
                                  float *__restrict__ sw, float *__restrict__ cs, float s_in) {
    __shared__ float red[32];
    const int n = blockIdx.x;
    const float *w = W + (int64_t)n * kin;
    float a = 0.0f;
    for (int k = threadIdx.x; k < in; k += blockDim.x) a = fmaxf(a, fabsf(w[k]));
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (warp == 0) {
        a = lane < nw ? red[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        if (lane == 0) red[0] = a;
    }
    __syncthreads();
    a = red[0];
    const float sc = a > 0.0f ? __fdiv_rn(a, kE4M3Max) : 1.0f;
    for (int k = threadIdx.x; k < kin8; k += blockDim.x)
        Wq[(int64_t)n * kin8 + k] = k < in ? __nv_cvt_float_to_fp8(__fdiv_rn(w[k], sc), __NV_SATFINITE, __NV_E4M3) : 0;
    if (threadIdx.x == 0) {
        sw[n] = sc;
        cs[n] = __fmul_rn(sc, s_in);
    }
}

// max |h| over rows [0, rows) x columns [0, cols) of a BF16 activation matrix, into *amax (float bits;
// the maximum of non-negative floats is the maximum of their bit patterns)
__global__ void amax_bf16_kernel(int64_t rows, int cols, int64_t ld, const __nv_bfloat16 *__restrict__ h,
                                 unsigned int *amax) {
    float a = 0.0f;
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols, c = e - r * cols;
        a = fmaxf(a, fabsf(__bfloat162float(h[r * ld + c])));
    }
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(a));
}

// ---------------------------------------------------------------------------
// output units of the per-species ensemble (Sec. 3.2: each network ends in one
// unit). Network g's last hidden layer is columns [g K, (g + 1) K) of h.
// ---------------------------------------------------------------------------

// u[i][g] = b[g] + sum_k W[g][k] h[i][g K + k]: one warp per (row, network), BF16 operands as the
// tensor-core layers store them, FP32 lane sums over 8-element slices, then a fixed butterfly.
// K % 8 == 0 and 16-byte aligned rows (K, ldh, ldw multiples of 8).
__global__ void group_dot_kernel(int64_t rows, int G, int K, const __nv_bfloat16 *__restrict__ h, int64_t ldh,
                                 const __nv_bfloat16 *__restrict__ W, int ldw, const float *__restrict__ b,
                                 float *__restrict__ u, int ldu) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= rows * G) return;                     // warp-uniform
    const int64_t i = w / G;
    const int g = (int)(w - i * G);
    const __nv_bfloat16 *hr = h + i * ldh + (int64_t)g * K;
    const __nv_bfloat16 *wr = W + (int64_t)g * ldw;
    float s = 0.0f;
    for (int k = lane * 8; k < K; k += 256) {
        const uint4 hv = *reinterpret_cast<const uint4 *>(hr + k);
        const uint4 wv = __ldg(reinterpret_cast<const uint4 *>(wr + k));
        const __nv_bfloat162 *hp = reinterpret_cast<const __nv_bfloat162 *>(&hv);
        const __nv_bfloat162 *wp = reinterpret_cast<const __nv_bfloat162 *>(&wv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 a = __bfloat1622float2(hp[j]), c = __bfloat1622float2(wp[j]);
            s = fmaf(a.x, c.x, s);
            s = fmaf(a.y, c.y, s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[i * ldu + g] = s + __ldg(b + g);
}

// backward of the output units: dz[i][g K + k] = bf16(dout[i][g] W[g][k] GELU'(z[i][g K + k]))
__global__ void group_dot_back_kernel(int64_t rows, int G, int K, const __nv_bfloat16 *__restrict__ dout, int lddo,
                                      const __nv_bfloat16 *__restrict__ W, int ldw, const float *__restrict__ z,
                                      int64_t ldz, __nv_bfloat16 *__restrict__ dz, int64_t lddz) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cols = (int64_t)G * K;
    if (t >= rows * cols) return;
    const int64_t i = t / cols;
    const int c = (int)(t - i * cols);
    const int g = c / K, k = c - g * K;
    const float d = __bfloat162float(dout[i * lddo + g]) * __bfloat162float(W[(int64_t)g * ldw + k]);
    dz[i * lddz + c] = __float2bfloat16_rn(d * gelu_grad(z[i * ldz + c]));
}

// weight gradient of the output units: gW[g][k] = sum_i dout[i][g] h[i][g K + k], rows in order
__global__ void __launch_bounds__(32 * kColsumRows) group_dot_wgrad_kernel(int64_t rows, int G, int K,
                                                                           const __nv_bfloat16 *__restrict__ dout,
                                                                           int lddo, const __nv_bfloat16 *__restrict__ h,
                                                                           int64_t ldh, float *__restrict__ gW, int ldgw) {
    // rows split over kColsumRows groups (thread y sums rows y, y + kColsumRows, ...), partial sums
    // added in ascending y: a fixed order
    __shared__ float part[kColsumRows][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float s = 0.0f;
    if (c < G * K) {
        const int g = c / K;
#pragma unroll 8
        for (int64_t i = threadIdx.y; i < rows; i += kColsumRows)
            s = fmaf(__bfloat162float(dout[i * lddo + g]), __bfloat162float(h[i * ldh + c]), s);
    }
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < G * K) {
        float t = 0.0f;
        for (int y = 0; y < kColsumRows; ++y) t += part[y][threadIdx.x];
        const int g = c / K, k = c - g * K;
        gW[(int64_t)g * ldgw + k] = t;
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int upload_norm(chem_mlp *m) {
    std::vector<float> mx(m->n_in_pad, 0.f), ix(m->n_in_pad, 0.f), mu(m->n_out_pad, 0.f), su(m->n_out_pad, 1.f);
    for (int j = 0; j < m->n_in; ++j) {
        mx[j] = (float)m->h_mu_x[j];
        ix[j] = (float)(1.0 / m->h_sd_x[j]);
    }
    for (int j = 0; j < m->n_out; ++j) {
        mu[j] = (float)m->h_mu_u[j];
        su[j] = (float)m->h_sd_u[j];
    }
    int rc = check_cuda(cudaMemcpy(m->mu_x, mx.data(), mx.size() * 4, cudaMemcpyHostToDevice), "norm upload");
    if (!rc) rc = check_cuda(cudaMemcpy(m->isd_x, ix.data(), ix.size() * 4, cudaMemcpyHostToDevice), "norm upload");
    if (!rc) rc = check_cuda(cudaMemcpy(m->mu_u, mu.data(), mu.size() * 4, cudaMemcpyHostToDevice), "norm upload");
    if (!rc) rc = check_cuda(cudaMemcpy(m->sd_u, su.data(), su.size() * 4, cudaMemcpyHostToDevice), "norm upload");
    return rc;
}

int64_t param_count(const chem_mlp *m) {
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)m->L[l].out * m->L[l].in + m->L[l].out;
    return n;
}

// host params (layer-major: W[out][in] row-major, then b[out]) <-> device master (padded rows)
int copy_params(const chem_mlp *m, float *host, bool to_host, bool grads) {
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        const Layer &L = m->L[l];
        float *W = grads ? L.gW : L.W;
        float *b = grads ? L.gb : L.b;
        cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
        int rc = check_cuda(to_host ? cudaMemcpy2D(host + off, L.in * 4, W, L.kin * 4, L.in * 4, L.out, kind)
                                    : cudaMemcpy2D(W, L.kin * 4, host + off, L.in * 4, L.in * 4, L.out, kind),
                            "parameter copy");
        if (rc) return rc;
        off += (int64_t)L.out * L.in;
        rc = check_cuda(to_host ? cudaMemcpy(host + off, b, L.out * 4, kind) : cudaMemcpy(b, host + off, L.out * 4, kind),
                        "parameter copy");
        if (rc) return rc;
        off += L.out;
    }
    return CHEM_OK;
}

int refresh_bf16(chem_mlp *m, cudaStream_t st) {
    for (int l = 0; l < kLayers; ++l) {
        const Layer &L = m->L[l];
        int64_t n = (int64_t)L.out * L.kin;
        refresh_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L.out, L.in, L.kin, L.kx, L.outp, L.W, L.Wb,
                                                                          L.Wt);
    }
    return check_cuda(cudaGetLastError(), "refresh_bf16");
}

int check_state_args(int64_t ncells, int64_t ld, const void *T, const void *p, const void *Y, const char *who) {
    if (ncells < 0 || ld < ncells || (ld & 3) != 0 || ncells > 0x7fffffff)
        return set_error(CHEM_EINVAL, std::string(who) + ": need 0 <= ncells <= ld < 2^31, ld a multiple of 4");
    if (ncells > 0 && (!T || !p || !Y)) return set_error(CHEM_EINVAL, std::string(who) + ": null state array");
    if ((T && !aligned16(T)) || (p && !aligned16(p)) || (Y && !aligned16(Y)))
        return set_error(CHEM_EINVAL, std::string(who) + ": arrays must be 16-byte aligned");
    return CHEM_OK;
}

// Hidden layer l >= 1 of the ensemble on n rows: G grouped products, network g's input columns
// [g in, (g + 1) in) of x (row stride G in), its stacked weight rows [g gout, (g + 1) gout),
// output columns [g gout, (g + 1) gout) of y; pre (optional) the FP32 pre-activations.
int ens_hidden(const chem_mlp *m, int l, int bn, int n, const __nv_bfloat16 *x, __nv_bfloat16 *y, float *pre,
               cudaStream_t st) {
    const Layer &L = m->L[l];
    const GemmOperand X{x, (int64_t)m->G * L.in, kMapColGrp, L.in};
    const GemmOperand W{L.Wb, L.kx, kMapRowGrp, (int64_t)L.gout * L.kx};
    return gemm_gelu_grouped(bn, X, W, m->G, n, L.gout, L.in, L.b, L.gout, y, L.out, L.gout, pre, L.out, L.gout,
                             m->err, st);
}

// the ensemble's output units on n rows of h (the last hidden layer of every network)
int ens_output(const chem_mlp *m, int64_t n, const __nv_bfloat16 *h, float *u, cudaStream_t st) {
    const Layer &L = m->L[kLayers - 1];
    const int64_t threads = n * m->G * 32;
    void *pb = prof_begin(st);
    group_dot_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, m->G, L.in, h, (int64_t)m->G * L.in, L.Wb,
                                                                        L.kx, L.b, u, m->n_out_pad);
    prof_end(pb, st, "group_dot_kernel", 2.0 * n * m->G * L.in, (double)n * (m->G * L.in * 2 + m->G * 4));
    return check_cuda(cudaGetLastError(), "ensemble output units");
}

// the training loss's physics terms as the loss kernel takes them (zero weights: Eq. 5 alone)
PhysLoss phys_loss(const chem_mlp *m) {
    PhysLoss p{};
    p.wm = (float)(m->lam_m / m->s_m);
    p.wq = (float)(m->lam_q / m->s_q);
    p.nasa_h = m->nasa_h;
    p.invW = m->invW;
    p.T_mid = m->T_mid;
    p.N = m->N;
    p.bath = m->bath;
    return p;
}

// whether the BF16 forward runs layers 1 and 2 as one fused launch (multi-output network, the
// first layer's K of 64 and widths the fused kernel takes)
// the same for layers 3 and 4 (the last hidden layer and the output layer)
bool fused34_on(const chem_mlp *m) {
    return m->fuse34 && !m->ens && fused34_supported(m->L[2].kx, m->L[2].out, m->L[3].out);
}

// prologue + the first nlayers layers on cells [0, n) of the given SoA pointers; with all four,
// the normalised outputs are in m->out. prec CHEM_PREC_FP8 runs the hidden-to-hidden layers on
// E4M3 operands: h1 and h2 are stored as E4M3 (scales act_scale) in the buffers of h[0] and h[1],
// h3 as BF16 for the BF16 output layer.
int forward_chunk(const chem_mlp *m, int64_t n, int64_t ld, const double *T, const double *p, const double *Y,
                  cudaStream_t st, int prec = CHEM_PREC_BF16, int nlayers = kLayers) {
    WaitLimitScope wl(m->wait_limit);
    void *pb = prof_begin(st);
    prologue_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, ld, T, p, Y, nullptr, m->N, m->n_in_pad, m->mu_x,
                                                                 m->isd_x, m->a0);
    prof_end(pb, st, "prologue_kernel", 0.0, (double)n * ((m->N + 2) * 8 + m->n_in_pad * 2 * kXTerms));
    int rc = check_cuda(cudaGetLastError(), "prologue");
    if (rc) return rc;
    const void *x = m->a0;
    int64_t ldx = kXTerms * m->n_in_pad;
    if (m->ens) {
        // the G first layers read the same input: one GEMM over their stacked weights
        const Layer &L0 = m->L[0];
        rc = gemm_gelu(L0.tile, x, ldx, L0.Wb, L0.kx, (int)n, L0.out, L0.kx, L0.b, m->h[0], L0.out, nullptr, 0, m->err,
                       st);
        for (int l = 1; l < 3 && l < nlayers && !rc; ++l)
            rc = ens_hidden(m, l, m->L[l].tile, (int)n, m->h[l - 1], m->h[l], nullptr, st);
        if (rc || nlayers < kLayers) return rc;
        return ens_output(m, n, m->h[2], m->out, st);
    }
    // layers 3 and 4 in one launch: h3 stays on chip, the outputs are written
    const bool f34 = prec == CHEM_PREC_BF16 && nlayers == kLayers && fused34_on(m);
    for (int l = 0; l < (f34 ? 2 : 3) && l < nlayers; ++l) {
        const Layer &L = m->L[l];
        if (prec == CHEM_PREC_FP8) {
            const bool f8in = fp8_layer(l), f8out = fp8_layer(l + 1);
            const int64_t ldo = f8out ? m->L[l + 1].kin8 : L.out;
            const float inv_so = f8out ? 1.0f / m->act_scale[l] : 1.0f;
            rc = gemm_gelu_q(f8in, f8out, L.tile, x, ldx, f8in ? (const void *)L.Wq : (const void *)L.Wb,
                             f8in ? L.kin8 : L.kx, (int)n, L.out, f8in ? L.in : L.kx, L.b, L.cs, m->h[l], ldo,
                             inv_so, m->err, st);
            ldx = ldo;
        } else {
            rc = gemm_gelu(L.tile, x, ldx, L.Wb, L.kx, (int)n, L.out, L.kx, L.b, m->h[l], L.out, nullptr, 0, m->err,
                           st);
            ldx = L.out;
        }
        if (rc) return rc;
        x = m->h[l];
    }
    if (nlayers < kLayers) return CHEM_OK;
    if (f34) {
        const Layer &L3 = m->L[2], &L4 = m->L[3];
        return gemm_fused34(x, ldx, L3.kx, L3.Wb, L3.kx, L4.Wb, L4.kx, (int)n, L3.out, L4.out, L3.b, L4.b, m->out,
                            m->n_out_pad, m->err, st);
    }
    const Layer &L = m->L[3];
    return gemm_linear(L.tile, x, ldx, L.Wb, L.kx, (int)n, L.out, L.kx, L.b, m->out, m->n_out_pad, m->err, st);
}

// E4M3 weights and scales of the hidden-to-hidden layers from the FP32 masters and act_scale
int quantize_fp8(chem_mlp *m, cudaStream_t st) {
    for (int l = 0; l < kLayers; ++l) {
        if (!fp8_layer(l)) continue;
        Layer &L = m->L[l];
        quant_rows_kernel<<<L.out, 256, 0, st>>>(L.in, L.kin, L.kin8, L.W, L.Wq, L.sw, L.cs, m->act_scale[l - 1]);
    }
    return check_cuda(cudaGetLastError(), "quantize_fp8");
}

// the fitted grids as the epilogue and flag kernels take them (queue fields unset)
OodRoute ood_route(const chem_mlp *m) {
    OodRoute r{};
    r.range = m->ood_range_dev;
    for (int g = 0; g < kOodMaxGrids; ++g) {
        r.mask[g] = m->ood_mask[g];
        r.species[g] = m->ood_species[g];
    }
    r.ngrids = m->ood_ngrids;
    r.nb = m->ood_nb;
    return r;
}

int check_prec(const chem_mlp *m, int prec, const char *who) {
    if (prec == CHEM_PREC_BF16) return CHEM_OK;
    if (prec != CHEM_PREC_FP8) return set_error(CHEM_EINVAL, std::string(who) + ": unknown precision");
    if (m->ens) return set_error(CHEM_EUNSUPPORTED, std::string(who) + ": the per-species ensemble runs in BF16 only");
    if (!m->fp8_ready)
        return set_error(CHEM_EINVAL, std::string(who) + ": no E4M3 scales for the current parameters (call "
                                                         "chem_mlp_calibrate_fp8 or chem_mlp_set_fp8_scales)");
    return CHEM_OK;
}

}  // namespace
}  // namespace chemgb

using namespace chemgb;

extern "C" int chem_mlp_free(chem_mlp *m);

extern "C" int chem_mlp_create(const chem_mech *mech, const chem_mlp_desc *desc, uint64_t seed, chem_mlp **out) {
    if (!mech || !desc || !out) return set_error(CHEM_EINVAL, "chem_mlp_create: null argument");
    *out = nullptr;
    for (int i = 0; i < 3; ++i)
        if (desc->n_hidden[i] < 8 || desc->n_hidden[i] % 8 != 0 || desc->n_hidden[i] > 8192)
            return set_error(CHEM_EINVAL, "chem_mlp_create: hidden widths must be multiples of 8 in [8, 8192]");
    if (!(desc->dt > 0.0)) return set_error(CHEM_EINVAL, "chem_mlp_create: dt must be positive");
    if (mech->N < 2) return set_error(CHEM_EINVAL, "chem_mlp_create: the mechanism needs at least 2 species");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_create: " + why);
    chem_mlp *m = new chem_mlp();
    m->N = mech->N;
    m->bath = mech->bath;
    m->n_in = mech->N + 2;
    m->n_in_pad = (int)pad8(m->n_in);
    m->n_out = mech->N - 1;
    m->n_out_pad = (int)pad8(m->n_out);
    for (int k = 0, j = 0; k < mech->N; ++k)
        if (k != mech->bath) m->out_species[j++] = k;
    m->dt = desc->dt;
    if (desc->ensemble != 0 && desc->ensemble != 1) {
        delete m;
        return set_error(CHEM_EINVAL, "chem_mlp_create: ensemble must be 0 or 1");
    }
    m->ens = desc->ensemble;
    m->G = m->ens ? m->n_out : 1;
    m->chunk = desc->chunk > 0 ? desc->chunk : (m->ens ? 65536 : 262144);
    m->chunk = (m->chunk + 127) / 128 * 128;
    m->max_batch = desc->max_batch > 0 ? (desc->max_batch + 7) / 8 * 8 : 4096;
    m->seed = seed;
    m->wait_limit = tc::kSpinLimit;
    m->fuse34 = 1;
    m->widths[0] = m->n_in;
    for (int i = 0; i < 3; ++i) m->widths[1 + i] = desc->n_hidden[i];
    m->widths[4] = m->n_out;
    for (int l = 0; l < kLayers; ++l) {
        Layer &L = m->L[l];
        L.in = m->widths[l];
        // an ensemble's layer l stacks G networks' layers: out = G x (one network's out), and a
        // network's output layer has one unit
        L.gout = (m->ens && l == kLayers - 1) ? 1 : m->widths[l + 1];
        L.out = m->ens ? m->G * L.gout : L.gout;
        L.kin = (int)pad8(L.in);
        L.kx = (l == 0) ? kXTerms * L.kin : L.kin;
        L.outp = (int)pad8(L.out);
        L.kin8 = (int)pad16(L.in);
        // an ensemble's grouped layers tile one network's width
        L.tile = default_tile_width((m->ens && l > 0) ? L.gout : L.out);
    }
    for (int j = 0; j < m->n_in; ++j) { m->h_mu_x[j] = 0.0; m->h_sd_x[j] = 1.0; }
    for (int j = 0; j < m->n_out; ++j) { m->h_mu_u[j] = 0.0; m->h_sd_u[j] = 1.0; }
    // one device blob: parameters, optimiser state, statistics, workspaces
    std::vector<std::pair<void **, size_t>> parts;
    for (int l = 0; l < kLayers; ++l) {
        Layer &L = m->L[l];
        size_t w = (size_t)L.out * L.kin, o = (size_t)L.outp;
        parts.push_back({(void **)&L.W, w * 4});
        parts.push_back({(void **)&L.b, o * 4});
        parts.push_back({(void **)&L.Wb, (size_t)L.out * L.kx * 2});
        parts.push_back({(void **)&L.Wt, (size_t)L.in * L.outp * 2});
        parts.push_back({(void **)&L.mW, w * 4});
        parts.push_back({(void **)&L.vW, w * 4});
        parts.push_back({(void **)&L.mb, o * 4});
        parts.push_back({(void **)&L.vb, o * 4});
        parts.push_back({(void **)&L.gW, w * 4});
        parts.push_back({(void **)&L.gb, o * 4});
        if (fp8_layer(l) && !m->ens) {
            parts.push_back({(void **)&L.Wq, (size_t)L.out * L.kin8});
            parts.push_back({(void **)&L.sw, (size_t)pad16(L.out) * 4});
            parts.push_back({(void **)&L.cs, (size_t)pad16(L.out) * 4});
        }
    }
    parts.push_back({(void **)&m->amax, 64});
    parts.push_back({(void **)&m->mu_x, (size_t)m->n_in_pad * 4});
    parts.push_back({(void **)&m->isd_x, (size_t)m->n_in_pad * 4});
    parts.push_back({(void **)&m->mu_u, (size_t)m->n_out_pad * 4});
    parts.push_back({(void **)&m->sd_u, (size_t)m->n_out_pad * 4});
    parts.push_back({(void **)&m->out_sp_dev, (size_t)64 * 4});
    parts.push_back({(void **)&m->err, 64});
    const int64_t C = m->chunk, B = m->max_batch;
    parts.push_back({(void **)&m->a0, (size_t)C * m->n_in_pad * 2 * kXTerms});
    for (int i = 0; i < 3; ++i) parts.push_back({(void **)&m->h[i], (size_t)C * m->L[i].out * 2});
    parts.push_back({(void **)&m->out, (size_t)C * m->n_out_pad * 4});
    int maxw = m->n_in_pad > m->n_out_pad ? m->n_in_pad : m->n_out_pad;
    for (int i = 0; i < 3; ++i) maxw = m->L[i].out > maxw ? m->L[i].out : maxw;
    parts.push_back({(void **)&m->tx0, (size_t)B * m->n_in_pad * 2 * kXTerms});
    for (int i = 0; i < 3; ++i) {
        parts.push_back({(void **)&m->th[i], (size_t)B * m->L[i].out * 2});
        parts.push_back({(void **)&m->tz[i], (size_t)B * m->L[i].out * 4});
        parts.push_back({(void **)&m->tdz[i], (size_t)B * m->L[i].out * 2});
    }
    parts.push_back({(void **)&m->tout, (size_t)B * m->n_out_pad * 4});
    parts.push_back({(void **)&m->tdout, (size_t)B * m->n_out_pad * 2});
    parts.push_back({(void **)&m->tT0, (size_t)B * maxw * 2});
    parts.push_back({(void **)&m->tT1, (size_t)B * maxw * 2});
    parts.push_back({(void **)&m->loss_part, (size_t)B * 4});
    for (int g = 0; g < kOodMaxGrids; ++g) {
        parts.push_back({(void **)&m->ood_counts[g], (size_t)kOodMaxBins * kOodMaxBins * kOodMaxBins * 4});
        parts.push_back({(void **)&m->ood_mask[g], (size_t)kOodMaxBins * kOodMaxBins * kOodMaxBins});
    }
    parts.push_back({(void **)&m->ood_range_dev, 6 * 4 * kOodMaxGrids});
    parts.push_back({(void **)&m->fb_queue, (size_t)(C > kFallbackQueue ? C : kFallbackQueue) * 4});
    parts.push_back({(void **)&m->fb_count, 64});
    parts.push_back({(void **)&m->fb_status, (size_t)C * 4});
    parts.push_back({(void **)&m->ood_part, (size_t)kOodBlocks * 6 * 4});
    parts.push_back({(void **)&m->nasa_h, (size_t)2 * m->N * 6 * 4});
    parts.push_back({(void **)&m->invW, (size_t)m->N * 4});
    size_t total = 0;
    for (auto &pp : parts) total = align256(total) + pp.second;
    total = align256(total);
    void *blob = nullptr;
    int rc = check_cuda(cudaMalloc(&blob, total), "chem_mlp_create: cudaMalloc");
    if (rc) { delete m; return rc; }
    rc = check_cuda(cudaMemset(blob, 0, total), "chem_mlp_create: memset");
    if (rc) { cudaFree(blob); delete m; return rc; }
    size_t off = 0;
    for (auto &pp : parts) {
        off = align256(off);
        *pp.first = static_cast<uint8_t *>(blob) + off;
        off += pp.second;
    }
    m->blob = blob;
    m->blob_bytes = total;
    cudaGetDevice(&m->device);
    rc = check_cuda(cudaMemcpy(m->out_sp_dev, m->out_species, sizeof(int) * m->n_out, cudaMemcpyHostToDevice),
                    "chem_mlp_create: species map");
    if (!rc)
        rc = check_cuda(cudaMemcpy(m->nasa_h, mech->dev.f32.nasa_h, sizeof(float) * 2 * m->N * 6,
                                   cudaMemcpyDeviceToDevice), "chem_mlp_create: enthalpy rows");
    if (!rc)
        rc = check_cuda(cudaMemcpy(m->invW, mech->dev.f32.invW, sizeof(float) * m->N, cudaMemcpyDeviceToDevice),
                        "chem_mlp_create: molar masses");
    m->T_mid = (float)mech->T_mid;
    m->lam_m = m->lam_q = 0.0;
    m->s_m = m->s_q = 1.0;
    // seeded U(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation (splitmix64 stream)
    std::vector<float> host(param_count(m));
    uint64_t s = seed;
    int64_t q = 0;
    for (int l = 0; l < kLayers; ++l) {
        const double a = 1.0 / std::sqrt((double)m->L[l].in);
        for (int64_t t = 0; t < (int64_t)m->L[l].out * m->L[l].in + m->L[l].out; ++t) {
            const double r = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            host[q++] = (float)((2.0 * r - 1.0) * a);
        }
    }
    if (!rc) rc = copy_params(m, host.data(), false, false);
    if (!rc) rc = upload_norm(m);
    if (!rc) rc = refresh_bf16(m, 0);
    if (!rc) rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_create");
    if (rc) {
        chem_mlp_free(m);
        return rc;
    }
    *out = m;
    return CHEM_OK;
}

extern "C" int chem_mlp_free(chem_mlp *m) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_free: null handle");
    cudaDeviceSynchronize();
    cudaFree(m->blob);
    delete m;
    return CHEM_OK;
}

extern "C" int chem_mlp_dims(const chem_mlp *m, int32_t *widths) {
    if (!m || !widths) return set_error(CHEM_EINVAL, "chem_mlp_dims: null argument");
    for (int i = 0; i < 5; ++i) widths[i] = m->widths[i];
    return CHEM_OK;
}

extern "C" int64_t chem_mlp_nparams(const chem_mlp *m) { return m ? param_count(m) : -1; }

extern "C" int chem_mlp_groups(const chem_mlp *m) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_groups: null handle");
    return m->G;
}

extern "C" int chem_mlp_set_params(chem_mlp *m, const float *host) {
    if (!m || !host) return set_error(CHEM_EINVAL, "chem_mlp_set_params: null argument");
    int rc = copy_params(m, const_cast<float *>(host), false, false);
    if (rc) return rc;
    for (int l = 0; l < kLayers; ++l) {
        Layer &L = m->L[l];
        cudaMemset(L.mW, 0, (size_t)L.out * L.kin * 4);
        cudaMemset(L.vW, 0, (size_t)L.out * L.kin * 4);
        cudaMemset(L.mb, 0, (size_t)L.outp * 4);
        cudaMemset(L.vb, 0, (size_t)L.outp * 4);
    }
    m->adam_t = 0;
    m->fp8_ready = 0;     // E4M3 weights and activation scales must be redone for new parameters
    rc = refresh_bf16(m, 0);
    if (rc) return rc;
    return check_cuda(cudaDeviceSynchronize(), "chem_mlp_set_params");
}

extern "C" int chem_mlp_get_params(const chem_mlp *m, float *host) {
    if (!m || !host) return set_error(CHEM_EINVAL, "chem_mlp_get_params: null argument");
    int rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_get_params");
    return rc ? rc : copy_params(m, host, true, false);
}

extern "C" int chem_mlp_get_grads(const chem_mlp *m, float *host) {
    if (!m || !host) return set_error(CHEM_EINVAL, "chem_mlp_get_grads: null argument");
    int rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_get_grads");
    return rc ? rc : copy_params(m, host, true, true);
}

extern "C" int chem_mlp_set_norm(chem_mlp *m, const double *mu_x, const double *sd_x, const double *mu_u,
                                 const double *sd_u) {
    if (!m || !mu_x || !sd_x || !mu_u || !sd_u) return set_error(CHEM_EINVAL, "chem_mlp_set_norm: null argument");
    for (int j = 0; j < m->n_in; ++j) {
        m->h_mu_x[j] = mu_x[j];
        m->h_sd_x[j] = (sd_x[j] < 1e-12) ? 1.0 : sd_x[j];
    }
    for (int j = 0; j < m->n_out; ++j) {
        m->h_mu_u[j] = mu_u[j];
        m->h_sd_u[j] = (sd_u[j] < 1e-30) ? 1.0 : sd_u[j];
    }
    m->fp8_ready = 0;     // the activation scales were calibrated under the old statistics
    return upload_norm(m);
}

extern "C" int chem_mlp_get_norm(const chem_mlp *m, double *mu_x, double *sd_x, double *mu_u, double *sd_u) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_get_norm: null handle");
    for (int j = 0; j < m->n_in; ++j) { if (mu_x) mu_x[j] = m->h_mu_x[j]; if (sd_x) sd_x[j] = m->h_sd_x[j]; }
    for (int j = 0; j < m->n_out; ++j) { if (mu_u) mu_u[j] = m->h_mu_u[j]; if (sd_u) sd_u[j] = m->h_sd_u[j]; }
    return CHEM_OK;
}

extern "C" int chem_mlp_fit_norm(chem_mlp *m, int64_t n, int64_t ld, const double *T, const double *p,
                                 const double *Y, const double *Y1, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_fit_norm: null handle");
    int rc = check_state_args(n, ld, T, p, Y, "chem_mlp_fit_norm");
    if (rc) return rc;
    if (n < 2 || !Y1 || !aligned16(Y1)) return set_error(CHEM_EINVAL, "chem_mlp_fit_norm: need n >= 2 and aligned Y1");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nf = m->n_in + m->n_out;
    double *dev = reinterpret_cast<double *>(m->loss_part);   // 2 nf doubles of scratch
    if ((size_t)2 * nf * 8 > (size_t)m->max_batch * 4)
        return set_error(CHEM_EINVAL, "chem_mlp_fit_norm: training batch workspace too small");
    norm_stats_kernel<<<nf, 256, 0, st>>>(n, ld, T, p, Y, Y1, m->N, m->n_in, m->out_sp_dev, dev, dev + nf);
    rc = check_cuda(cudaGetLastError(), "chem_mlp_fit_norm launch");
    if (rc) return rc;
    std::vector<double> h(2 * nf);
    rc = check_cuda(cudaMemcpyAsync(h.data(), dev, 2 * nf * 8, cudaMemcpyDeviceToHost, st), "chem_mlp_fit_norm copy");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "chem_mlp_fit_norm sync");
    if (rc) return rc;
    return chem_mlp_set_norm(m, h.data(), h.data() + nf, h.data() + m->n_in, h.data() + nf + m->n_in);
}

extern "C" int chem_mlp_forward_prec(const chem_mlp *m, int prec, int64_t ncells, int64_t ld, const double *T,
                                     const double *p, const double *Y, float *u, int64_t ldu, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_forward: null handle");
    int rc = check_state_args(ncells, ld, T, p, Y, "chem_mlp_forward");
    if (rc) return rc;
    if ((rc = check_prec(m, prec, "chem_mlp_forward"))) return rc;
    if (ncells == 0) return CHEM_OK;
    if (!u || ldu < m->n_out) return set_error(CHEM_EINVAL, "chem_mlp_forward: null u or ldu < n_out");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int64_t c0 = 0; c0 < ncells; c0 += m->chunk) {
        const int64_t n = (ncells - c0 < m->chunk) ? ncells - c0 : m->chunk;
        rc = forward_chunk(m, n, ld, T + c0, p + c0, Y + c0, st, prec);
        if (rc) return rc;
        rc = check_cuda(cudaMemcpy2DAsync(u + c0 * ldu, ldu * 4, m->out, m->n_out_pad * 4, m->n_out * 4, n,
                                          cudaMemcpyDeviceToDevice, st), "chem_mlp_forward copy");
        if (rc) return rc;
    }
    return CHEM_OK;
}

extern "C" int chem_mlp_forward(const chem_mlp *m, int64_t ncells, int64_t ld, const double *T, const double *p,
                                const double *Y, float *u, int64_t ldu, chem_stream_t stream) {
    return chem_mlp_forward_prec(m, CHEM_PREC_BF16, ncells, ld, T, p, Y, u, ldu, stream);
}

extern "C" int chem_mlp_set_fp8_scales(chem_mlp *m, const float *act_scale) {
    if (!m || !act_scale) return set_error(CHEM_EINVAL, "chem_mlp_set_fp8_scales: null argument");
    if (m->ens) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_set_fp8_scales: the ensemble runs in BF16 only");
    for (int i = 0; i < 2; ++i)
        if (!(act_scale[i] > 0.0f) || !std::isfinite(act_scale[i]))
            return set_error(CHEM_EINVAL, "chem_mlp_set_fp8_scales: scales must be positive and finite");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_set_fp8_scales: " + why);
    m->act_scale[0] = act_scale[0];
    m->act_scale[1] = act_scale[1];
    int rc = quantize_fp8(m, 0);
    if (!rc) rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_set_fp8_scales");
    m->fp8_ready = rc == 0;
    return rc;
}

extern "C" int chem_mlp_get_fp8_scales(const chem_mlp *m, float *act_scale) {
    if (!m || !act_scale) return set_error(CHEM_EINVAL, "chem_mlp_get_fp8_scales: null argument");
    if (!m->fp8_ready) return set_error(CHEM_EINVAL, "chem_mlp_get_fp8_scales: not calibrated");
    act_scale[0] = m->act_scale[0];
    act_scale[1] = m->act_scale[1];
    return CHEM_OK;
}

extern "C" int chem_mlp_calibrate_fp8(chem_mlp *m, int64_t n, int64_t ld, const double *T, const double *p,
                                      const double *Y, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_calibrate_fp8: null handle");
    if (m->ens) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_calibrate_fp8: the ensemble runs in BF16 only");
    int rc = check_state_args(n, ld, T, p, Y, "chem_mlp_calibrate_fp8");
    if (rc) return rc;
    if (n == 0) return set_error(CHEM_EINVAL, "chem_mlp_calibrate_fp8: no cells");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_calibrate_fp8: " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    rc = check_cuda(cudaMemsetAsync(m->amax, 0, 2 * sizeof(unsigned int), st), "chem_mlp_calibrate_fp8");
    for (int64_t c0 = 0; c0 < n && !rc; c0 += m->chunk) {
        const int64_t k = (n - c0 < m->chunk) ? n - c0 : m->chunk;
        rc = forward_chunk(m, k, ld, T + c0, p + c0, Y + c0, st, CHEM_PREC_BF16, 2);
        for (int i = 0; i < 2 && !rc; ++i) {
            amax_bf16_kernel<<<1024, 256, 0, st>>>(k, m->L[i].out, m->L[i].out, m->h[i], m->amax + i);
            rc = check_cuda(cudaGetLastError(), "chem_mlp_calibrate_fp8");
        }
    }
    unsigned int bits[2] = {0, 0};
    if (!rc) rc = check_cuda(cudaMemcpyAsync(bits, m->amax, sizeof(bits), cudaMemcpyDeviceToHost, st),
                             "chem_mlp_calibrate_fp8");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "chem_mlp_calibrate_fp8");
    if (rc) return rc;
    float sc[2];
    for (int i = 0; i < 2; ++i) {
        float a;
        std::memcpy(&a, &bits[i], 4);
        if (!(a > 0.0f) || !std::isfinite(a))
            return set_error(CHEM_EINVAL, "chem_mlp_calibrate_fp8: hidden activations are all zero or not finite");
        sc[i] = a / kE4M3Max;
    }
    return chem_mlp_set_fp8_scales(m, sc);
}

extern "C" int chem_mlp_get_fp8_weights(const chem_mlp *m, int layer, uint8_t *Wq, float *sw) {
    if (!m || !Wq || !sw) return set_error(CHEM_EINVAL, "chem_mlp_get_fp8_weights: null argument");
    if (m->ens) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_get_fp8_weights: the ensemble runs in BF16 only");
    if (layer < 0 || layer >= kLayers || !fp8_layer(layer))
        return set_error(CHEM_EINVAL, "chem_mlp_get_fp8_weights: layer has no E4M3 weights (layers 1 and 2 have)");
    if (!m->fp8_ready) return set_error(CHEM_EINVAL, "chem_mlp_get_fp8_weights: not calibrated");
    const Layer &L = m->L[layer];
    int rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_get_fp8_weights");
    if (!rc) rc = check_cuda(cudaMemcpy2D(Wq, L.in, L.Wq, L.kin8, L.in, L.out, cudaMemcpyDeviceToHost),
                             "chem_mlp_get_fp8_weights");
    if (!rc) rc = check_cuda(cudaMemcpy(sw, L.sw, (size_t)L.out * 4, cudaMemcpyDeviceToHost), "chem_mlp_get_fp8_weights");
    return rc;
}

namespace chemgb {
namespace {

// FP32 property outputs of the fused entry point (all null: none)
struct PropsOut {
    float *cp, *h, *mu, *lam, *Dk;
    bool any() const { return cp || h || mu || lam || Dk; }
};

int step_ann_impl(const chem_mech *mech, const chem_mlp *m, int64_t ncells, int64_t ld, double dt, int prec,
                  const chem_ode_opts *fallback, double *T, const double *p, double *Y, int32_t *status,
                  const PropsOut &po, chem_stream_t stream, const char *who) {
    if (!mech || !m) return set_error(CHEM_EINVAL, std::string(who) + ": null handle");
    if (mech->N != m->N || mech->bath != m->bath)
        return set_error(CHEM_EINVAL, std::string(who) + ": network and mechanism disagree on the species");
    if (!(std::fabs(dt - m->dt) <= 1e-12 * m->dt))
        return set_error(CHEM_EINVAL, std::string(who) + ": dt differs from the step the network was trained for");
    int rc = check_state_args(ncells, ld, T, p, Y, who);
    if (rc) return rc;
    if ((rc = check_prec(m, prec, who))) return rc;
    if (ncells == 0) return CHEM_OK;
    if (status && !aligned16(status)) return set_error(CHEM_EINVAL, std::string(who) + ": status must be 16-byte aligned");
    const void *outs[] = {po.cp, po.h, po.mu, po.lam, po.Dk};
    for (const void *q : outs)
        if (q && !aligned16(q)) return set_error(CHEM_EINVAL, std::string(who) + ": outputs must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, std::string(who) + ": " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (m->ood_enabled && !status && ncells > m->chunk)
        return set_error(CHEM_EINVAL, std::string(who) + ": with the out-of-distribution guard, calls of more than "
                                                          "one chunk need a status array");
    const int64_t qcap = m->chunk > kFallbackQueue ? m->chunk : kFallbackQueue;
    chem_ode_opts fo;
    chem_ode_opts_default(&fo);
    if (fallback) fo = *fallback;
    int64_t queued = 0, flush_base = 0;     // cells of chunks routed since the last flush, first cell of them
    // integrates every queued cell in one launch (cells are independent: one launch hides their latencies)
    auto flush = [&](int64_t base) -> int {
        if (!m->ood_enabled || queued == 0) return CHEM_OK;
        int32_t *stq = status ? status + base : m->fb_status;
        void *pf = prof_begin(st);
        int r = launch_stiff_list(mech, queued, ld, dt, fo, T + base, p + base, Y + base, stq, m->fb_queue,
                                  m->fb_count, CHEM_CELL_FALLBACK, st);
        prof_end(pf, st, "stiff_kernel (fallback)", 0.0, 0.0);
        queued = 0;
        return r;
    };
    for (int64_t c0 = 0; c0 < ncells; c0 += m->chunk) {
        const int64_t n = (ncells - c0 < m->chunk) ? ncells - c0 : m->chunk;
        if (m->ood_enabled && queued + n > qcap) {
            if ((rc = flush(flush_base))) return rc;
        }
        rc = forward_chunk(m, n, ld, T + c0, p + c0, Y + c0, st, prec);
        if (rc) return rc;
        OodRoute route{};
        int32_t *st_chunk = status ? status + c0 : m->fb_status;
        if (m->ood_enabled) {
            if (queued == 0) {
                flush_base = c0;
                rc = check_cuda(cudaMemsetAsync(m->fb_count, 0, sizeof(unsigned int), st), "chem_step_ann: queue reset");
                if (rc) return rc;
            }
            route = ood_route(m);
            route.queue = m->fb_queue;
            route.count = m->fb_count;
            route.base = c0 - flush_base;
            queued += n;
        }
        void *pb = prof_begin(st);
        const unsigned eg = (unsigned)((n + 127) / 128);
        if (m->N <= 16)
            epilogue_kernel<16><<<eg, 128, 0, st>>>(n, ld, m->out, m->n_out_pad, m->N, m->bath, m->mu_u, m->sd_u,
                                                    mech->dev.f32, (float)mech->T_mid, T + c0, Y + c0,
                                                    st_chunk, route);
        else if (m->N <= 32)
            epilogue_kernel<32><<<eg, 128, 0, st>>>(n, ld, m->out, m->n_out_pad, m->N, m->bath, m->mu_u, m->sd_u,
                                                    mech->dev.f32, (float)mech->T_mid, T + c0, Y + c0,
                                                    st_chunk, route);
        else
            epilogue_kernel<64><<<eg, 128, 0, st>>>(n, ld, m->out, m->n_out_pad, m->N, m->bath, m->mu_u, m->sd_u,
                                                    mech->dev.f32, (float)mech->T_mid, T + c0, Y + c0,
                                                    st_chunk, route);
        prof_end(pb, st, "epilogue_kernel", 0.0, (double)n * (m->N * 16 + 16 + m->n_out_pad * 4));
        rc = check_cuda(cudaGetLastError(), "chem_step_ann epilogue");
        if (rc) return rc;
    }
    rc = flush(flush_base);
    if (rc || !po.any()) return rc;
    // the properties of the advanced state, after the fallback. (Run beside the fallback on a
    // second stream, they took the issue slots its latency-bound FP64 warps need: measured on
    // GB300, the fallback slowed from 5.5 to 10.8 ms while the properties saved 4 ms.)
    return props_f64_in_f32(mech, ncells, ld, T, p, Y, po.cp, po.h, po.mu, po.lam, po.Dk, st);
}

}  // namespace
}  // namespace chemgb

extern "C" int chem_step_ann(const chem_mech *mech, const chem_mlp *m, int64_t ncells, int64_t ld, double dt, int prec,
                             const chem_ode_opts *fallback, double *T, const double *p, double *Y, int32_t *status,
                             chem_stream_t stream) {
    return step_ann_impl(mech, m, ncells, ld, dt, prec, fallback, T, p, Y, status,
                         PropsOut{nullptr, nullptr, nullptr, nullptr, nullptr}, stream, "chem_step_ann");
}

extern "C" int chem_step_ann_props(const chem_mech *mech, const chem_mlp *m, int64_t ncells, int64_t ld, double dt,
                                   int prec, const chem_ode_opts *fallback, double *T, const double *p, double *Y,
                                   int32_t *status, float *cp, float *h, float *mu, float *lambda, float *Dk,
                                   chem_stream_t stream) {
    return step_ann_impl(mech, m, ncells, ld, dt, prec, fallback, T, p, Y, status,
                         PropsOut{cp, h, mu, lambda, Dk}, stream, "chem_step_ann_props");
}

extern "C" int chem_mlp_fit_ood_multi(chem_mlp *m, const chem_mech *mech, int64_t n, int64_t ld, const double *T,
                                      const double *p, const double *Y, const int32_t *species, int32_t ngrids,
                                      int32_t nbins, int32_t min_count, chem_stream_t stream) {
    if (!m || !mech || !species) return set_error(CHEM_EINVAL, "chem_mlp_fit_ood: null argument");
    int rc = check_state_args(n, ld, T, p, Y, "chem_mlp_fit_ood");
    if (rc) return rc;
    if (ngrids < 1 || ngrids > kOodMaxGrids)
        return set_error(CHEM_EINVAL, "chem_mlp_fit_ood: 1 or 2 grids (feature species)");
    for (int g = 0; g < ngrids; ++g)
        if (species[g] < 0 || species[g] >= m->N) return set_error(CHEM_EINVAL, "chem_mlp_fit_ood: bad species");
    if (n < 1 || nbins < 2 || nbins > kOodMaxBins || min_count < 1)
        return set_error(CHEM_EINVAL, "chem_mlp_fit_ood: need n >= 1, 2 <= nbins <= 64, min_count >= 1");
    if (mech->N != m->N) return set_error(CHEM_EINVAL, "chem_mlp_fit_ood: network and mechanism disagree");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_fit_ood: " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float Tmid = (float)mech->T_mid;
    float range[6 * kOodMaxGrids];
    for (int g = 0; g < ngrids; ++g) {
        ood_extrema_kernel<<<kOodBlocks, 256, 0, st>>>(n, ld, T, Y, mech->dev.f32, m->N, Tmid, species[g], m->ood_part);
        std::vector<float> part(kOodBlocks * 6);
        rc = check_cuda(cudaMemcpyAsync(part.data(), m->ood_part, part.size() * 4, cudaMemcpyDeviceToHost, st),
                        "chem_mlp_fit_ood extrema");
        if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "chem_mlp_fit_ood sync");
        if (rc) return rc;
        float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
        for (int b = 0; b < kOodBlocks; ++b)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::fmin(lo[d], part[b * 6 + d]);
                hi[d] = std::fmax(hi[d], part[b * 6 + 3 + d]);
            }
        for (int d = 0; d < 3; ++d) {
            float w = hi[d] - lo[d];
            if (!(w > 0.0f)) w = std::fmax(std::fabs(lo[d]) * 1e-3f, 1e-30f);
            m->ood_lo[g][d] = lo[d] - 0.05f * w;                 // 5 % margin on both sides
            m->ood_hi[g][d] = hi[d] + 0.05f * w;
            range[6 * g + d] = m->ood_lo[g][d];
            range[6 * g + 3 + d] = (float)nbins / (m->ood_hi[g][d] - m->ood_lo[g][d]);
        }
    }
    rc = check_cuda(cudaMemcpyAsync(m->ood_range_dev, range, sizeof(float) * 6 * ngrids, cudaMemcpyHostToDevice, st),
                    "ood range");
    const int nbins3 = nbins * nbins * nbins;
    for (int g = 0; g < ngrids && !rc; ++g) {
        rc = check_cuda(cudaMemsetAsync(m->ood_counts[g], 0, (size_t)nbins3 * 4, st), "ood reset");
        if (rc) break;
        ood_hist_kernel<<<kOodBlocks, 256, 0, st>>>(n, ld, T, Y, mech->dev.f32, m->N, Tmid, species[g],
                                                    m->ood_range_dev + 6 * g, nbins, m->ood_counts[g]);
        ood_mask_kernel<<<(nbins3 + 255) / 256, 256, 0, st>>>(nbins, min_count, m->ood_counts[g], m->ood_mask[g]);
        rc = check_cuda(cudaGetLastError(), "chem_mlp_fit_ood");
    }
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "chem_mlp_fit_ood sync");
    if (rc) return rc;
    m->ood_nb = nbins;
    m->ood_kmin = min_count;
    m->ood_ngrids = ngrids;
    for (int g = 0; g < ngrids; ++g) m->ood_species[g] = species[g];
    m->ood_fitted = 1;
    m->ood_enabled = 1;
    return CHEM_OK;
}

extern "C" int chem_mlp_fit_ood(chem_mlp *m, const chem_mech *mech, int64_t n, int64_t ld, const double *T,
                                const double *p, const double *Y, int32_t species, int32_t nbins, int32_t min_count,
                                chem_stream_t stream) {
    return chem_mlp_fit_ood_multi(m, mech, n, ld, T, p, Y, &species, 1, nbins, min_count, stream);
}

extern "C" int chem_mlp_set_ood(chem_mlp *m, int enable) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_set_ood: null handle");
    if (enable && !m->ood_fitted) return set_error(CHEM_EINVAL, "chem_mlp_set_ood: fit the grid first");
    m->ood_enabled = enable ? 1 : 0;
    return CHEM_OK;
}

extern "C" int chem_mlp_ood_flags(const chem_mlp *m, const chem_mech *mech, int64_t ncells, int64_t ld,
                                  const double *T, const double *p, const double *Y, uint8_t *flags,
                                  chem_stream_t stream) {
    if (!m || !mech) return set_error(CHEM_EINVAL, "chem_mlp_ood_flags: null handle");
    if (!m->ood_fitted) return set_error(CHEM_EINVAL, "chem_mlp_ood_flags: fit the grid first");
    int rc = check_state_args(ncells, ld, T, p, Y, "chem_mlp_ood_flags");
    if (rc) return rc;
    if (ncells == 0) return CHEM_OK;
    if (!flags) return set_error(CHEM_EINVAL, "chem_mlp_ood_flags: null flags");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ood_flags_kernel<<<(unsigned)((ncells + 255) / 256), 256, 0, st>>>(ncells, ld, T, Y, mech->dev.f32, m->N,
                                                                        (float)mech->T_mid, ood_route(m), flags);
    return check_cuda(cudaGetLastError(), "chem_mlp_ood_flags");
}

extern "C" int chem_mlp_get_ood(const chem_mlp *m, float *lo3, float *hi3, int32_t *nbins, int32_t *species,
                                int32_t *min_count) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_get_ood: null handle");
    if (!m->ood_fitted) return set_error(CHEM_EINVAL, "chem_mlp_get_ood: the grid is not fitted");
    for (int d = 0; d < 3; ++d) { if (lo3) lo3[d] = m->ood_lo[0][d]; if (hi3) hi3[d] = m->ood_hi[0][d]; }
    if (nbins) *nbins = m->ood_nb;
    if (species) *species = m->ood_species[0];
    if (min_count) *min_count = m->ood_kmin;
    return CHEM_OK;
}

extern "C" int chem_mlp_get_ood_grid(const chem_mlp *m, int32_t grid, float *lo3, float *hi3, int32_t *species) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_get_ood_grid: null handle");
    if (!m->ood_fitted || grid < 0 || grid >= m->ood_ngrids)
        return set_error(CHEM_EINVAL, "chem_mlp_get_ood_grid: no such fitted grid");
    for (int d = 0; d < 3; ++d) { if (lo3) lo3[d] = m->ood_lo[grid][d]; if (hi3) hi3[d] = m->ood_hi[grid][d]; }
    if (species) *species = m->ood_species[grid];
    return CHEM_OK;
}

namespace chemgb {
namespace {

// Forward (saving pre-activations), Eq. 5 loss and backward of the per-species ensemble on the B
// rows already in tx0. Each network's loss is its own output's term of the summed L1 loss, so the
// gradients are those of G independent trainings. The stacked layers' gradients land in the
// layers' gW, gb like a single network's.
int ens_train_passes(chem_mlp *m, int B, const int32_t *idx, int64_t ld, const double *Y, const double *Y1,
                     float *loss_dev, cudaStream_t st) {
    const int G = m->G;
    const Layer &L0 = m->L[0];
    int rc = gemm_gelu(L0.tile, m->tx0, kXTerms * m->n_in_pad, L0.Wb, L0.kx, B, L0.out, L0.kx, L0.b, m->th[0], L0.out,
                       m->tz[0], L0.out, m->err, st);
    for (int l = 1; l < 3 && !rc; ++l) rc = ens_hidden(m, l, m->L[l].tile, B, m->th[l - 1], m->th[l], m->tz[l], st);
    if (!rc) rc = ens_output(m, B, m->th[2], m->tout, st);
    if (rc) return rc;
    l1_loss_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, m->tout, m->n_out_pad, idx, ld, Y, Y1, m->n_out, m->out_sp_dev,
                                                     m->mu_u, m->sd_u, m->tdout, m->n_out_pad, m->loss_part, nullptr,
                                                     PhysLoss{});
    if (loss_dev) loss_reduce_kernel<<<1, 256, 0, st>>>(B, m->loss_part, loss_dev);
    if ((rc = check_cuda(cudaGetLastError(), "ensemble loss"))) return rc;
    // output units
    {
        const Layer &L = m->L[3];
        const int64_t ldh = (int64_t)G * L.in;
        group_dot_wgrad_kernel<<<(G * L.in + 31) / 32, dim3(32, kColsumRows), 0, st>>>(B, G, L.in, m->tdout, m->n_out_pad, m->th[2],
                                                                        ldh, L.gW, L.kin);
        colsum_kernel<<<(G + 31) / 32, dim3(32, kColsumRows), 0, st>>>(B, G, m->tdout, m->n_out_pad, L.gb);
        const int64_t ne = (int64_t)B * ldh;
        group_dot_back_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(B, G, L.in, m->tdout, m->n_out_pad, L.Wb,
                                                                            L.kx, m->tz[2], ldh, m->tdz[2], ldh);
        if ((rc = check_cuda(cudaGetLastError(), "ensemble output backward"))) return rc;
    }
    dim3 tb(32, 8);
    // grouped hidden layers: dW_g = dZ_g^T H_g (stacked rows of the transposes), dZ_{l-1} = (dZ_g W_g) GELU'
    for (int l = 2; l >= 1; --l) {
        const Layer &L = m->L[l];
        const int64_t ldz = (int64_t)G * L.gout, ldh = (int64_t)G * L.in;
        transpose_kernel<<<dim3((unsigned)((ldz + 31) / 32), (B + 31) / 32), tb, 0, st>>>(B, (int)ldz, m->tdz[l], ldz,
                                                                                         m->tT0, B);
        transpose_kernel<<<dim3((unsigned)((ldh + 31) / 32), (B + 31) / 32), tb, 0, st>>>(B, (int)ldh, m->th[l - 1],
                                                                                         ldh, m->tT1, B);
        if ((rc = check_cuda(cudaGetLastError(), "ensemble transpose"))) return rc;
        rc = gemm_linear_grouped(default_tile_width(L.in), GemmOperand{m->tT0, B, kMapRowGrp, (int64_t)L.gout * B},
                                 GemmOperand{m->tT1, B, kMapRowGrp, (int64_t)L.in * B}, G, L.gout, L.in, B, nullptr, 0,
                                 L.gW, L.kin, (int64_t)L.gout * L.kin, m->err, st);
        if (rc) return rc;
        colsum_kernel<<<(unsigned)((ldz + 31) / 32), dim3(32, kColsumRows), 0, st>>>(B, (int)ldz, m->tdz[l], (int)ldz, L.gb);
        if ((rc = check_cuda(cudaGetLastError(), "ensemble bias grad"))) return rc;
        rc = gemm_gelu_grad_grouped(default_tile_width(L.in), GemmOperand{m->tdz[l], ldz, kMapColGrp, L.gout},
                                    GemmOperand{L.Wt, L.outp, kMapColGrp, L.gout}, G, B, L.in, L.gout, m->tz[l - 1],
                                    ldh, L.in, m->tdz[l - 1], ldh, L.in, m->err, st);
        if (rc) return rc;
    }
    // the stacked first layers: one product over all networks (their input is shared)
    transpose_kernel<<<dim3((L0.out + 31) / 32, (B + 31) / 32), tb, 0, st>>>(B, L0.out, m->tdz[0], L0.out, m->tT0, B);
    transpose_kernel<<<dim3((m->n_in_pad + 31) / 32, (B + 31) / 32), tb, 0, st>>>(B, m->n_in_pad, m->tx0,
                                                                                  kXTerms * m->n_in_pad, m->tT1, B);
    if ((rc = check_cuda(cudaGetLastError(), "ensemble transpose"))) return rc;
    rc = gemm_linear(default_tile_width(L0.kin), m->tT0, B, m->tT1, B, L0.out, L0.kin, B, nullptr, L0.gW, L0.kin,
                     m->err, st);
    if (rc) return rc;
    colsum_kernel<<<(L0.out + 31) / 32, dim3(32, kColsumRows), 0, st>>>(B, L0.out, m->tdz[0], L0.out, L0.gb);
    return check_cuda(cudaGetLastError(), "ensemble bias grad");
}

}  // namespace
}  // namespace chemgb

namespace chemgb {
namespace {

// forward with saved activations, loss (Eq. 5 and the physics terms) and back-propagation: the
// gradients of one batch in the handle's gW / gb
int train_grads_impl(chem_mlp *m, int64_t batch, const int32_t *idx, int64_t ld, const double *T, const double *p,
                     const double *Y, const double *Y1, float *loss_dev, cudaStream_t st, const char *who) {
    const std::string w(who);
    if (!m) return set_error(CHEM_EINVAL, w + ": null handle");
    if (batch < 8 || batch > m->max_batch || batch % 8 != 0)
        return set_error(CHEM_EINVAL, w + ": batch must be a multiple of 8 in [8, max_batch]");
    int rc = check_state_args(idx ? ld : batch, ld, T, p, Y, who);
    if (rc) return rc;
    if (!Y1 || !aligned16(Y1) || (loss_dev && !aligned16(loss_dev)))
        return set_error(CHEM_EINVAL, w + ": Y1 and loss must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, w + ": " + why);
    WaitLimitScope wl(m->wait_limit);
    const int B = (int)batch;
    // forward with saved pre-activations
    prologue_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, ld, T, p, Y, idx, m->N, m->n_in_pad, m->mu_x, m->isd_x, m->tx0);
    if ((rc = check_cuda(cudaGetLastError(), "train prologue"))) return rc;
    if (m->ens) {
        rc = ens_train_passes(m, B, idx, ld, Y, Y1, loss_dev, st);
        if (rc) return rc;
    } else {
        const __nv_bfloat16 *x = m->tx0;
        int64_t ldx = kXTerms * m->n_in_pad;
        for (int l = 0; l < 3; ++l) {
            const Layer &L = m->L[l];
            rc = gemm_gelu(L.tile, x, ldx, L.Wb, L.kx, B, L.out, L.kx, L.b, m->th[l], L.out, m->tz[l], L.out, m->err, st);
            if (rc) return rc;
            x = m->th[l];
            ldx = L.out;
        }
        {
            const Layer &L = m->L[3];
            rc = gemm_linear(L.tile, x, ldx, L.Wb, L.kx, B, L.out, L.kx, L.b, m->tout, m->n_out_pad, m->err, st);
            if (rc) return rc;
        }
        // loss and dL/du
        l1_loss_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, m->tout, m->n_out_pad, idx, ld, Y, Y1, m->n_out, m->out_sp_dev,
                                                         m->mu_u, m->sd_u, m->tdout, m->n_out_pad, m->loss_part, T,
                                                         phys_loss(m));
        if (loss_dev) loss_reduce_kernel<<<1, 256, 0, st>>>(B, m->loss_part, loss_dev);
        if ((rc = check_cuda(cudaGetLastError(), "train loss"))) return rc;
        // backward, top layer down: dW_l = dZ_l^T H_{l-1}, db_l = colsum dZ_l, dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
        const __nv_bfloat16 *dz = m->tdout;
        int lddz = m->n_out_pad;
        for (int l = 3; l >= 0; --l) {
            const Layer &L = m->L[l];
            // the first layer's weight gradient takes the hi input term (BF16 precision suffices for a gradient)
            const __nv_bfloat16 *hin = (l == 0) ? m->tx0 : m->th[l - 1];
            const int wh = (l == 0) ? m->n_in_pad : m->L[l - 1].out;
            const int ldh = (l == 0) ? kXTerms * m->n_in_pad : wh;
            dim3 tb(32, 8);
            transpose_kernel<<<dim3((lddz + 31) / 32, (B + 31) / 32), tb, 0, st>>>(B, lddz, dz, lddz, m->tT0, B);
            transpose_kernel<<<dim3((wh + 31) / 32, (B + 31) / 32), tb, 0, st>>>(B, wh, hin, ldh, m->tT1, B);
            if ((rc = check_cuda(cudaGetLastError(), "train transpose"))) return rc;
            rc = gemm_linear(default_tile_width(L.kin), m->tT0, B, m->tT1, B, L.out, L.kin, B, nullptr, L.gW, L.kin, m->err,
                             st);
            if (rc) return rc;
            colsum_kernel<<<(L.out + 31) / 32, dim3(32, kColsumRows), 0, st>>>(B, L.out, dz, lddz, L.gb);
            if ((rc = check_cuda(cudaGetLastError(), "train bias grad"))) return rc;
            if (l > 0) {
                const Layer &Lb = m->L[l - 1];
                rc = gemm_gelu_grad(default_tile_width(Lb.out), dz, lddz, L.Wt, L.outp, B, Lb.out, L.outp, m->tz[l - 1],
                                    Lb.out, m->tdz[l - 1], Lb.out, m->err, st);
                if (rc) return rc;
                dz = m->tdz[l - 1];
                lddz = Lb.out;
            }
        }
    }
    return CHEM_OK;
}

// Adam on the gradients in the handle's gW / gb
int adam_impl(chem_mlp *m, float lr, cudaStream_t st) {
    m->adam_t += 1;
    m->fp8_ready = 0;
    const float bc1 = 1.0f - std::pow(kAdamB1, (float)m->adam_t);
    const float bc2 = 1.0f - std::pow(kAdamB2, (float)m->adam_t);
    for (int l = 0; l < kLayers; ++l) {
        Layer &L = m->L[l];
        const int64_t n = (int64_t)L.out * L.in + L.out;
        adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L.out, L.in, L.kin, L.kx, L.outp, L.W, L.b, L.gW, L.gb, L.mW,
                                                                 L.vW, L.mb, L.vb, L.Wb, L.Wt, lr, bc1, bc2);
    }
    return check_cuda(cudaGetLastError(), "train adam");
}

}  // namespace
}  // namespace chemgb

extern "C" int mlp_train_step(chem_mlp *m, int64_t batch, const int32_t *idx, int64_t ld, const double *T,
                              const double *p, const double *Y, const double *Y1, float lr, float *loss_dev,
                              chem_stream_t stream) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = train_grads_impl(m, batch, idx, ld, T, p, Y, Y1, loss_dev, st, "mlp_train_step");
    return rc ? rc : adam_impl(m, lr, st);
}

extern "C" int mlp_train_grads(chem_mlp *m, int64_t batch, const int32_t *idx, int64_t ld, const double *T,
                               const double *p, const double *Y, const double *Y1, float *loss_dev,
                               chem_stream_t stream) {
    return train_grads_impl(m, batch, idx, ld, T, p, Y, Y1, loss_dev, reinterpret_cast<cudaStream_t>(stream),
                            "mlp_train_grads");
}

extern "C" int mlp_adam_step(chem_mlp *m, float lr, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "mlp_adam_step: null handle");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "mlp_adam_step: " + why);
    return adam_impl(m, lr, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int chem_mlp_grad_buffers(const chem_mlp *m, int layer, float **gW, int64_t *nW, float **gb, int64_t *nb) {
    if (!m || !gW || !nW || !gb || !nb || layer < 0 || layer >= kLayers)
        return set_error(CHEM_EINVAL, "chem_mlp_grad_buffers: null argument or layer outside 0..3");
    const Layer &L = m->L[layer];
    *gW = L.gW;
    *nW = (int64_t)L.out * L.kin;
    *gb = L.gb;
    *nb = (int64_t)L.outp;
    return CHEM_OK;
}

extern "C" int chem_mlp_set_physics_loss(chem_mlp *m, double lam_m, double lam_q, double s_m, double s_q) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_set_physics_loss: null handle");
    if (!(lam_m >= 0.0) || !(lam_q >= 0.0) || !(s_m > 0.0) || !(s_q > 0.0) || !std::isfinite(lam_m) ||
        !std::isfinite(lam_q) || !std::isfinite(s_m) || !std::isfinite(s_q))
        return set_error(CHEM_EINVAL, "chem_mlp_set_physics_loss: weights must be >= 0 and scales > 0, finite");
    if (m->ens && (lam_m != 0.0 || lam_q != 0.0))
        return set_error(CHEM_EUNSUPPORTED, "chem_mlp_set_physics_loss: the per-species ensemble trains each network "
                                            "on its own output; the physics terms couple the outputs");
    m->lam_m = lam_m;
    m->lam_q = lam_q;
    m->s_m = s_m;
    m->s_q = s_q;
    return CHEM_OK;
}

extern "C" int chem_mlp_fit_physics_scales(chem_mlp *m, int64_t n, int64_t ld, const double *T, const double *Y,
                                           const double *Y1, double *s_m, double *s_q, chem_stream_t stream) {
    if (!m || !s_m || !s_q) return set_error(CHEM_EINVAL, "chem_mlp_fit_physics_scales: null argument");
    if (n < 1 || ld < n || (ld & 3) != 0 || !T || !Y || !Y1 || !aligned16(T) || !aligned16(Y) || !aligned16(Y1))
        return set_error(CHEM_EINVAL, "chem_mlp_fit_physics_scales: need 1 <= n <= ld, ld % 4 == 0, aligned arrays");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_fit_physics_scales: " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the block partials and the result reuse the out-of-distribution fit's scratch (512 x 6 floats)
    const int nb = 256;
    double *part = reinterpret_cast<double *>(m->ood_part);
    phys_scales_kernel<<<nb, 256, 0, st>>>(n, ld, T, Y, Y1, m->n_out, m->out_sp_dev, phys_loss(m), part);
    phys_scales_reduce_kernel<<<1, 32, 0, st>>>(nb, n, part, part + 2 * nb);
    int rc = check_cuda(cudaGetLastError(), "chem_mlp_fit_physics_scales launch");
    double h[2] = {0.0, 0.0};
    if (!rc) rc = check_cuda(cudaMemcpyAsync(h, part + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, st),
                             "chem_mlp_fit_physics_scales copy");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "chem_mlp_fit_physics_scales sync");
    if (rc) return rc;
    *s_m = h[0];
    *s_q = h[1];
    return CHEM_OK;
}

extern "C" int chem_mlp_set_fusion(chem_mlp *m, int mask) {
    if (!m || (mask != 0 && mask != CHEM_FUSE_34))
        return set_error(CHEM_EINVAL, "chem_mlp_set_fusion: null handle or mask other than 0 or CHEM_FUSE_34");
    m->fuse34 = (mask & CHEM_FUSE_34) ? 1 : 0;
    return CHEM_OK;
}

extern "C" int chem_mlp_get_fusion(const chem_mlp *m) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_get_fusion: null handle");
    return fused34_on(m) ? CHEM_FUSE_34 : 0;
}

extern "C" int chem_mlp_set_wait_limit(chem_mlp *m, uint32_t tries) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_set_wait_limit: null handle");
    m->wait_limit = tries == 0 ? tc::kSpinLimit : tries;
    return CHEM_OK;
}

extern "C" int chem_mlp_error(const chem_mlp *m, int *host_err) {
    if (!m || !host_err) return set_error(CHEM_EINVAL, "chem_mlp_error: null argument");
    int rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_error");
    if (rc) return rc;
    return check_cuda(cudaMemcpy(host_err, m->err, sizeof(int), cudaMemcpyDeviceToHost), "chem_mlp_error");
}

// ---------------------------------------------------------------------------
// checkpoint: header, statistics, parameters and Adam state, FNV-1a checksum
// ---------------------------------------------------------------------------
namespace chemgb {
namespace {

constexpr char kMlpMagic[8] = {'C', 'H', 'M', 'L', 'P', '0', '0', '1'};

uint64_t fnv1a(const uint8_t *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

// Adam moments in the host parameter layout (W[out][in] then b[out] per layer)
int copy_moments(const chem_mlp *m, float *host, bool to_host, bool second) {
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        const Layer &L = m->L[l];
        float *W = second ? L.vW : L.mW;
        float *b = second ? L.vb : L.mb;
        cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
        int rc = check_cuda(to_host ? cudaMemcpy2D(host + off, L.in * 4, W, L.kin * 4, L.in * 4, L.out, kind)
                                    : cudaMemcpy2D(W, L.kin * 4, host + off, L.in * 4, L.in * 4, L.out, kind),
                            "moment copy");
        if (rc) return rc;
        off += (int64_t)L.out * L.in;
        rc = check_cuda(to_host ? cudaMemcpy(host + off, b, L.out * 4, kind) : cudaMemcpy(b, host + off, L.out * 4, kind),
                        "moment copy");
        if (rc) return rc;
        off += L.out;
    }
    return CHEM_OK;
}

}  // namespace
}  // namespace chemgb

extern "C" int chem_mlp_save(const chem_mlp *m, const char *path) {
    if (!m || !path) return set_error(CHEM_EINVAL, "chem_mlp_save: null argument");
    int rc = check_cuda(cudaDeviceSynchronize(), "chem_mlp_save");
    if (rc) return rc;
    const int64_t np = param_count(m);
    std::vector<uint8_t> body;
    auto put = [&](const void *p, size_t n) {
        const uint8_t *b = static_cast<const uint8_t *>(p);
        body.insert(body.end(), b, b + n);
    };
    // version 1: one multi-output network; version 2: followed by {ensemble flag, 0}
    int32_t hdr[8] = {m->ens ? 2 : 1, m->N, m->bath, m->widths[0], m->widths[1], m->widths[2], m->widths[3],
                      m->widths[4]};
    put(hdr, sizeof(hdr));
    if (m->ens) {
        const int32_t ext[2] = {1, 0};
        put(ext, sizeof(ext));
    }
    put(&m->dt, 8);
    put(&m->adam_t, 8);
    put(m->h_mu_x, 8 * m->n_in);
    put(m->h_sd_x, 8 * m->n_in);
    put(m->h_mu_u, 8 * m->n_out);
    put(m->h_sd_u, 8 * m->n_out);
    std::vector<float> buf(np);
    if ((rc = copy_params(m, buf.data(), true, false))) return rc;
    put(buf.data(), 4 * np);
    if ((rc = copy_moments(m, buf.data(), true, false))) return rc;
    put(buf.data(), 4 * np);
    if ((rc = copy_moments(m, buf.data(), true, true))) return rc;
    put(buf.data(), 4 * np);
    const uint64_t sum = fnv1a(body.data(), body.size());
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(CHEM_EIO, std::string("chem_mlp_save: cannot open ") + path);
    bool ok = std::fwrite(kMlpMagic, 1, 8, f) == 8 && std::fwrite(body.data(), 1, body.size(), f) == body.size() &&
              std::fwrite(&sum, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? CHEM_OK : set_error(CHEM_EIO, "chem_mlp_save: write failed");
}

extern "C" int chem_mlp_load(const chem_mech *mech, const char *path, chem_mlp **out) {
    if (!mech || !path || !out) return set_error(CHEM_EINVAL, "chem_mlp_load: null argument");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(CHEM_EIO, std::string("chem_mlp_load: cannot open ") + path);
    std::vector<uint8_t> all;
    uint8_t tmp[65536];
    size_t n;
    while ((n = std::fread(tmp, 1, sizeof(tmp), f)) > 0) all.insert(all.end(), tmp, tmp + n);
    std::fclose(f);
    if (all.size() < 8 + 32 + 16 + 8 || std::memcmp(all.data(), kMlpMagic, 8) != 0)
        return set_error(CHEM_EIO, "chem_mlp_load: not a network checkpoint");
    const uint8_t *body = all.data() + 8;
    const size_t blen = all.size() - 16;
    uint64_t sum;
    std::memcpy(&sum, all.data() + all.size() - 8, 8);
    if (fnv1a(body, blen) != sum) return set_error(CHEM_EIO, "chem_mlp_load: checksum mismatch");
    int32_t hdr[8];
    std::memcpy(hdr, body, sizeof(hdr));
    if (hdr[0] != 1 && hdr[0] != 2) return set_error(CHEM_EIO, "chem_mlp_load: unknown checkpoint version");
    if (hdr[1] != mech->N || hdr[2] != mech->bath)
        return set_error(CHEM_EINVAL, "chem_mlp_load: checkpoint species do not match the mechanism");
    chem_mlp_desc d;
    std::memset(&d, 0, sizeof(d));
    for (int i = 0; i < 3; ++i) d.n_hidden[i] = hdr[4 + i];
    size_t off = sizeof(hdr);
    if (hdr[0] == 2) {
        int32_t ext[2];
        if (blen < off + sizeof(ext)) return set_error(CHEM_EIO, "chem_mlp_load: truncated checkpoint");
        std::memcpy(ext, body + off, sizeof(ext));
        if (ext[0] != 0 && ext[0] != 1) return set_error(CHEM_EIO, "chem_mlp_load: bad ensemble flag");
        d.ensemble = ext[0];
        off += sizeof(ext);
    }
    std::memcpy(&d.dt, body + off, 8);
    off += 8;
    int64_t adam_t;
    std::memcpy(&adam_t, body + off, 8);
    off += 8;
    chem_mlp *m = nullptr;
    int rc = chem_mlp_create(mech, &d, 0, &m);
    if (rc) return rc;
    const int64_t np = param_count(m);
    const size_t need = off + 8 * (size_t)(2 * m->n_in + 2 * m->n_out) + 12 * (size_t)np;
    if (need != blen) { chem_mlp_free(m); return set_error(CHEM_EIO, "chem_mlp_load: truncated checkpoint"); }
    std::vector<double> st(2 * m->n_in + 2 * m->n_out);
    std::memcpy(st.data(), body + off, 8 * st.size());
    off += 8 * st.size();
    rc = chem_mlp_set_norm(m, st.data(), st.data() + m->n_in, st.data() + 2 * m->n_in,
                           st.data() + 2 * m->n_in + m->n_out);
    std::vector<float> buf(np);
    if (!rc) {
        std::memcpy(buf.data(), body + off, 4 * np);
        off += 4 * np;
        rc = chem_mlp_set_params(m, buf.data());
    }
    if (!rc) {
        std::memcpy(buf.data(), body + off, 4 * np);
        off += 4 * np;
        rc = copy_moments(m, buf.data(), false, false);
    }
    if (!rc) {
        std::memcpy(buf.data(), body + off, 4 * np);
        rc = copy_moments(m, buf.data(), false, true);
    }
    if (rc) { chem_mlp_free(m); return rc; }
    m->adam_t = adam_t;
    *out = m;
    return CHEM_OK;
}

// ---------------------------------------------------------------------------
// autotuner: the fastest compiled tile width per layer, timed on the inference
// workspace with CUDA events (the operands' values do not change the work)
// ---------------------------------------------------------------------------
extern "C" int chem_mlp_autotune(chem_mlp *m, int64_t rows, int32_t *tiles_out, chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mlp_autotune: null handle");
    WaitLimitScope wl(m->wait_limit);
    if (rows < 128) rows = 128;
    if (rows > m->chunk) rows = m->chunk;
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mlp_autotune: " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    float best_ms[kLayers] = {0.0f, 0.0f, 0.0f, 0.0f};
    int rc = check_cuda(cudaEventCreate(&e0), "autotune event");
    if (rc) return rc;
    rc = check_cuda(cudaEventCreate(&e1), "autotune event");
    if (rc) { cudaEventDestroy(e0); return rc; }
    for (int l = 0; l < kLayers && !rc; ++l) {
        Layer &L = m->L[l];
        if (m->ens && l == kLayers - 1) {           // the ensemble's output units are not a GEMM
            if (tiles_out) tiles_out[l] = 0;
            continue;
        }
        const __nv_bfloat16 *x = (l == 0) ? m->a0 : m->h[l - 1];
        const int64_t ldx = (l == 0) ? kXTerms * m->n_in_pad : m->L[l - 1].out;
        const int width = (m->ens && l > 0) ? L.gout : L.out;    // output columns of one product
        float best = 3.4e38f;
        int best_bn = L.tile;
        best_ms[l] = 0.0f;
        // the two-CTA variant is not a candidate: measured on GB300 it runs at half the single-CTA rate
        const std::vector<int> codes(std::begin(kTileWidths), std::end(kTileWidths));
        for (int bn : codes) {
            const int w = bn & 0xFFFF;
            if (w < 64 && width > 64) continue;
            if (w > 2 * ((width + 15) / 16) * 16 && w > 64) continue;   // tiles far wider than the layer
            float ms_sum = 0.0f;
            for (int rep = 0; rep < 4 && !rc; ++rep) {
                rc = check_cuda(cudaEventRecord(e0, st), "autotune record");
                if (rc) break;
                if (m->ens && l > 0)
                    rc = ens_hidden(m, l, bn, (int)rows, m->h[l - 1], m->h[l], nullptr, st);
                else if (l < 3)
                    rc = gemm_gelu(bn, x, ldx, L.Wb, L.kx, (int)rows, L.out, L.kx, L.b, m->h[l], L.out, nullptr, 0,
                                   m->err, st);
                else
                    rc = gemm_linear(bn, x, ldx, L.Wb, L.kx, (int)rows, L.out, L.kx, L.b, m->out, m->n_out_pad,
                                     m->err, st);
                if (rc) break;
                rc = check_cuda(cudaEventRecord(e1, st), "autotune record");
                if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "autotune sync");
                float ms = 0.0f;
                if (!rc) cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_sum += ms;                               // the first launch warms up
            }
            if (!rc && ms_sum < best) { best = ms_sum; best_bn = bn; }
        }
        L.tile = best_bn;
        best_ms[l] = best;
        if (tiles_out) tiles_out[l] = best_bn;
    }
    // layers 3 and 4 fused into one launch, against the best two-launch pair
    if (!rc && !m->ens && fused34_supported(m->L[2].kx, m->L[2].out, m->L[3].out)) {
        const Layer &L3 = m->L[2], &L4 = m->L[3];
        float ms_sum = 0.0f;
        for (int rep = 0; rep < 4 && !rc; ++rep) {
            rc = check_cuda(cudaEventRecord(e0, st), "autotune record");
            if (!rc)
                rc = gemm_fused34(m->h[1], m->L[1].out, L3.kx, L3.Wb, L3.kx, L4.Wb, L4.kx, (int)rows, L3.out, L4.out,
                                  L3.b, L4.b, m->out, m->n_out_pad, m->err, st);
            if (!rc) rc = check_cuda(cudaEventRecord(e1, st), "autotune record");
            if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "autotune sync");
            float ms = 0.0f;
            if (!rc) cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ms_sum += ms;
        }
        if (!rc) m->fuse34 = ms_sum < best_ms[2] + best_ms[3] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
