// props.cu -- props_eval: NASA-7 mixture thermo and mixture-averaged
// transport for every cell (Sec. 2: thermal and transport properties on the
// GPU; Sec. 3.1: Hirschfelder-Curtiss mixture-averaged model).
//
// One thread per cell, persistent grid-stride loop. Cell data are SoA, so a
// warp's loads of T, p and each Y_k row are 128-byte coalesced. The per-pair
// tables (Wilke weights, binary-resistance fits) are read with uniform
// addresses (one broadcast per warp) through the read-only cache. The
// per-cell vectors X_j and 1 / r_j (r = sqrt(mu)) live in registers: the inner
// species loop is unrolled to a compile-time bound NMAX.
//
// Wilke: sum_j X_j Phi_kj with Phi_kj = c_kj (1 + w_jk r_k / r_j)^2 is
// evaluated per pair as T0 + t (T1 + t T2), t = r_k / r_j, with constant tables
// T0 = c, T1 = 2 c w, T2 = c w^2 (expanded once at load time): one multiply
// more per pair than three separate sums, for a third fewer registers (which
// bound the kernel's occupancy).
#include <cmath>

#include "internal.cuh"
#include "tc.cuh"

namespace chemgb {
namespace {

template <typename real>
__device__ __forceinline__ void load4(const real *p, real &a, real &b, real &c, real &d) {
    if constexpr (sizeof(real) == 4) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        a = v.x; b = v.y; c = v.z; d = v.w;
    } else {
        double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
        double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        a = v0.x; b = v0.y; c = v1.x; d = v1.y;
    }
}

// FP32 tables always fit (8 N Np floats <= 131 KB for N <= 64); FP64 tables stay in global memory.
constexpr size_t kPropsSmemMax = (8 * 64 * 64 + 28 * 64) * 4;
template <typename real>
__host__ __device__ constexpr bool tables_in_smem() { return sizeof(real) == 4; }

// Copies the per-pair tables (3 Wilke + 5 resistance rows per species) into
// shared memory when they fit; the inner loops then read them with broadcast
// LDS.128 instead of uniform global loads.
template <typename real>
__device__ __forceinline__ void stage_pair_tables(const PropTables<real> &tb, int N, int Np, real *sh) {
    const int nw = 3 * N * Np, nd = 5 * N * Np;
    for (int e = threadIdx.x; e < nw; e += blockDim.x) sh[e] = tb.wilke[e];
    for (int e = threadIdx.x; e < nd; e += blockDim.x) sh[nw + e] = tb.diff[e];
    __syncthreads();
}

// Per-species coefficient rows (NASA cp and h of both ranges, the ln(mu) fit, 1/W) in
// the global tables' own layout, copied to shared memory after the pair tables so
// that the species loops read them as broadcasts.
constexpr int kSpeciesFloats = 2 * 5 + 2 * 6 + 5 + 1;   // floats per species
template <typename real>
__device__ __forceinline__ void stage_species_tables(const PropTables<real> &tb, int N, real *sh) {
    for (int e = threadIdx.x; e < 10 * N; e += blockDim.x) sh[e] = tb.nasa_cp[e];
    for (int e = threadIdx.x; e < 12 * N; e += blockDim.x) sh[10 * N + e] = tb.nasa_h[e];
    for (int e = threadIdx.x; e < 5 * N; e += blockDim.x) sh[22 * N + e] = tb.visc[e];
    for (int e = threadIdx.x; e < N; e += blockDim.x) sh[27 * N + e] = tb.invW[e];
    __syncthreads();
}

template <typename real>
__device__ __forceinline__ void load4s(const real *p, real &a, real &b, real &c, real &d) {
    if constexpr (sizeof(real) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a = v.x; b = v.y; c = v.z; d = v.w;
    } else {
        const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
        a = v0.x; b = v0.y; c = v1.x; d = v1.y;
    }
}

// state value -> working precision; FP64 -> FP32 on the integer pipe (truncation, < 2^-23 relative)
template <typename real, typename in_t>
__device__ __forceinline__ real to_real(in_t x) {
    if constexpr (sizeof(real) == 4 && sizeof(in_t) == 8) return f64_to_f32_trunc(x);
    else return real(x);
}

template <typename real, typename in_t, int NMAX>
__global__ void __launch_bounds__(128, sizeof(real) == 4 && NMAX <= 32 ? 4 : 1) props_kernel(int N, int Np, real T_mid, PropTables<real> tb, int64_t ncells,
                                                    int64_t ld, const in_t *__restrict__ Tg,
                                                    const in_t *__restrict__ pg, const in_t *__restrict__ Yg,
                                                    real *__restrict__ cpg, real *__restrict__ hg,
                                                    real *__restrict__ mug, real *__restrict__ lamg,
                                                    real *__restrict__ Dkg) {
    const real R = real(kR);
    const bool transport = (mug != nullptr) || (lamg != nullptr) || (Dkg != nullptr);
    extern __shared__ __align__(16) unsigned char props_smem[];
    real *shtab = reinterpret_cast<real *>(props_smem);
    constexpr bool in_smem = tables_in_smem<real>();
    if (in_smem && transport) stage_pair_tables(tb, N, Np, shtab);
    real *sp = shtab + (transport ? 8 * N * Np : 0);
    if (in_smem) stage_species_tables(tb, N, sp);
    const real *wil = in_smem ? shtab : tb.wilke;
    const real *dif = in_smem ? shtab + 3 * N * Np : tb.diff;
    const real *t_cp = in_smem ? sp : tb.nasa_cp;
    const real *t_h = in_smem ? sp + 10 * N : tb.nasa_h;
    const real *t_visc = in_smem ? sp + 22 * N : tb.visc;
    const real *t_iw = in_smem ? sp + 27 * N : tb.invW;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += stride) {
        const real T = to_real<real>(Tg[i]);
        const real p = to_real<real>(pg[i]);
        const int rng = (T >= T_mid) ? 1 : 0;
        const real iT = real(1) / T;
        const real x = log(T) - real(6.907755278982137);   // ln(T / 1000)
        real S = 0, cpm = 0, hm = 0;
        real X[NMAX], ir[NMAX];
        // pass 1: thermo sums; keep Y_k / W_k
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k < N) {
                const real y = to_real<real>(Yg[(int64_t)k * ld + i]);
                const real iw = t_iw[k];
                const real *a = t_cp + (rng * N + k) * 5;
                const real *b = t_h + (rng * N + k) * 6;
                real cpR = a[4];
                cpR = fma(cpR, T, a[3]);
                cpR = fma(cpR, T, a[2]);
                cpR = fma(cpR, T, a[1]);
                cpR = fma(cpR, T, a[0]);
                real hR = b[4];
                hR = fma(hR, T, b[3]);
                hR = fma(hR, T, b[2]);
                hR = fma(hR, T, b[1]);
                hR = fma(hR, T, b[0]);
                hR = fma(b[5], iT, hR);                          // H_k / (R T)
                const real yw = y * iw;
                S += yw;
                cpm = fma(yw, cpR, cpm);
                hm = fma(yw, hR, hm);
                X[k] = yw;
            } else {
                X[k] = 0;
            }
        }
        if (cpg) cpg[i] = cpm * R;
        if (hg) hg[i] = hm * R * T;
        if (!transport) continue;
        const real Wbar = real(1) / S;
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k < N) {
                const real *c = t_visc + k * 5;
                real lm = c[4];
                lm = fma(lm, x, c[3]);
                lm = fma(lm, x, c[2]);
                lm = fma(lm, x, c[1]);
                lm = fma(lm, x, c[0]);
                ir[k] = exp(real(-0.5) * lm);                      // 1 / sqrt(mu_k)
                X[k] = X[k] * Wbar;
            } else {
                ir[k] = 0;
            }
        }
        const real T15 = T * sqrt(T);
        real mu = 0, lam = 0;
        real y_next = to_real<real>(Yg[i]);
        for (int k = 0; k < N; ++k) {
            // per-species values, recomputed from the tables (no dynamic register indexing);
            // the next species' mass fraction is loaded one iteration ahead
            const real y = y_next;
            if (k + 1 < N) y_next = to_real<real>(Yg[(int64_t)(k + 1) * ld + i]);
            const real iw = t_iw[k];
            const real Xk = y * iw * Wbar;
            const real *c = t_visc + k * 5;
            real lm = c[4];
            lm = fma(lm, x, c[3]);
            lm = fma(lm, x, c[2]);
            lm = fma(lm, x, c[1]);
            lm = fma(lm, x, c[0]);
            const real muk = exp(lm);
            const real rk = sqrt(muk);
            const real *a = t_cp + (rng * N + k) * 5;
            real cpR = a[4];
            cpR = fma(cpR, T, a[3]);
            cpR = fma(cpR, T, a[2]);
            cpR = fma(cpR, T, a[1]);
            cpR = fma(cpR, T, a[0]);
            const real lamk = muk * (cpR + real(1.25)) * R * iw;   // Eucken
            const real *t0 = wil + (0 * N + k) * Np;
            const real *t1 = wil + (1 * N + k) * Np;
            const real *t2 = wil + (2 * N + k) * Np;
            const real *d0 = dif + (0 * N + k) * Np;
            const real *d1 = dif + (1 * N + k) * Np;
            const real *d2 = dif + (2 * N + k) * Np;
            const real *d3 = dif + (3 * N + k) * Np;
            const real *d4 = dif + (4 * N + k) * Np;
            real a0 = 0, ds = 0, gs = 0;
            [[maybe_unused]] uint64_t a02 = 0, ds2 = 0, gs2 = 0;       // FP32: (even j, odd j) sums
            [[maybe_unused]] const uint64_t rk2 = sizeof(real) == 4 ? pk2(float(rk), float(rk)) : 0;
            [[maybe_unused]] const uint64_t x2 = sizeof(real) == 4 ? pk2(float(x), float(x)) : 0;
#pragma unroll
            for (int j4 = 0; j4 < NMAX; j4 += 4) {
                if (j4 < N) {
                    real w0[4], w1[4], w2[4], g0[4], g1[4], g2[4], g3[4], g4[4];
                    if constexpr (in_smem) {
                        load4s(t0 + j4, w0[0], w0[1], w0[2], w0[3]);
                        load4s(t1 + j4, w1[0], w1[1], w1[2], w1[3]);
                        load4s(t2 + j4, w2[0], w2[1], w2[2], w2[3]);
                        load4s(d0 + j4, g0[0], g0[1], g0[2], g0[3]);
                        load4s(d1 + j4, g1[0], g1[1], g1[2], g1[3]);
                        load4s(d2 + j4, g2[0], g2[1], g2[2], g2[3]);
                        load4s(d3 + j4, g3[0], g3[1], g3[2], g3[3]);
                        load4s(d4 + j4, g4[0], g4[1], g4[2], g4[3]);
                    } else {
                        load4(t0 + j4, w0[0], w0[1], w0[2], w0[3]);
                        load4(t1 + j4, w1[0], w1[1], w1[2], w1[3]);
                        load4(t2 + j4, w2[0], w2[1], w2[2], w2[3]);
                        load4(d0 + j4, g0[0], g0[1], g0[2], g0[3]);
                        load4(d1 + j4, g1[0], g1[1], g1[2], g1[3]);
                        load4(d2 + j4, g2[0], g2[1], g2[2], g2[3]);
                        load4(d3 + j4, g3[0], g3[1], g3[2], g3[3]);
                        load4(d4 + j4, g4[0], g4[1], g4[2], g4[3]);
                    }
                    if constexpr (sizeof(real) == 4) {
                        // two species j at a time on the packed FP32x2 pipe (even and odd j summed
                        // apart, joined after the loop)
#pragma unroll
                        for (int u = 0; u < 4; u += 2) {
                            const int j = j4 + u;   // padded columns have zero weights
                            // Phi_kj = T0 + t (T1 + t T2) with t = r_k / r_j
                            const uint64_t t = mul2(pk2(ir[j], ir[j + 1]), rk2);
                            const uint64_t phi =
                                fma2(t, fma2(t, pk2(w2[u], w2[u + 1]), pk2(w1[u], w1[u + 1])), pk2(w0[u], w0[u + 1]));
                            const uint64_t Xj = pk2(X[j], X[j + 1]);
                            a02 = fma2(phi, Xj, a02);
                            uint64_t g = fma2(pk2(g4[u], g4[u + 1]), x2, pk2(g3[u], g3[u + 1]));
                            g = fma2(g, x2, pk2(g2[u], g2[u + 1]));
                            g = fma2(g, x2, pk2(g1[u], g1[u + 1]));
                            g = fma2(g, x2, pk2(g0[u], g0[u + 1]));
                            ds2 = fma2(g, Xj, ds2);
                            gs2 = add2(gs2, g);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = j4 + u;   // padded columns have zero weights
                            // Phi_kj = T0 + t (T1 + t T2) with t = r_k / r_j
                            const real t = ir[j] * rk;
                            a0 = fma(fma(t, fma(t, w2[u], w1[u]), w0[u]), X[j], a0);
                            real g = fma(fma(fma(fma(g4[u], x, g3[u]), x, g2[u]), x, g1[u]), x, g0[u]);
                            ds = fma(g, X[j], ds);
                            gs += g;
                        }
                    }
                }
            }
            if constexpr (sizeof(real) == 4) {
                float e, o;
                upk2(a02, e, o);
                a0 = e + o;
                upk2(ds2, e, o);
                ds = e + o;
                upk2(gs2, e, o);
                gs = e + o;
            }
            const real den = a0;
            mu = fma(Xk, muk / den, mu);
            lam = fma(Xk, lamk / den, lam);
            if (Dkg) {
                real D;
                if (real(1) - Xk < real(1e-12)) D = T15 / (p * gs / real(N - 1));   // pure species k
                else D = (real(1) - y) * T15 / (p * ds);
                Dkg[(int64_t)k * ld + i] = D;
            }
        }
        if (mug) mug[i] = mu;
        if (lamg) lamg[i] = lam;
    }
}

// Thermo only (cp and h; the memory-bound part of props_eval), FP32 arithmetic,
// with the state staged through shared memory by bulk copies.
//
// A CTA (one per SM) takes tiles of kThTile consecutive cells. The tile's state
// rows (T, then Y_0 .. Y_{N-1}) arrive in groups of kThRows rows, one 1-D bulk
// copy (cp.async.bulk) per row segment, into a ring of stages: a producer warp
// keeps up to kStages groups in flight (about 190 KB per SM for FP64 state, far
// more bytes than the HBM latency needs), while kThTile consumer threads, one
// per cell, read their column of each landed group, accumulate cp and h and
// release the stage. Row segments are read once and in whole 16-byte units: a
// tile's last segment is rounded up to 4 cells, which stays inside ld (a
// multiple of 4). The NASA-7 rows of both ranges and 1/W sit in shared memory (3
// float4 per species and range). The arithmetic and the species order per cell
// are those of props_kernel's first pass, so cp and h are bitwise the full
// pass's. A copy wait that runs out (bounded, spin tries) records
// kPropsErrCounter, writes NaN to the tile's cp and h and stops the CTA after
// its issued copies have landed.
constexpr int kThTile = 512;                  // cells per tile = consumer threads
constexpr int kThRows = 8;                    // state rows per stage
constexpr int kThThreads = kThTile + 32;      // + the producer warp

template <typename in_t>
struct ThLayout {
    static constexpr int kStages = sizeof(in_t) == 8 ? 6 : 8;
    static constexpr uint32_t kRowBytes = kThTile * sizeof(in_t);
    static constexpr uint32_t kStage = kThRows * kRowBytes;
    static constexpr uint32_t kStageTotal = kStages * kStage;
    static size_t bytes(int N) { return kStageTotal + (size_t)6 * N * sizeof(float4) + 2 * kStages * 8; }
};

template <typename in_t>
__global__ void __launch_bounds__(kThThreads, 1)
    thermo_kernel(int N, float T_mid, PropTables<float> tb, int64_t ncells, int64_t ld,
                  const in_t *__restrict__ Tg, const in_t *__restrict__ Yg, float *__restrict__ cpg,
                  float *__restrict__ hg, unsigned int *err, uint32_t spin) {
    using L = ThLayout<in_t>;
    constexpr int S = L::kStages;
    extern __shared__ __align__(128) uint8_t th_smem[];
    uint8_t *stages = th_smem;
    float4 *tab = reinterpret_cast<float4 *>(th_smem + L::kStageTotal);
    uint64_t *full = reinterpret_cast<uint64_t *>(tab + 6 * N);
    uint64_t *empty = full + S;
    for (int e = threadIdx.x; e < 2 * N; e += blockDim.x) {
        const int rg = e / N, k = e % N;
        const float *a = tb.nasa_cp + (rg * N + k) * 5;
        const float *b = tb.nasa_h + (rg * N + k) * 6;
        tab[e * 3 + 0] = make_float4(a[0], a[1], a[2], a[3]);
        tab[e * 3 + 1] = make_float4(a[4], b[0], b[1], b[2]);
        tab[e * 3 + 2] = make_float4(b[3], b[4], b[5], tb.invW[k]);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kThTile / 32);
        }
        tc::fence_barrier_init();
    }
    __syncthreads();
    const int64_t ntiles = (ncells + kThTile - 1) / kThTile;
    const int groups = (N + 1 + kThRows - 1) / kThRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == kThTile / 32) {
        if (lane == 0) {
            int u = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int64_t c0 = t * kThTile;
                const int64_t cells = ncells - c0 < kThTile ? ncells - c0 : kThTile;
                const uint32_t bytes = (uint32_t)(((cells + 3) & ~int64_t(3)) * sizeof(in_t));
                for (int g = 0; g < groups; ++g, ++u) {
                    const int s = u % S;
                    if (!tc::mbar_wait(&empty[s], (uint32_t)((u / S) & 1) ^ 1u, spin)) {
                        atomicExch(err, 1u);
                        ok = false;
                        break;
                    }
                    const int r0 = g * kThRows, rows = (N + 1 - r0) < kThRows ? N + 1 - r0 : kThRows;
                    tc::mbar_arrive_expect_tx(&full[s], rows * bytes);
                    for (int r = 0; r < rows; ++r) {
                        const int q = r0 + r;          // state row: 0 = T, q = Y_{q-1}
                        const in_t *src = (q == 0 ? Tg : Yg + (int64_t)(q - 1) * ld) + c0;
                        tc::bulk_load_1d(stages + s * L::kStage + r * L::kRowBytes, src, bytes, &full[s]);
                    }
                }
            }
            // the last fill of each stage lands before the CTA may exit (full limit); u counts the
            // groups whose copies were issued
            for (int j = (u > S ? u - S : 0); j < u; ++j)
                if (!tc::mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u)) {
                    atomicExch(err, 1u);
                    break;
                }
        }
        return;
    }
    const float R = float(kR);
    int u = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i = t * kThTile + threadIdx.x;
        float T = 300.0f, iT = 1.0f / 300.0f, cpm = 0.0f, hm = 0.0f;
        const float4 *tr = tab;
        bool ok = true;
        for (int g = 0; g < groups; ++g, ++u) {
            const int s = u % S;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[s], (uint32_t)(u / S) & 1u, spin))) {
                ok = false;
                break;
            }
            const in_t *col = reinterpret_cast<const in_t *>(stages + s * L::kStage) + threadIdx.x;
            const int r0 = g * kThRows;
#pragma unroll
            for (int r = 0; r < kThRows; ++r) {
                const int q = r0 + r;
                if (q > N) break;
                const float v = to_real<float>(col[r * kThTile]);
                if (q == 0) {
                    T = v;
                    iT = 1.0f / T;
                    tr = tab + ((T >= T_mid) ? 3 * N : 0);
                    continue;
                }
                const int k = q - 1;
                const float4 q0 = tr[3 * k], q1 = tr[3 * k + 1], q2 = tr[3 * k + 2];
                float cpR = q1.x;
                cpR = fmaf(cpR, T, q0.w);
                cpR = fmaf(cpR, T, q0.z);
                cpR = fmaf(cpR, T, q0.y);
                cpR = fmaf(cpR, T, q0.x);
                float hR = q2.y;
                hR = fmaf(hR, T, q2.x);
                hR = fmaf(hR, T, q1.w);
                hR = fmaf(hR, T, q1.z);
                hR = fmaf(hR, T, q1.y);
                hR = fmaf(q2.z, iT, hR);
                const float yw = v * q2.w;
                cpm = fmaf(yw, cpR, cpm);
                hm = fmaf(yw, hR, hm);
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
        }
        if (!ok) {
            if (lane == 0) atomicExch(err, 1u);
            if (i < ncells) {
                if (cpg) cpg[i] = __int_as_float(0x7fc00000);
                if (hg) hg[i] = __int_as_float(0x7fc00000);
            }
            break;
        }
        if (i < ncells) {
            if (cpg) __stcs(cpg + i, cpm * R);
            if (hg) __stcs(hg + i, hm * R * T);
        }
    }
}

template <typename in_t>
int launch_thermo(const chem_mech *m, int64_t ncells, int64_t ld, const void *T, const void *Y, void *cp, void *h,
                  cudaStream_t st) {
    using L = ThLayout<in_t>;
    if (!aligned16(T) || !aligned16(Y) || (ld & 3) != 0)
        return set_error(CHEM_EINVAL, "props_eval: the state arrays must be 16-byte aligned and ld a multiple of 4");
    const size_t smem = L::bytes(m->N);
    static bool configured = false;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(thermo_kernel<in_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)L::bytes(kMaxSpecies)),
                            "props_eval (thermo) smem attribute");
        if (rc) return rc;
        configured = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (ncells + kThTile - 1) / kThTile;
    const int blocks = (int)(ntiles < sms ? ntiles : sms);
    void *pb = prof_begin(st);
    thermo_kernel<in_t><<<blocks, kThThreads, smem, st>>>(m->N, float(m->T_mid), m->dev.f32, ncells, ld,
                                                          static_cast<const in_t *>(T), static_cast<const in_t *>(Y),
                                                          static_cast<float *>(cp), static_cast<float *>(h),
                                                          m->dev.counters + kPropsErrCounter, tc::kSpinLimit);
    prof_end(pb, st, "thermo_kernel", (double)ncells * 24.0 * m->N,
             (double)ncells * ((m->N + 1) * sizeof(in_t) + 2 * sizeof(float)));
    return check_cuda(cudaGetLastError(), "props_eval (thermo) launch");
}

template <typename real, typename in_t, int NMAX>
int launch_props(const chem_mech *m, int64_t ncells, int64_t ld, const void *T, const void *p, const void *Y,
                 void *cp, void *h, void *mu, void *lam, void *Dk, cudaStream_t st) {
    const bool transport = mu || lam || Dk;
    const size_t smem = tables_in_smem<real>() ? ((transport ? (size_t)8 * m->N * m->dev.Np : 0) +
                                                  (size_t)kSpeciesFloats * m->N) * sizeof(real)
                                               : 0;
    static size_t configured = 0;
    if (smem > configured) {
        int rc = check_cuda(cudaFuncSetAttribute(props_kernel<real, in_t, NMAX>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPropsSmemMax),
                            "props_eval smem attribute");
        if (rc) return rc;
        configured = kPropsSmemMax;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, props_kernel<real, in_t, NMAX>, 128, smem);
    const int max_blocks = sms * (per_sm > 0 ? per_sm : 1);
    int64_t need = (ncells + 127) / 128;
    int blocks = (int)(need < max_blocks ? need : max_blocks);
    const PropTables<real> &tb = (sizeof(real) == 4) ? *reinterpret_cast<const PropTables<real> *>(&m->dev.f32)
                                                      : *reinterpret_cast<const PropTables<real> *>(&m->dev.f64);
    void *pb = prof_begin(st);
    props_kernel<real, in_t, NMAX><<<blocks, 128, smem, st>>>(
        m->N, m->dev.Np, real(m->T_mid), tb, ncells, ld, static_cast<const in_t *>(T), static_cast<const in_t *>(p),
        static_cast<const in_t *>(Y), static_cast<real *>(cp), static_cast<real *>(h), static_cast<real *>(mu),
        static_cast<real *>(lam), static_cast<real *>(Dk));
    prof_end(pb, st, std::string("props_kernel<") + (sizeof(real) == 4 ? "f32" : "f64") + ">",
             (double)ncells * (16.0 * m->N * m->N + 30.0 * m->N),
             (double)ncells * ((m->N + 2) * sizeof(in_t) + (4 + m->N) * sizeof(real)));
    return check_cuda(cudaGetLastError(), "props_eval launch");
}

template <typename real, typename in_t>
int dispatch_props(const chem_mech *m, int64_t ncells, int64_t ld, const void *T, const void *p, const void *Y,
                   void *cp, void *h, void *mu, void *lam, void *Dk, cudaStream_t st) {
    if constexpr (sizeof(real) == 4) {
        if (!mu && !lam && !Dk) return launch_thermo<in_t>(m, ncells, ld, T, Y, cp, h, st);
    }
    if (m->N <= 16) return launch_props<real, in_t, 16>(m, ncells, ld, T, p, Y, cp, h, mu, lam, Dk, st);
    if (m->N <= 32) return launch_props<real, in_t, 32>(m, ncells, ld, T, p, Y, cp, h, mu, lam, Dk, st);
    return launch_props<real, in_t, 64>(m, ncells, ld, T, p, Y, cp, h, mu, lam, Dk, st);
}

}  // namespace

// Properties (FP32 outputs from the FP64 state) of cells [0, ncells) for the learned step's
// fused entry point; the same kernels as props_eval(CHEM_F64_IN_F32).
int props_f64_in_f32(const chem_mech *m, int64_t ncells, int64_t ld, const double *T, const double *p,
                     const double *Y, float *cp, float *h, float *mu, float *lam, float *Dk, cudaStream_t st) {
    if (ncells <= 0) return CHEM_OK;
    return dispatch_props<float, double>(m, ncells, ld, T, p, Y, cp, h, mu, lam, Dk, st);
}

}  // namespace chemgb

using namespace chemgb;

extern "C" int props_eval(const chem_mech *m, int64_t ncells, int64_t ld, int dtype, const void *T, const void *p,
                          const void *Y, void *cp, void *h, void *mu, void *lambda, void *Dk,
                          chem_stream_t stream) {
    if (!m) return set_error(CHEM_EINVAL, "props_eval: null mechanism");
    if (ncells < 0 || ld < ncells || (ld & 3) != 0)
        return set_error(CHEM_EINVAL, "props_eval: need 0 <= ncells <= ld and ld a multiple of 4");
    if (dtype != CHEM_F32 && dtype != CHEM_F64 && dtype != CHEM_F64_IN_F32)
        return set_error(CHEM_EINVAL, "props_eval: bad dtype");
    if (ncells == 0) return CHEM_OK;
    if (!T || !p || !Y) return set_error(CHEM_EINVAL, "props_eval: null input array");
    const void *ptrs[] = {T, p, Y, cp, h, mu, lambda, Dk};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return set_error(CHEM_EINVAL, "props_eval: arrays must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "props_eval: " + why);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == CHEM_F32) return dispatch_props<float, float>(m, ncells, ld, T, p, Y, cp, h, mu, lambda, Dk, st);
    if (dtype == CHEM_F64_IN_F32)
        return dispatch_props<float, double>(m, ncells, ld, T, p, Y, cp, h, mu, lambda, Dk, st);
    return dispatch_props<double, double>(m, ncells, ld, T, p, Y, cp, h, mu, lambda, Dk, st);
}
