// gemm.cuh -- persistent, warp-specialised GEMM on the 5th-generation tensor
// cores: Y[M][N] = epilogue(X[M][K] * W[N][K]^T), FP32 accumulation, BF16 or
// FP8-E4M3 operands (the epilogue type says which). This is the dense
// contraction of every MLP layer (Sec. 3.2: hidden layers of 1600, 800 and 400
// GELU units), forward and backward.
//
// Roles (576 threads per CTA, one CTA per SM, static round-robin over tiles):
//   warp 0      TMA producer: 128-row tile of X and BN-row tile of W, 128 bytes
//               of K per row (64 BF16 or 128 E4M3), per k-block into a
//               STAGES-deep ring (128-byte swizzle).
//   warp 1      TMEM allocation and the single MMA-issuing thread:
//               tcgen05.mma kind::f16 (K = 16) or kind::f8f6f4 (K = 32),
//               M = 128, N = BN, four instructions per k-block,
//               accumulating in one of two TMEM buffers (columns 0 and 256).
//   warps 2..17 epilogue: four warps per TMEM lane quadrant (warp w reads TMEM
//               lanes 32 (w % 4) .. +31, i.e. output rows) split the 16-column
//               chunks between them; tcgen05.ld, then the functor. BF16 or
//               E4M3 GELU outputs are staged per warp in shared memory (double
//               buffered) and written by TMA tensor stores.
// Ragged M, N and K: TMA fills out-of-range operand elements with zeros, TMA
// stores clip at the tensor bounds, and direct stores mask rows >= M and
// columns >= N.
// Groups: one launch computes G independent products Y_g = epi_g(X_g W_g^T)
// of the same M, N, K (the per-species networks of Sec. 3.2 side by side).
// Each operand is either shared by all groups (a 2-D map) or a 3-D map whose
// third coordinate picks the group: stacked rows (group g's rows follow group
// g - 1's, as stacked weights) or side-by-side columns (group g's K columns
// follow group g - 1's in every row, as the activations of G networks). The
// 3-D box holds one group, so a ragged K or N clips at the group's own bound.
// Tiles run group-major, so a wave of CTAs shares one group's weights.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "tc.cuh"

namespace chemgb {

constexpr int kEpiWarps = 16;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kStageBytesPerWarp = 32 * 16 * 2;   // one 32 x 16 BF16 chunk
constexpr int kBM = 128;
constexpr int kBK = 64;                     // BF16 elements per k-block row (128 bytes)
constexpr int kBK8 = 128;                   // E4M3 elements per k-block row (128 bytes)
constexpr uint32_t kTmemCols = 512;

// operand / output map kinds of a grouped launch
enum : int { kMap2D = 0, kMapRowGrp = 1, kMapColGrp = 2 };
struct GemmGroups {
    int count;           // G >= 1
    int a, b, c;         // map kinds of X, W and the TMA-store output
    uint32_t spin;       // tries of a pipeline wait before it gives up (the closing drains always
                         // take tc::kSpinLimit, so that nothing is in flight when the CTA exits)
};

// load one box of a (k, row) tile of group g from a map of the given kind
__device__ __forceinline__ void load_tile(void *dst, const CUtensorMap *map, uint64_t *bar, int kind, int k, int row,
                                          int g) {
    if (kind == kMap2D) tc::tma_load_2d(dst, map, bar, k, row);
    else if (kind == kMapRowGrp) tc::tma_load_3d(dst, map, bar, k, row, g);
    else tc::tma_load_3d(dst, map, bar, k, g, row);
}
__device__ __forceinline__ void store_tile(const CUtensorMap *map, const void *src, int kind, int col, int row, int g) {
    if (kind == kMap2D) tc::tma_store_2d(map, src, col, row);
    else if (kind == kMapRowGrp) tc::tma_store_3d(map, src, col, row, g);
    else tc::tma_store_3d(map, src, col, g, row);
}

template <int BN, int STAGES>
struct GemmSmem {
    static constexpr uint32_t kABytes = kBM * kBK * 2;
    static constexpr uint32_t kBBytes = BN * kBK * 2;
    static constexpr uint32_t kTiles = STAGES * (kABytes + kBBytes);
    static constexpr uint32_t kStaging = kEpiWarps * 2 * kStageBytesPerWarp;
    static constexpr uint32_t kBars = (2 * STAGES + 5) * 8 + 16;
    static constexpr uint32_t kTotal = 1024 + kTiles + kStaging + kBars;
    static_assert(kBBytes % 1024 == 0, "B tile must keep 1024-byte alignment");
};

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- GELU (Sec. 3.2) ---------------------------------------------------------
// GELU(z) = z Phi(z) = h + |h| erf(sqrt(2) |h|) with h = z / 2. For a >= 0,
// erf(a) = 1 - erfcx(a) exp(-a^2), erfcx(a) = exp(a^2) erfc(a) (smooth, from 1 at 0
// down to about 1 / (sqrt(pi) a)). exp(-2 h^2) comes from the hardware exp2
// approximation, the one special-function operation per value; erfcx(sqrt(2) x),
// x = min(|h|, 4.5 / sqrt 2), from a degree-7 polynomial fitted by fit_erfcx.py
// (error of erf at most 8.0e-6 in FP32 Horner evaluation, so the GELU is within
// 3.3e-6 (1 + |z|) of z Phi(z), far below the BF16 rounding of the stored
// activations; past the clamp erfc < 4e-10). The coefficients are stored negated:
// the Horner sum is -erfcx. The packed form runs two values per FP32x2 instruction
// with the same operations in the same order as the scalar form, so both give the
// same bits.
constexpr float kGeluXmax = 3.18198052f;     // 4.5 / sqrt 2
constexpr float kNeg2Log2e = -2.88539008f;   // -2 log2(e): exp(-2 h^2) = exp2(h (h kNeg2Log2e))
// -erfcx(sqrt(2) x) on [0, 4.5 / sqrt 2]: Horner form of the fitted polynomial (coefficients negated)
__device__ __forceinline__ float neg_erfcx(float x) {
    float y = fmaf(0.0431515984f, x, -0.296845883f);
    y = fmaf(y, x, 0.891121089f);
    y = fmaf(y, x, -1.59809208f);
    y = fmaf(y, x, 2.01323724f);
    y = fmaf(y, x, -1.98367882f);
    y = fmaf(y, x, 1.59488058f);
    y = fmaf(y, x, -0.999992073f);
    return y;
}
__device__ __forceinline__ uint64_t neg_erfcx2(uint64_t x) {
    uint64_t y = fma2(pk2(0.0431515984f, 0.0431515984f), x, pk2(-0.296845883f, -0.296845883f));
    y = fma2(y, x, pk2(0.891121089f, 0.891121089f));
    y = fma2(y, x, pk2(-1.59809208f, -1.59809208f));
    y = fma2(y, x, pk2(2.01323724f, 2.01323724f));
    y = fma2(y, x, pk2(-1.98367882f, -1.98367882f));
    y = fma2(y, x, pk2(1.59488058f, 1.59488058f));
    y = fma2(y, x, pk2(-0.999992073f, -0.999992073f));
    return y;
}

__device__ __forceinline__ float gelu_exact(float z) {
    const float h = z * 0.5f;
    const float y = neg_erfcx(fminf(fabsf(h), kGeluXmax));
    const float e = ex2_approx((h * kNeg2Log2e) * h);
    const float s = fmaf(y, e, 1.0f);                 // erf(sqrt(2) |h|)
    return fmaf(fabsf(h), s, h);
}
// GELU(v0 + b0), GELU(v1 + b1): the scalar operations above, two lanes at a time
__device__ __forceinline__ void gelu_pair(float v0, float v1, float b0, float b1, float &g0, float &g1) {
    const uint64_t h = mul2(add2(pk2(v0, v1), pk2(b0, b1)), pk2(0.5f, 0.5f));
    float h0, h1;
    upk2(h, h0, h1);
    const uint64_t y = neg_erfcx2(pk2(fminf(fabsf(h0), kGeluXmax), fminf(fabsf(h1), kGeluXmax)));
    float m0, m1;
    upk2(mul2(mul2(h, pk2(kNeg2Log2e, kNeg2Log2e)), h), m0, m1);
    const uint64_t s = fma2(y, pk2(ex2_approx(m0), ex2_approx(m1)), pk2(1.0f, 1.0f));
    upk2(fma2(pk2(fabsf(h0), fabsf(h1)), s, h), g0, g1);
}
// dGELU/dz = Phi(z) + z phi(z), with the same erf and exp(-z^2 / 2) = exp(-2 h^2)
__device__ __forceinline__ float gelu_grad(float z) {
    const float h = z * 0.5f;
    const float y = neg_erfcx(fminf(fabsf(h), kGeluXmax));
    const float e = ex2_approx((h * kNeg2Log2e) * h);
    const float s = fmaf(y, e, 1.0f);                 // erf(|z| / sqrt 2)
    return fmaf(z * 0.39894228f, e, 0.5f + copysignf(0.5f * s, z));
}

// ---- epilogue functors: (row, first column, 16 accumulator values) --------

// Y = bf16(GELU(acc + b)); optionally also the FP32 pre-activation acc + b.
// Without a pre-activation the kernel stages the BF16 chunk and stores it by TMA.
struct EpiGelu {
    static constexpr bool kF8 = false;       // operand type: BF16
    static constexpr int kOutBytes = 32;     // bytes of a 16-column output chunk row (TMA store)
    int M, N;
    const float *bias;
    __nv_bfloat16 *out;
    int64_t ldo;
    float *pre;      // may be null
    int64_t ldp;
    int64_t g_out = 0, g_bias = 0, g_pre = 0;   // element offsets of group g's out, bias, pre: g x these
    __device__ __forceinline__ EpiGelu group(int g) const {
        EpiGelu e = *this;
        e.out += g * g_out;
        if (bias) e.bias += g * g_bias;
        if (pre) e.pre += g * g_pre;
        return e;
    }
    // TMA stores clip at 16-byte granularity in the row, so they are used only
    // when rows end on whole 16-column chunks (N % 16 == 0) with a 16-byte
    // aligned bias (read as float4)
    __host__ __device__ __forceinline__ bool tma_store() const {
        return pre == nullptr && (N & 15) == 0 && bias != nullptr && (reinterpret_cast<uintptr_t>(bias) & 15) == 0;
    }
    const void *tma_ptr() const { return tma_store() ? out : nullptr; }
    // the 16 BF16 values of (row, col0..col0+15), two per 32-bit word (N % 8 == 0 on this path,
    // and the bias is padded to whole 16-float groups)
    __device__ __forceinline__ void compute(int col0, const float (&v)[16], uint32_t (&w)[8]) const {
        float b[16];
        const float4 *bp = reinterpret_cast<const float4 *>(bias + col0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 q = __ldg(bp + i);
            b[4 * i] = q.x; b[4 * i + 1] = q.y; b[4 * i + 2] = q.z; b[4 * i + 3] = q.w;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float g0, g1;
            gelu_pair(v[2 * i], v[2 * i + 1], b[2 * i], b[2 * i + 1], g0, g1);
            __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
    }
    __device__ __forceinline__ void operator()(int row, int col0, const float (&v)[16]) const {
        if (row >= M) return;
        float z[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = v[i] + ((col0 + i < N && bias) ? __ldg(bias + col0 + i) : 0.0f);
        __nv_bfloat16 *o = out + (int64_t)row * ldo + col0;
        if (col0 + 16 <= N && (ldo & 7) == 0) {
            __align__(16) __nv_bfloat162 h[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(gelu_exact(z[2 * i]), gelu_exact(z[2 * i + 1]));
            reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(h)[0];
            reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(h)[1];
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (col0 + i < N) o[i] = __float2bfloat16_rn(gelu_exact(z[i]));
        }
        if (pre) {
            float *q = pre + (int64_t)row * ldp + col0;
            if (col0 + 16 <= N && (ldp & 3) == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    reinterpret_cast<float4 *>(q)[i] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (col0 + i < N) q[i] = z[i];
            }
        }
    }
};

// Y = acc + b in FP32 (b may be null).
struct EpiLinear {
    static constexpr bool kF8 = false;
    static constexpr int kOutBytes = 32;
    int M, N;
    const float *bias;
    float *out;
    int64_t ldo;
    int64_t g_out = 0, g_bias = 0;
    __device__ __forceinline__ EpiLinear group(int g) const {
        EpiLinear e = *this;
        e.out += g * g_out;
        if (bias) e.bias += g * g_bias;
        return e;
    }
    __host__ __device__ __forceinline__ bool tma_store() const { return false; }
    const void *tma_ptr() const { return nullptr; }
    __device__ __forceinline__ void compute(int, const float (&)[16], uint32_t (&)[8]) const {}
    __device__ __forceinline__ void operator()(int row, int col0, const float (&v)[16]) const {
        if (row >= M) return;
        float *o = out + (int64_t)row * ldo + col0;
        if (col0 + 16 <= N && (ldo & 3) == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float4 t;
                t.x = v[4 * i] + (bias ? __ldg(bias + col0 + 4 * i) : 0.0f);
                t.y = v[4 * i + 1] + (bias ? __ldg(bias + col0 + 4 * i + 1) : 0.0f);
                t.z = v[4 * i + 2] + (bias ? __ldg(bias + col0 + 4 * i + 2) : 0.0f);
                t.w = v[4 * i + 3] + (bias ? __ldg(bias + col0 + 4 * i + 3) : 0.0f);
                reinterpret_cast<float4 *>(o)[i] = t;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (col0 + i < N) o[i] = v[i] + (bias ? __ldg(bias + col0 + i) : 0.0f);
        }
    }
};

// Y = bf16(acc * GELU'(Z)), Z the FP32 pre-activation of the layer below (backward pass).
struct EpiGeluGrad {
    static constexpr bool kF8 = false;
    static constexpr int kOutBytes = 32;
    int M, N;
    const float *z;
    int64_t ldz;
    __nv_bfloat16 *out;
    int64_t ldo;
    int64_t g_z = 0, g_out = 0;
    __device__ __forceinline__ EpiGeluGrad group(int g) const {
        EpiGeluGrad e = *this;
        e.z += g * g_z;
        e.out += g * g_out;
        return e;
    }
    __host__ __device__ __forceinline__ bool tma_store() const { return false; }
    const void *tma_ptr() const { return nullptr; }
    __device__ __forceinline__ void compute(int, const float (&)[16], uint32_t (&)[8]) const {}
    __device__ __forceinline__ void operator()(int row, int col0, const float (&v)[16]) const {
        if (row >= M) return;
        const float *zr = z + (int64_t)row * ldz + col0;
        __nv_bfloat16 *o = out + (int64_t)row * ldo + col0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (col0 + i < N) o[i] = __float2bfloat16_rn(v[i] * gelu_grad(zr[i]));
    }
};

// Hidden layers of the reduced-precision forward. z = acc * cs[n] + b[n], where
// cs = (weight scale of output n) x (input activation scale) when the operands
// are E4M3 (F8IN) and 1 otherwise; h = GELU(z), stored as E4M3(h * inv_so)
// with round-to-nearest-even and saturation at +-448 (F8OUT) or as BF16(h).
template <bool F8IN, bool F8OUT>
struct EpiGeluQ {
    static constexpr bool kF8 = F8IN;
    static constexpr int kOutBytes = F8OUT ? 16 : 32;
    int M, N;
    const float *bias;    // [N, padded to a multiple of 16]
    const float *cs;      // [N, padded to a multiple of 16]; used when F8IN
    void *out;
    int64_t ldo;          // elements
    float inv_so;         // used when F8OUT
    __device__ __forceinline__ EpiGeluQ group(int) const { return *this; }   // launched ungrouped
    __host__ __device__ __forceinline__ bool tma_store() const {
        return (N & 15) == 0 && (reinterpret_cast<uintptr_t>(bias) & 15) == 0 &&
               (!F8IN || (reinterpret_cast<uintptr_t>(cs) & 15) == 0);
    }
    const void *tma_ptr() const { return tma_store() ? out : nullptr; }
    __device__ __forceinline__ float act(float v, float c, float b) const {
        return gelu_exact(F8IN ? fmaf(v, c, b) : v + b);
    }
    __device__ __forceinline__ void compute(int col0, const float (&v)[16], uint32_t (&w)[8]) const {
        float b[16], c[16];
        const float4 *bp = reinterpret_cast<const float4 *>(bias + col0);
        const float4 *cp = reinterpret_cast<const float4 *>(cs + col0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 q = __ldg(bp + i);
            b[4 * i] = q.x; b[4 * i + 1] = q.y; b[4 * i + 2] = q.z; b[4 * i + 3] = q.w;
            if (F8IN) {
                const float4 r = __ldg(cp + i);
                c[4 * i] = r.x; c[4 * i + 1] = r.y; c[4 * i + 2] = r.z; c[4 * i + 3] = r.w;
            } else {
                c[4 * i] = c[4 * i + 1] = c[4 * i + 2] = c[4 * i + 3] = 1.0f;
            }
        }
        if (F8OUT) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
                    make_float2(act(v[4 * i], c[4 * i], b[4 * i]) * inv_so,
                                act(v[4 * i + 1], c[4 * i + 1], b[4 * i + 1]) * inv_so),
                    __NV_SATFINITE, __NV_E4M3);
                const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                    make_float2(act(v[4 * i + 2], c[4 * i + 2], b[4 * i + 2]) * inv_so,
                                act(v[4 * i + 3], c[4 * i + 3], b[4 * i + 3]) * inv_so),
                    __NV_SATFINITE, __NV_E4M3);
                w[i] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                __nv_bfloat162 h = __floats2bfloat162_rn(act(v[2 * i], c[2 * i], b[2 * i]),
                                                         act(v[2 * i + 1], c[2 * i + 1], b[2 * i + 1]));
                w[i] = *reinterpret_cast<uint32_t *>(&h);
            }
        }
    }
    // ragged output widths: element stores, columns >= N skipped
    __device__ __forceinline__ void operator()(int row, int col0, const float (&v)[16]) const {
        if (row >= M) return;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int col = col0 + i;
            if (col >= N) break;
            const float h = act(v[i], F8IN ? __ldg(cs + col) : 1.0f, __ldg(bias + col));
            if (F8OUT)
                static_cast<__nv_fp8_storage_t *>(out)[(int64_t)row * ldo + col] =
                    __nv_cvt_float_to_fp8(h * inv_so, __NV_SATFINITE, __NV_E4M3);
            else
                static_cast<__nv_bfloat16 *>(out)[(int64_t)row * ldo + col] = __float2bfloat16_rn(h);
        }
    }
};

// ---- kernel ---------------------------------------------------------------

template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, int M, int N, int K, GemmGroups grp, Epi epi, int *err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    using L = GemmSmem<BN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * L::kABytes;
    uint8_t *staging = smem + L::kTiles;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kTiles + L::kStaging);
    uint64_t *full = bars;
    uint64_t *empty = bars + STAGES;
    uint64_t *tfull = bars + 2 * STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (M + kBM - 1) / kBM, n_tiles = (N + BN - 1) / BN;
    const int group_tiles = m_tiles * n_tiles;
    const int tiles = group_tiles * grp.count;
    constexpr int kBKe = Epi::kF8 ? kBK8 : kBK;   // elements of K per k-block
    const int kblocks = (K + kBKe - 1) / kBKe;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&tfull[a], 1); tc::mbar_init(&tempty[a], kEpiWarps); }
        tc::mbar_init(drain, 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmA);
            tc::tma_prefetch_desc(&tmB);
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
                const int g = tile / group_tiles, r = tile - g * group_tiles;
                const int m_blk = r / n_tiles, n_blk = r % n_tiles;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1u, grp.spin)) { atomicExch(err, tc::kErrTimeoutEmpty); ok = false; break; }
                    tc::mbar_arrive_expect_tx(&full[s], L::kABytes + L::kBBytes);
                    load_tile(sA + s * L::kABytes, &tmA, &full[s], grp.a, kb * kBKe, m_blk * kBM, g);
                    load_tile(sB + s * L::kBBytes, &tmB, &full[s], grp.b, kb * kBKe, n_blk * BN, g);
                }
            }
            // every issued load lands before the CTA may exit (bounded)
            for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
                if (!tc::mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u)) {
                    atomicExch(err, tc::kErrTimeoutDrain);
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = Epi::kF8 ? tc::idesc_e4m3_f32(kBM, BN) : tc::idesc_bf16_f32(kBM, BN);
            int it = 0, t = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++t) {
                const int acc = t & 1;
                const uint32_t aph = (uint32_t)(t >> 1) & 1u;
                if (!tc::mbar_wait(&tempty[acc], aph ^ 1u, grp.spin)) { atomicExch(err, tc::kErrTimeoutTmemEmpty); break; }
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)acc * 256u;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!tc::mbar_wait(&full[s], ph, grp.spin)) { atomicExch(err, tc::kErrTimeoutFull); ok = false; break; }
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(sA + s * L::kABytes);
                    const uint32_t b0 = tc::smem_u32(sB + s * L::kBBytes);
                    // four instructions of 32 bytes of K each (16 BF16 or 32 E4M3)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = tc::sdesc_kmajor_sw128(a0 + kk * 32), bd = tc::sdesc_kmajor_sw128(b0 + kk * 32);
                        if (Epi::kF8) tc::umma_f8(d_tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                        else tc::umma_f16(d_tmem, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    tc::umma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::umma_commit(&tfull[acc]);
            }
            // all MMAs issued by this thread complete before TMEM is released (bounded)
            tc::umma_commit(drain);
            if (!tc::mbar_wait(drain, 0)) atomicExch(err, tc::kErrTimeoutDrain);
        }
    } else {
        const int quad = warp & 3;
        const int group = (warp - 2) >> 2;          // 0..3: which quarter of the column chunks
        const bool tma = epi.tma_store();
        uint8_t *my_stage = staging + (size_t)(warp - 2) * 2 * kStageBytesPerWarp;
        int nstore = 0;
        if (tma && lane == 0) tc::tma_prefetch_desc(&tmC);
        int t = 0;
        for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++t) {
            const int acc = t & 1;
            const uint32_t aph = (uint32_t)(t >> 1) & 1u;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&tfull[acc], aph, grp.spin))) {   // warp-uniform outcome
                if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                break;
            }
            tc::tc_fence_after();
            const int g = tile / group_tiles, r = tile - g * group_tiles;
            const int m_blk = r / n_tiles, n_blk = r % n_tiles;
            const Epi ge = epi.group(g);
            const int row0 = m_blk * kBM + quad * 32;
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)acc * 256u;
#pragma unroll 1
            for (int c = group; c < BN / 16; c += kEpiWarps / 4) {
                const int col0 = n_blk * BN + c * 16;
                if (col0 >= N) break;               // warp-uniform
                float v[16];
                tc::tmem_ld16(tbase + (uint32_t)(c * 16), v);
                if (tma) {
                    if (row0 >= M) continue;            // warp-uniform: nothing of this slice is in range
                    uint32_t w[8];
                    ge.compute(col0, v, w);
                    uint8_t *buf = my_stage + (nstore & 1) * kStageBytesPerWarp;
                    if (nstore >= 2 && lane == 0) tc::bulk_wait_read<1>();   // this buffer's previous store has read it
                    __syncwarp();
                    uint4 *dst = reinterpret_cast<uint4 *>(buf + lane * Epi::kOutBytes);
                    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    if (Epi::kOutBytes == 32) dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        store_tile(&tmC, buf, grp.c, col0, row0, g);
                        tc::bulk_commit();
                    }
                    ++nstore;
                } else {
                    ge(row0 + lane, col0, v);
                }
            }
            // one arrival per warp once all its lanes' TMEM reads are done
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[acc]);
        }
        if (tma && lane == 0) tc::bulk_wait<0>();    // stores complete before the CTA exits
        __syncwarp();
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace chemgb
