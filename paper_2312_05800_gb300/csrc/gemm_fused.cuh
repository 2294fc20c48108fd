// gemm_fused.cuh -- the network's first two layers in one persistent launch:
// h2 = GELU(GELU(X W1^T + b1) W2^T + b2) (Sec. 3.2: the hidden layers of 1600
// and 800 GELU units), with the first hidden layer h1 made on chip and never
// written to memory.
//
// Per 128-row tile of X (the prologue's hi|lo BF16 rows, one 128-byte k-block)
// and per pass over NP columns of layer 2's output:
//   for each 64-column chunk c of h1:
//     MMA1   D1 = X W1[64c .. 64c + 63]^T                 (TMEM, 64 columns)
//     GELU   A2 = bf16(GELU(D1 + b1)), written by the epilogue warps straight
//            into shared memory in the 128-byte-swizzled K-major layout a TMA
//            load would produce, so it is layer 2's A operand for k-block c
//     MMA2   D2 += A2 W2[pass rows][64c .. 64c + 63]^T    (TMEM, NP columns)
//   epilogue: h2 = bf16(GELU(D2 + b2)) by TMA stores.
// D2 (NP <= 448 columns) and D1 (64 columns) share the SM's 512 TMEM columns,
// so layer 2's 800 outputs take two passes, each recomputing h1: the extra
// GELUs cost less than the 2 x 1600 x 2 bytes per row that an h1 round trip
// through HBM would (h1 is 13 GB per 4M-cell step). The MMA thread issues
// MMA1 for chunk c + 1 before MMA2 for chunk c, so the tensor pipe works on
// layer 2 while the epilogue warps apply GELU to the next chunk.
// Every element's FP32 sums take the same k order as the two-launch path
// (gemm_tn_kernel), so the results are bitwise those of layer 1 then layer 2.
//
// Roles (576 threads, one CTA per SM):
//   warp 0      TMA producer: X tiles (2-stage ring, one per row tile), W1
//               chunks (3-stage ring), W2 chunks (2-stage ring, two boxes of
//               NP/2 rows).
//   warp 1      TMEM allocation; one thread issues every tcgen05.mma.
//   warps 2-17  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows);
//               for h1 each takes 16 of a chunk's 64 columns, for h2 the
//               16-column slices of the pass in turn.
// Every wait is bounded (a.spin tries); one that runs out records its code
// and the kernel unwinds as gemm_tn_kernel does.
#pragma once

#include "gemm.cuh"

namespace chemgb {

constexpr int kF12Chunk = 64;             // h1 columns per chunk = layer-2 K per k-block
constexpr int kF12XStages = 2;
constexpr int kF12W1Stages = 3;
constexpr int kF12W2Stages = 2;
constexpr int kF12A2Stages = 2;
constexpr uint32_t kF12D1Col = 448;       // TMEM column of D1 (D2 takes columns 0 .. NP - 1, NP <= 448)

template <int NP>
struct F12Smem {
    static_assert(NP % 16 == 0 && NP >= 32 && NP <= 448, "pass width: UMMA N pieces of <= 256, D1 after D2");
    static constexpr uint32_t kX = kBM * 128;                 // 128 rows x 128 bytes
    static constexpr uint32_t kW1 = kF12Chunk * 128;          // 64 rows x 128 bytes
    static constexpr uint32_t kW2 = NP * 128;                 // NP rows x 128 bytes
    static constexpr uint32_t kA2 = kBM * 128;
    static constexpr uint32_t kStaging = kEpiWarps * 2 * kStageBytesPerWarp;
    static constexpr uint32_t oX = 0;
    static constexpr uint32_t oW1 = oX + kF12XStages * kX;
    static constexpr uint32_t oW2 = oW1 + kF12W1Stages * kW1;
    static constexpr uint32_t oA2 = oW2 + kF12W2Stages * kW2;
    static constexpr uint32_t oStage = oA2 + kF12A2Stages * kA2;
    static constexpr uint32_t oBars = oStage + kStaging;
    static constexpr int kNumBars = 2 * kF12XStages + 2 * kF12W1Stages + 2 * kF12W2Stages + 2 + 2 * kF12A2Stages + 2 + 1;
    static constexpr uint32_t kTotal = 1024 + oBars + kNumBars * 8 + 16;
    static_assert(kW2 % 1024 == 0 && (NP / 2) % 8 == 0, "W2 boxes keep 1024-byte alignment");
    static_assert(kTotal <= 232448, "shared memory per CTA");
};

struct F12Args {
    int M;               // rows
    int N1;              // layer-1 outputs (a multiple of 64)
    int N2;              // layer-2 outputs
    int passes;          // ceil(N2 / NP)
    const float *b1;     // [N1], 16-byte aligned
    const float *b2;     // [passes x NP] readable (padded), 16-byte aligned
    uint32_t spin;       // tries of a pipeline wait
};

template <int NP>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_fused12_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                        const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmH2, F12Args a,
                        int *err) {
    using L = F12Smem<NP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sX = smem + L::oX;
    uint8_t *sW1 = smem + L::oW1;
    uint8_t *sW2 = smem + L::oW2;
    uint8_t *sA2 = smem + L::oA2;
    uint8_t *staging = smem + L::oStage;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::oBars);
    uint64_t *x_full = bars, *x_empty = bars + kF12XStages;
    uint64_t *w1_full = x_empty + kF12XStages, *w1_empty = w1_full + kF12W1Stages;
    uint64_t *w2_full = w1_empty + kF12W1Stages, *w2_empty = w2_full + kF12W2Stages;
    uint64_t *d1_full = w2_empty + kF12W2Stages, *d1_empty = d1_full + 1;
    uint64_t *a2_full = d1_empty + 1, *a2_empty = a2_full + kF12A2Stages;
    uint64_t *d2_full = a2_empty + kF12A2Stages, *d2_empty = d2_full + 1;
    uint64_t *drain = d2_empty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (a.M + kBM - 1) / kBM;
    const int chunks = a.N1 / kF12Chunk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kF12XStages; ++s) { tc::mbar_init(&x_full[s], 1); tc::mbar_init(&x_empty[s], 1); }
        for (int s = 0; s < kF12W1Stages; ++s) { tc::mbar_init(&w1_full[s], 1); tc::mbar_init(&w1_empty[s], 1); }
        for (int s = 0; s < kF12W2Stages; ++s) { tc::mbar_init(&w2_full[s], 1); tc::mbar_init(&w2_empty[s], 1); }
        tc::mbar_init(d1_full, 1);
        tc::mbar_init(d1_empty, kEpiWarps);
        for (int s = 0; s < kF12A2Stages; ++s) { tc::mbar_init(&a2_full[s], kEpiWarps); tc::mbar_init(&a2_empty[s], 1); }
        tc::mbar_init(d2_full, 1);
        tc::mbar_init(d2_empty, kEpiWarps);
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
            tc::tma_prefetch_desc(&tmX);
            tc::tma_prefetch_desc(&tmW1);
            tc::tma_prefetch_desc(&tmW2);
            int xi = 0, w1i = 0, w2i = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x, ++xi) {
                const int sx = xi % kF12XStages;
                if (!tc::mbar_wait(&x_empty[sx], (uint32_t)((xi / kF12XStages) & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutEmpty);
                    ok = false;
                    break;
                }
                tc::mbar_arrive_expect_tx(&x_full[sx], L::kX);
                tc::tma_load_2d(sX + sx * L::kX, &tmX, &x_full[sx], 0, tile * kBM);
                for (int p = 0; p < a.passes && ok; ++p) {
                    for (int c = 0; c < chunks; ++c) {
                        const int s1 = w1i % kF12W1Stages;
                        if (!tc::mbar_wait(&w1_empty[s1], (uint32_t)((w1i / kF12W1Stages) & 1) ^ 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutEmpty);
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&w1_full[s1], L::kW1);
                        tc::tma_load_2d(sW1 + s1 * L::kW1, &tmW1, &w1_full[s1], 0, c * kF12Chunk);
                        ++w1i;
                        const int s2 = w2i % kF12W2Stages;
                        if (!tc::mbar_wait(&w2_empty[s2], (uint32_t)((w2i / kF12W2Stages) & 1) ^ 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutEmpty);
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&w2_full[s2], L::kW2);
                        uint8_t *dst = sW2 + s2 * L::kW2;
                        tc::tma_load_2d(dst, &tmW2, &w2_full[s2], c * kF12Chunk, p * NP);
                        tc::tma_load_2d(dst + (NP / 2) * 128, &tmW2, &w2_full[s2], c * kF12Chunk, p * NP + NP / 2);
                        ++w2i;
                    }
                }
            }
            // every issued load lands before the CTA may exit (full limit): the last load into each
            // stage of each ring (xi counts the X tiles whose load was issued: a failed wait on
            // x_empty leaves the loop before the increment, any later failure after it)
            for (int j = (xi > kF12XStages ? xi - kF12XStages : 0); j < xi; ++j)
                if (!tc::mbar_wait(&x_full[j % kF12XStages], (uint32_t)(j / kF12XStages) & 1u)) {
                    atomicExch(err, tc::kErrTimeoutDrain);
                    break;
                }
            for (int j = (w1i > kF12W1Stages ? w1i - kF12W1Stages : 0); j < w1i; ++j)
                if (!tc::mbar_wait(&w1_full[j % kF12W1Stages], (uint32_t)(j / kF12W1Stages) & 1u)) {
                    atomicExch(err, tc::kErrTimeoutDrain);
                    break;
                }
            for (int j = (w2i > kF12W2Stages ? w2i - kF12W2Stages : 0); j < w2i; ++j)
                if (!tc::mbar_wait(&w2_full[j % kF12W2Stages], (uint32_t)(j / kF12W2Stages) & 1u)) {
                    atomicExch(err, tc::kErrTimeoutDrain);
                    break;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc1 = tc::idesc_bf16_f32(kBM, kF12Chunk);
            constexpr int kNA = NP > 256 ? 256 : NP;          // D2 in at most two UMMA N pieces
            constexpr int kNB = NP - kNA;
            constexpr uint32_t idescA = tc::idesc_bf16_f32(kBM, kNA);
            constexpr uint32_t idescB = tc::idesc_bf16_f32(kBM, kNB > 0 ? kNB : 16);
            const uint32_t d1 = tmem + kF12D1Col, d2 = tmem;
            int xi = 0, w1i = 0, w2i = 0, d1i = 0, a2i = 0, pi = 0;
            bool ok = true;
            // MMA1 for h1 chunk c: D1 = X W1_c^T (one k-block, four K = 16 steps)
            auto mma1 = [&](int) -> bool {
                const int s1 = w1i % kF12W1Stages;
                if (!tc::mbar_wait(&w1_full[s1], (uint32_t)(w1i / kF12W1Stages) & 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    return false;
                }
                if (!tc::mbar_wait(d1_empty, (uint32_t)(d1i & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutTmemEmpty);
                    return false;
                }
                tc::tc_fence_after();
                const uint32_t xa = tc::smem_u32(sX + (xi % kF12XStages) * L::kX), wb = tc::smem_u32(sW1 + s1 * L::kW1);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::umma_f16(d1, tc::sdesc_kmajor_sw128(xa + kk * 32), tc::sdesc_kmajor_sw128(wb + kk * 32),
                                 idesc1, kk > 0 ? 1u : 0u);
                tc::umma_commit(&w1_empty[s1]);
                tc::umma_commit(d1_full);
                ++w1i;
                ++d1i;
                return true;
            };
            // MMA2 for chunk c of a pass: D2 (+)= A2_c W2_c^T
            auto mma2 = [&](int c) -> bool {
                const int sa = a2i % kF12A2Stages, s2 = w2i % kF12W2Stages;
                if (c == 0 && !tc::mbar_wait(d2_empty, (uint32_t)(pi & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutTmemEmpty);
                    return false;
                }
                if (!tc::mbar_wait(&w2_full[s2], (uint32_t)(w2i / kF12W2Stages) & 1u, a.spin) ||
                    !tc::mbar_wait(&a2_full[sa], (uint32_t)(a2i / kF12A2Stages) & 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    return false;
                }
                tc::tc_fence_after();
                const uint32_t aa = tc::smem_u32(sA2 + sa * L::kA2), wb = tc::smem_u32(sW2 + s2 * L::kW2);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = tc::sdesc_kmajor_sw128(aa + kk * 32);
                    const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                    tc::umma_f16(d2, ad, tc::sdesc_kmajor_sw128(wb + kk * 32), idescA, acc);
                    if (kNB > 0)
                        tc::umma_f16(d2 + kNA, ad, tc::sdesc_kmajor_sw128(wb + kNA * 128 + kk * 32), idescB, acc);
                }
                tc::umma_commit(&w2_empty[s2]);
                tc::umma_commit(&a2_empty[sa]);
                ++w2i;
                ++a2i;
                return true;
            };
            for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x, ++xi) {
                if (!tc::mbar_wait(&x_full[xi % kF12XStages], (uint32_t)((xi / kF12XStages) & 1), a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    break;
                }
                for (int p = 0; p < a.passes && ok; ++p, ++pi) {
                    if (!mma1(0)) { ok = false; break; }
                    for (int c = 0; c < chunks; ++c) {
                        if (c + 1 < chunks && !mma1(c + 1)) { ok = false; break; }
                        if (!mma2(c)) { ok = false; break; }
                    }
                    if (!ok) break;
                    tc::umma_commit(d2_full);
                }
                if (!ok) break;
                tc::umma_commit(&x_empty[xi % kF12XStages]);     // the tile's MMA1s are done with X
            }
            // all MMAs issued by this thread complete before TMEM is released (full limit)
            tc::umma_commit(drain);
            if (!tc::mbar_wait(drain, 0)) atomicExch(err, tc::kErrTimeoutDrain);
        }
    } else {
        const int quad = warp & 3;                  // TMEM lane quadrant = rows 32 quad .. + 31 of the tile
        const int group = (warp - 2) >> 2;          // 0..3
        const int r = quad * 32 + lane;             // this thread's row of the tile
        uint8_t *my_stage = staging + (size_t)(warp - 2) * 2 * kStageBytesPerWarp;
        int nstore = 0, d1i = 0, a2i = 0, pi = 0;
        bool ok = true;
        if (lane == 0) tc::tma_prefetch_desc(&tmH2);
        const uint32_t tq = (uint32_t)(quad * 32) << 16;
        for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x) {
            const int row0 = tile * kBM + quad * 32;
            for (int p = 0; p < a.passes && ok; ++p, ++pi) {
                // this warp's 16 biases of chunk 0, then of each next chunk ahead of its wait
                float4 bq[4];
                {
                    const float4 *bp = reinterpret_cast<const float4 *>(a.b1 + group * 16);
#pragma unroll
                    for (int i = 0; i < 4; ++i) bq[i] = __ldg(bp + i);
                }
                for (int c = 0; c < chunks; ++c, ++d1i, ++a2i) {
                    float b[16];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        b[4 * i] = bq[i].x; b[4 * i + 1] = bq[i].y; b[4 * i + 2] = bq[i].z; b[4 * i + 3] = bq[i].w;
                    }
                    if (c + 1 < chunks) {
                        const float4 *bp = reinterpret_cast<const float4 *>(a.b1 + (c + 1) * kF12Chunk + group * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i) bq[i] = __ldg(bp + i);
                    }
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(d1_full, (uint32_t)(d1i & 1), a.spin))) {
                        if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    float v[16];
                    tc::tmem_ld16(tmem + tq + kF12D1Col + (uint32_t)(group * 16), v);
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(d1_empty);
                    // GELU(D1 + b1) of columns 64 c + 16 group .. + 15 as 8 packed BF16 pairs
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float g0, g1;
                        gelu_pair(v[2 * i], v[2 * i + 1], b[2 * i], b[2 * i + 1], g0, g1);
                        __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
                        w[i] = *reinterpret_cast<uint32_t *>(&h);
                    }
                    // layer 2's A operand: row r, 16-byte chunks 2 group and 2 group + 1 of the 128-byte
                    // k-block, at the 128-byte swizzle positions chunk ^ (r % 8)
                    const int sa = a2i % kF12A2Stages;
                    if (!__all_sync(0xffffffffu,
                                    tc::mbar_wait(&a2_empty[sa], (uint32_t)((a2i / kF12A2Stages) & 1) ^ 1u, a.spin))) {
                        if (lane == 0) atomicExch(err, tc::kErrTimeoutEmpty);
                        ok = false;
                        break;
                    }
                    uint8_t *rowp = sA2 + sa * L::kA2 + r * 128;
                    const int j0 = group * 2;
                    *reinterpret_cast<uint4 *>(rowp + (((j0) ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(rowp + (((j0 + 1) ^ (r & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&a2_full[sa]);
                }
                if (!ok) break;
                // the pass's h2 columns p NP .. + NP - 1: GELU(D2 + b2), BF16, TMA stores
                if (!__all_sync(0xffffffffu, tc::mbar_wait(d2_full, (uint32_t)(pi & 1), a.spin))) {
                    if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
#pragma unroll 1
                for (int j = group; j < NP / 16; j += kEpiWarps / 4) {
                    const int col0 = p * NP + j * 16;
                    if (col0 >= a.N2) break;             // warp-uniform
                    float v[16];
                    tc::tmem_ld16(tmem + tq + (uint32_t)(j * 16), v);
                    if (row0 >= a.M) continue;           // warp-uniform: no row of this slice is in range
                    float b[16];
                    const float4 *bp = reinterpret_cast<const float4 *>(a.b2 + col0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 q = __ldg(bp + i);
                        b[4 * i] = q.x; b[4 * i + 1] = q.y; b[4 * i + 2] = q.z; b[4 * i + 3] = q.w;
                    }
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float g0, g1;
                        gelu_pair(v[2 * i], v[2 * i + 1], b[2 * i], b[2 * i + 1], g0, g1);
                        __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
                        w[i] = *reinterpret_cast<uint32_t *>(&h);
                    }
                    uint8_t *buf = my_stage + (nstore & 1) * kStageBytesPerWarp;
                    if (nstore >= 2 && lane == 0) tc::bulk_wait_read<1>();
                    __syncwarp();
                    uint4 *dst = reinterpret_cast<uint4 *>(buf + lane * 32);
                    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tc::tma_store_2d(&tmH2, buf, col0, row0);
                        tc::bulk_commit();
                    }
                    ++nstore;
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(d2_empty);
            }
        }
        if (lane == 0) tc::bulk_wait<0>();         // stores complete before the CTA exits
        __syncwarp();
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace chemgb
