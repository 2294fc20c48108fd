// gemm_fused34.cuh -- the network's last hidden layer and its output layer in
// one persistent launch: u = GELU(X W3^T + b3) W4^T + b4 (Sec. 3.2: the hidden
// layer of 400 GELU units and the linear output of the normalised dY), with
// the hidden activation h3 made on chip and never written to memory.
//
// Per 128-row tile of X (= h2, K3 columns) the layer-3 accumulator is split in
// two halves held in TMEM side by side, D3A (columns 0 .. NA - 1) and D3B
// (NA .. N3 - 1), each computed over all K3 by its own pass over X and W3.
// While the MMA thread computes one half, the epilogue warps turn the other
// half into bf16(GELU(D3 + b3)) and write it into shared memory as 64-column
// k-blocks of the output layer's A operand (the 128-byte-swizzled K-major
// layout a TMA load would produce). A second MMA thread multiplies each such
// k-block with the resident W4 (N4 <= 32 rows) into D4 (double-buffered, 32
// TMEM columns each); after a tile's last k-block the epilogue warps add b4
// and store u in FP32. Every element's sums take the same k order as the
// two-launch path (layer 3, then layer 4 on the stored h3), so u is bitwise
// that of the two launches.
//
// Roles (608 threads, one CTA per SM):
//   warp 0      TMA producer: X and W3 k-blocks in a 3-stage ring (W3 rows of
//               the half being computed), W4 once per CTA.
//   warp 1      TMEM allocation; one thread issues the layer-3 MMAs.
//   warp 2      one thread issues the output layer's MMAs.
//   warps 3-18  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31.
// Every wait is bounded (a.spin tries); one that runs out records its code
// and the kernel unwinds: the producer waits (full limit) for its issued
// copies, each MMA thread for its issued MMAs, then TMEM is freed.
#pragma once

#include "gemm.cuh"

namespace chemgb {

constexpr int kF34Stages = 3;            // X / W3 ring
constexpr int kF34A4Stages = 4;          // output-layer A operand ring (64-column k-blocks of h3)
constexpr int kF34Threads = 32 * 19;
constexpr uint32_t kF34D4Col = 448;      // TMEM columns of D4: 448 .. 479 and 480 .. 511

template <int NA, int NB>
struct F34Smem {
    static_assert(NA % 64 == 0 && NB % 16 == 0 && NA + NB <= 448 && NB <= 256 && NA <= 256, "halves");
    static constexpr int kK4 = (NA + NB + 63) / 64;           // output-layer k-blocks (64 columns)
    static constexpr uint32_t kX = kBM * 128;
    static constexpr uint32_t kW3 = (NA > NB ? NA : NB) * 128;
    static constexpr uint32_t kA4 = kBM * 128;
    static constexpr uint32_t kW4 = 32 * 128;                 // one 64-column k-block of W4 (32 rows)
    static constexpr uint32_t oX = 0;
    static constexpr uint32_t oW3 = oX + kF34Stages * kX;
    static constexpr uint32_t oA4 = oW3 + kF34Stages * kW3;
    static constexpr uint32_t oW4 = oA4 + kF34A4Stages * kA4;
    static constexpr uint32_t oBars = oW4 + kK4 * kW4;
    static constexpr int kNumBars = 2 * kF34Stages + 2 * kF34A4Stages + 1 + 2 + 2 + 2 + 2 + 2;
    static constexpr uint32_t kTotal = 1024 + oBars + kNumBars * 8 + 16;
    static_assert(kW3 % 1024 == 0, "1024-byte aligned stages");
    static_assert(kTotal <= 232448, "shared memory per CTA");
};

struct F34Args {
    int M, K3, N3, N4;   // rows, layer-3 K, layer-3 outputs (NA + NB), output-layer outputs (<= 32)
    const float *b3;     // [N3 rounded up to 16] (16-byte aligned)
    const float *b4;     // [N4]
    float *u;            // [M][ldu] FP32
    int64_t ldu;
    uint32_t spin;
};

template <int NA, int NB>
__global__ void __launch_bounds__(kF34Threads, 1)
    gemm_fused34_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW3a,
                        const __grid_constant__ CUtensorMap tmW3b, const __grid_constant__ CUtensorMap tmW4, F34Args a,
                        int *err) {
    using L = F34Smem<NA, NB>;
    constexpr int K4 = L::kK4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sX = smem + L::oX;
    uint8_t *sW3 = smem + L::oW3;
    uint8_t *sA4 = smem + L::oA4;
    uint8_t *sW4 = smem + L::oW4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::oBars);
    uint64_t *full = bars, *empty = bars + kF34Stages;
    uint64_t *a4_full = empty + kF34Stages, *a4_empty = a4_full + kF34A4Stages;
    uint64_t *w4_full = a4_empty + kF34A4Stages;
    uint64_t *d3_full = w4_full + 1, *d3_empty = d3_full + 2;       // [half]
    uint64_t *d4_full = d3_empty + 2, *d4_empty = d4_full + 2;      // [buffer]
    uint64_t *drain = d4_empty + 2;                                  // [MMA thread]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tiles = (a.M + kBM - 1) / kBM;
    const int kb3 = (a.K3 + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kF34Stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        for (int s = 0; s < kF34A4Stages; ++s) {
            tc::mbar_init(&a4_full[s], kEpiWarps);
            tc::mbar_init(&a4_empty[s], 1);
        }
        tc::mbar_init(w4_full, 1);
        for (int h = 0; h < 2; ++h) {
            tc::mbar_init(&d3_full[h], 1);
            tc::mbar_init(&d3_empty[h], kEpiWarps);
            tc::mbar_init(&d4_full[h], 1);
            tc::mbar_init(&d4_empty[h], kEpiWarps);
            tc::mbar_init(&drain[h], 1);
        }
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
            tc::tma_prefetch_desc(&tmW3a);
            tc::tma_prefetch_desc(&tmW3b);
            tc::tma_prefetch_desc(&tmW4);
            // W4, resident for the whole launch: K4 boxes of 32 rows x 64 columns
            tc::mbar_arrive_expect_tx(w4_full, K4 * L::kW4);
            for (int j = 0; j < K4; ++j) tc::tma_load_2d(sW4 + j * L::kW4, &tmW4, w4_full, j * 64, 0);
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x) {
                for (int h = 0; h < 2 && ok; ++h) {
                    const uint32_t wbytes = (h == 0 ? NA : NB) * 128;
                    for (int kb = 0; kb < kb3; ++kb, ++it) {
                        const int s = it % kF34Stages;
                        if (!tc::mbar_wait(&empty[s], (uint32_t)((it / kF34Stages) & 1) ^ 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutEmpty);
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&full[s], L::kX + wbytes);
                        tc::tma_load_2d(sX + s * L::kX, &tmX, &full[s], kb * kBK, tile * kBM);
                        if (h == 0) tc::tma_load_2d(sW3 + s * L::kW3, &tmW3a, &full[s], kb * kBK, 0);
                        else tc::tma_load_2d(sW3 + s * L::kW3, &tmW3b, &full[s], kb * kBK, NA);
                    }
                }
            }
            // every issued load lands before the CTA may exit (full limit)
            for (int j = (it > kF34Stages ? it - kF34Stages : 0); j < it; ++j)
                if (!tc::mbar_wait(&full[j % kF34Stages], (uint32_t)(j / kF34Stages) & 1u)) {
                    atomicExch(err, tc::kErrTimeoutDrain);
                    break;
                }
            if (!tc::mbar_wait(w4_full, 0)) atomicExch(err, tc::kErrTimeoutDrain);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idA = tc::idesc_bf16_f32(kBM, NA);
            constexpr uint32_t idB = tc::idesc_bf16_f32(kBM, NB);
            int it = 0, t = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x, ++t) {
                for (int h = 0; h < 2 && ok; ++h) {
                    // the half's accumulator has been read by the epilogue of the previous tile
                    if (!tc::mbar_wait(&d3_empty[h], (uint32_t)(t & 1) ^ 1u, a.spin)) {
                        atomicExch(err, tc::kErrTimeoutTmemEmpty);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d = tmem + (h == 0 ? 0u : (uint32_t)NA);
                    for (int kb = 0; kb < kb3; ++kb, ++it) {
                        const int s = it % kF34Stages;
                        if (!tc::mbar_wait(&full[s], (uint32_t)(it / kF34Stages) & 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutFull);
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t xa = tc::smem_u32(sX + s * L::kX), wb = tc::smem_u32(sW3 + s * L::kW3);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = tc::sdesc_kmajor_sw128(xa + kk * 32);
                            const uint64_t bd = tc::sdesc_kmajor_sw128(wb + kk * 32);
                            tc::umma_f16(d, ad, bd, h == 0 ? idA : idB, (kb > 0 || kk > 0) ? 1u : 0u);
                        }
                        tc::umma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    tc::umma_commit(&d3_full[h]);
                }
            }
            tc::umma_commit(&drain[0]);
            if (!tc::mbar_wait(&drain[0], 0)) atomicExch(err, tc::kErrTimeoutDrain);
        }
    } else if (warp == 2) {
        if (lane == 0) {
            constexpr uint32_t id4 = tc::idesc_bf16_f32(kBM, 32);
            int j4 = 0, t = 0;
            bool ok = tc::mbar_wait(w4_full, 0, a.spin);
            if (!ok) atomicExch(err, tc::kErrTimeoutFull);
            for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x, ++t) {
                const int buf = t & 1;
                if (!tc::mbar_wait(&d4_empty[buf], (uint32_t)((t >> 1) & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutTmemEmpty);
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d = tmem + kF34D4Col + (uint32_t)buf * 32u;
                for (int j = 0; j < K4; ++j, ++j4) {
                    const int s = j4 % kF34A4Stages;
                    if (!tc::mbar_wait(&a4_full[s], (uint32_t)(j4 / kF34A4Stages) & 1u, a.spin)) {
                        atomicExch(err, tc::kErrTimeoutFull);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t aa = tc::smem_u32(sA4 + s * L::kA4), wb = tc::smem_u32(sW4 + j * L::kW4);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::umma_f16(d, tc::sdesc_kmajor_sw128(aa + kk * 32), tc::sdesc_kmajor_sw128(wb + kk * 32), id4,
                                     (j > 0 || kk > 0) ? 1u : 0u);
                    tc::umma_commit(&a4_empty[s]);
                }
                if (!ok) break;
                tc::umma_commit(&d4_full[buf]);
            }
            tc::umma_commit(&drain[1]);
            if (!tc::mbar_wait(&drain[1], 0)) atomicExch(err, tc::kErrTimeoutDrain);
        }
    } else {
        const int quad = warp & 3;
        const int group = (warp - 3) >> 2;          // 0..3
        const int r = quad * 32 + lane;             // this thread's row of the tile
        const uint32_t tq = (uint32_t)(quad * 32) << 16;
        int j4 = 0, t = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < m_tiles && ok; tile += gridDim.x, ++t) {
            // the two halves of h3: k-blocks of 64 columns, this warp's 16 of each
            for (int h = 0; h < 2 && ok; ++h) {
                if (!__all_sync(0xffffffffu, tc::mbar_wait(&d3_full[h], (uint32_t)(t & 1), a.spin))) {
                    if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const int c_lo = h == 0 ? 0 : NA, width = h == 0 ? NA : NB;
                const int nblk = (width + 63) / 64;
                for (int i = 0; i < nblk; ++i, ++j4) {
                    const int col = c_lo + 64 * i + 16 * group;          // h3 column of this warp's slice
                    uint32_t w[8];
                    if (col < c_lo + width) {
                        float v[16];
                        tc::tmem_ld16(tmem + tq + (uint32_t)col, v);
                        float b[16];
                        const float4 *bp = reinterpret_cast<const float4 *>(a.b3 + col);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 x = __ldg(bp + q);
                            b[4 * q] = x.x; b[4 * q + 1] = x.y; b[4 * q + 2] = x.z; b[4 * q + 3] = x.w;
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float g0, g1;
                            gelu_pair(v[2 * q], v[2 * q + 1], b[2 * q], b[2 * q + 1], g0, g1);
                            __nv_bfloat162 hb = __floats2bfloat162_rn(g0, g1);
                            w[q] = *reinterpret_cast<uint32_t *>(&hb);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) w[q] = 0u;            // columns past N3: zero K for layer 4
                    }
                    const int s = j4 % kF34A4Stages;
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(&a4_empty[s],
                                                               (uint32_t)((j4 / kF34A4Stages) & 1) ^ 1u, a.spin))) {
                        if (lane == 0) atomicExch(err, tc::kErrTimeoutEmpty);
                        ok = false;
                        break;
                    }
                    uint8_t *rowp = sA4 + s * L::kA4 + r * 128;
                    const int c0 = 2 * group;                            // 16-byte chunks of the k-block row
                    *reinterpret_cast<uint4 *>(rowp + ((c0 ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(rowp + (((c0 + 1) ^ (r & 7)) << 4)) =
                        make_uint4(w[4], w[5], w[6], w[7]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&a4_full[s]);
                }
                if (!ok) break;
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&d3_empty[h]);
            }
            if (!ok) break;
            // the output layer: u = D4 + b4 for this tile's rows (warps of groups 0 and 1)
            const int buf = t & 1;
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&d4_full[buf], (uint32_t)((t >> 1) & 1), a.spin))) {
                if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                ok = false;
                break;
            }
            tc::tc_fence_after();
            if (group < 2) {
                float v[16];
                tc::tmem_ld16(tmem + tq + kF34D4Col + (uint32_t)buf * 32u + (uint32_t)(group * 16), v);
                const int row = tile * kBM + r;
                if (row < a.M) {
                    float *o = a.u + (int64_t)row * a.ldu + group * 16;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (group * 16 + q < a.N4) o[q] = v[q] + __ldg(a.b4 + group * 16 + q);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d4_empty[buf]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace chemgb
