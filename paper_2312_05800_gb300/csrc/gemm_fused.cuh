// gemm_fused.cuh -- the network's first two layers in one persistent launch of
// CTA pairs: h2 = GELU(GELU(X W1^T + b1) W2^T + b2) (Sec. 3.2: the hidden
// layers of 1600 and 800 GELU units), with the first hidden layer h1 made on
// chip, shared between the two CTAs of a cluster and never written to memory.
//
// Both CTAs of a cluster take the same 128-row tile of X (the prologue's hi|lo
// BF16 rows, one 128-byte k-block). CTA `rank` owns layer 2's output columns
// (2p + rank) NP .. + NP - 1 of pass p (one pass when h2 <= 2 NP). The 64-column
// chunks of h1 are made alternately by the two CTAs: chunk q (counted over the
// CTA's whole sequence of tiles, passes and chunks, the same in both CTAs) is
// made by CTA q % 2, which
//   MMA1   D1 = X W1[64c .. 64c + 63]^T             (TMEM, 64 columns)
//   GELU   A2 = bf16(GELU(D1 + b1)), written by its epilogue warps in the 128-
//          byte-swizzled K-major layout a TMA load would produce, into its A2
//          stage q % 2, then sent whole (16 KB) into the same stage of the peer
//          by one bulk copy through distributed shared memory, which completes
//          on the peer's mbarrier (the async proxy end to end: no fences or
//          releases on the epilogue's path)
// and both CTAs then accumulate
//   MMA2   D2 += A2 W2[own rows][64c .. 64c + 63]^T (TMEM, NP columns)
// before h2 = bf16(GELU(D2 + b2)) goes out by TMA stores. Each h1 element is
// computed once per row tile, half of the chunks on each SM, instead of once
// per pass of a single CTA whose D2 cannot hold all 800 columns in TMEM.
// Every element's FP32 sums take the same k order as the two-launch path
// (gemm_tn_kernel), so the results are bitwise those of layer 1 then layer 2.
// Measured on GB300 the exchange bounds it: a 16 KB copy between the SMs of a
// pair takes about 1 us to land, and with one A2 stage per maker each own chunk
// waits for the previous one's round trip (write, copy, both MMAs), about one
// chunk per microsecond against 0.5 us of tensor work; at 1600/800 units it is
// about 7 % slower than the two tuned launches, and chem_mlp_autotune keeps
// whichever is faster. (Deeper rings do not fit beside the 51 KB W2 stages in
// 227 KB of shared memory.)
//
// Roles (640 threads, one CTA per SM, clusters of two):
//   warp 0      TMA producer of X tiles (2-stage ring) and of W1 for its own chunks (3-stage ring)
//   warp 1      TMEM allocation; one thread issues every tcgen05.mma
//   warp 2      TMA producer of W2 chunks (2-stage ring, two boxes of NP/2 rows)
//   warp 3      one thread sends each own chunk to the peer as soon as the epilogue has written it
//               (apart from the MMA thread, which takes the chunks in order and would hold a send
//               back behind the wait for the peer's previous chunk)
//   warps 4-19  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows);
//               for h1 each takes 16 of its chunks' 64 columns, for h2 the
//               16-column slices of the pass in turn.
// Hand-offs: A2 stage r is always written by CTA r. It is full for CTA r when
// its 16 epilogue warps have arrived (a2_ready) and for the peer when the bulk
// copy's bytes have landed (a2_full, armed by the peer's MMA thread with
// expect_tx); it is empty again when the layer-2 MMAs of both CTAs that read
// it have completed (each commits to a2_empty of CTA r, the peer's by a
// multicast tcgen05.commit). Every wait is bounded (a.spin tries); one that
// runs out records its code and the kernel unwinds as gemm_tn_kernel does;
// both CTAs meet at a cluster barrier before either leaves, so no CTA exits
// while a copy or a commit of its peer may still reach its shared memory.
#pragma once

#include "gemm.cuh"

namespace chemgb {

constexpr int kF12Chunk = 64;             // h1 columns per chunk = layer-2 K per k-block
constexpr int kF12XStages = 2;
constexpr int kF12W1Stages = 3;
constexpr int kF12W2Stages = 2;
constexpr int kF12EpiWarps = 16;
constexpr int kF12Threads = 128 + 32 * kF12EpiWarps;
constexpr uint32_t kF12D1Col = 448;       // TMEM columns of D1 (D2: 0 .. NP - 1, NP <= 448)

template <int NP>
struct F12Smem {
    static_assert(NP % 16 == 0 && NP >= 32 && NP <= 448, "pass width: UMMA N pieces of <= 256, D1 after D2");
    static constexpr uint32_t kX = kBM * 128;                 // 128 rows x 128 bytes
    static constexpr uint32_t kW1 = kF12Chunk * 128;          // 64 rows x 128 bytes
    static constexpr uint32_t kW2 = NP * 128;                 // NP rows x 128 bytes
    static constexpr uint32_t kA2 = kBM * 128;
    static constexpr uint32_t kStaging = kF12EpiWarps * 2 * kStageBytesPerWarp;
    static constexpr uint32_t oX = 0;
    static constexpr uint32_t oW1 = oX + kF12XStages * kX;
    static constexpr uint32_t oW2 = oW1 + kF12W1Stages * kW1;
    static constexpr uint32_t oA2 = oW2 + kF12W2Stages * kW2;
    static constexpr uint32_t oStage = oA2 + 2 * kA2;
    static constexpr uint32_t oBars = oStage + kStaging;
    static constexpr int kNumBars = 2 * kF12XStages + 2 * kF12W1Stages + 2 * kF12W2Stages + 2 + 6 + 2 + 1;
    static constexpr uint32_t kTotal = 1024 + oBars + kNumBars * 8 + 16;
    static_assert(kW2 % 1024 == 0 && (NP / 2) % 8 == 0, "W2 boxes keep 1024-byte alignment");
    static_assert(kTotal <= 232448, "shared memory per CTA");
};

struct F12Args {
    int M;               // rows
    int N1;              // layer-1 outputs (a multiple of 64)
    int N2;              // layer-2 outputs
    int passes;          // ceil(N2 / (2 NP))
    const float *b1;     // [N1], 16-byte aligned
    const float *b2;     // [N2], 16-byte aligned
    uint32_t spin;       // tries of a pipeline wait
};

template <int NP>
__global__ void __launch_bounds__(kF12Threads, 1)
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
    uint64_t *a2_ready = d1_empty + 1, *a2_full = a2_ready + 2, *a2_empty = a2_full + 2;
    uint64_t *d2_full = a2_empty + 2, *d2_empty = d2_full + 1;
    uint64_t *drain = d2_empty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    uint32_t *peer_sent = tmem_slot + 1;      // written by the peer at the end: the copies it sent here

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)tc::cluster_ctarank();
    const int peer = rank ^ 1;
    const int m_tiles = (a.M + kBM - 1) / kBM;
    const int chunks = a.N1 / kF12Chunk;
    const int cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
    int mma_nr = 0, mma_na = 0;                // the MMA thread's count of the peer's chunks landed / armed

    if (threadIdx.x == 0) {
        for (int s = 0; s < kF12XStages; ++s) { tc::mbar_init(&x_full[s], 1); tc::mbar_init(&x_empty[s], 1); }
        for (int s = 0; s < kF12W1Stages; ++s) { tc::mbar_init(&w1_full[s], 1); tc::mbar_init(&w1_empty[s], 1); }
        for (int s = 0; s < kF12W2Stages; ++s) { tc::mbar_init(&w2_full[s], 1); tc::mbar_init(&w2_empty[s], 1); }
        tc::mbar_init(d1_full, 1);
        tc::mbar_init(d1_empty, kF12EpiWarps);
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&a2_ready[s], kF12EpiWarps);       // this CTA's epilogue wrote its stage
            tc::mbar_init(&a2_full[s], 1);                   // armed by the MMA thread; the peer's copy's bytes
            tc::mbar_init(&a2_empty[s], 2);                  // the layer-2 MMAs of both CTAs
        }
        tc::mbar_init(d2_full, 1);
        tc::mbar_init(d2_empty, kF12EpiWarps);
        tc::mbar_init(drain, 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncwarp();
    tc::cluster_sync();                 // both CTAs' barriers exist before any copy or commit reaches them
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmX);
            tc::tma_prefetch_desc(&tmW1);
            int xi = 0, w1i = 0, q = 0;
            bool ok = true;
            for (int tile = cluster; tile < m_tiles && ok; tile += nclusters, ++xi) {
                const int sx = xi % kF12XStages;
                if (!tc::mbar_wait(&x_empty[sx], (uint32_t)((xi / kF12XStages) & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutEmpty);
                    ok = false;
                    break;
                }
                tc::mbar_arrive_expect_tx(&x_full[sx], L::kX);
                tc::tma_load_2d(sX + sx * L::kX, &tmX, &x_full[sx], 0, tile * kBM);
                for (int p = 0; p < a.passes && ok; ++p)
                    for (int c = 0; c < chunks; ++c, ++q) {
                        if ((q & 1) != rank) continue;           // the peer makes this chunk
                        const int s1 = w1i % kF12W1Stages;
                        if (!tc::mbar_wait(&w1_empty[s1], (uint32_t)((w1i / kF12W1Stages) & 1) ^ 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutEmpty);
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&w1_full[s1], L::kW1);
                        tc::tma_load_2d(sW1 + s1 * L::kW1, &tmW1, &w1_full[s1], 0, c * kF12Chunk);
                        ++w1i;
                    }
            }
            // every issued load lands before the CTA may exit (full limit): the last load into each
            // stage of each ring (xi and w1i count the loads issued)
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
        }
    } else if (warp == 2) {
        if (lane == 0) {
            tc::tma_prefetch_desc(&tmW2);
            int w2i = 0;
            bool ok = true;
            for (int tile = cluster; tile < m_tiles && ok; tile += nclusters)
                for (int p = 0; p < a.passes && ok; ++p) {
                    const int row0 = (2 * p + rank) * NP;
                    for (int c = 0; c < chunks; ++c, ++w2i) {
                        const int s2 = w2i % kF12W2Stages;
                        if (!tc::mbar_wait(&w2_empty[s2], (uint32_t)((w2i / kF12W2Stages) & 1) ^ 1u, a.spin)) {
                            atomicExch(err, tc::kErrTimeoutEmpty);
                            ok = false;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&w2_full[s2], L::kW2);
                        uint8_t *dst = sW2 + s2 * L::kW2;
                        tc::tma_load_2d(dst, &tmW2, &w2_full[s2], c * kF12Chunk, row0);
                        tc::tma_load_2d(dst + (NP / 2) * 128, &tmW2, &w2_full[s2], c * kF12Chunk, row0 + NP / 2);
                    }
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
            // nl: own chunks consumed; na / nr: the peer's chunks armed (expect_tx) / landed
            int xi = 0, w1i = 0, w2i = 0, n1 = 0, nl = 0, na = 0, nr = 0, pi = 0, q = 0;
            bool ok = true;
            // MMA1 of this CTA's n1-th chunk, h1 columns 64 c ..: D1 = X W1_c^T (one k-block, four K = 16 steps)
            auto mma1 = [&]() -> bool {
                const int s1 = w1i % kF12W1Stages;
                if (!tc::mbar_wait(&w1_full[s1], (uint32_t)(w1i / kF12W1Stages) & 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    return false;
                }
                if (!tc::mbar_wait(d1_empty, (uint32_t)(n1 & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutTmemEmpty);
                    return false;
                }
                tc::tc_fence_after();
                const uint32_t xa = tc::smem_u32(sX + (xi % kF12XStages) * L::kX), wb = tc::smem_u32(sW1 + s1 * L::kW1);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::umma_f16(tmem + kF12D1Col, tc::sdesc_kmajor_sw128(xa + kk * 32),
                                 tc::sdesc_kmajor_sw128(wb + kk * 32), idesc1, kk > 0 ? 1u : 0u);
                tc::umma_commit(&w1_empty[s1]);
                tc::umma_commit(d1_full);
                ++w1i;
                ++n1;
                return true;
            };
            // MMA2 of chunk c (global chunk q) of a pass: D2 (+)= A2[q % 2] W2_c^T
            auto mma2 = [&](int c) -> bool {
                const int s2 = w2i % kF12W2Stages, g = q & 1;
                if (c == 0 && !tc::mbar_wait(d2_empty, (uint32_t)(pi & 1) ^ 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutTmemEmpty);
                    return false;
                }
                if (g == rank) {
                    // this CTA's chunk: its epilogue wrote stage `rank`
                    if (!tc::mbar_wait(&a2_ready[g], (uint32_t)(nl & 1), a.spin)) {
                        atomicExch(err, tc::kErrTimeoutFull);
                        return false;
                    }
                    ++nl;
                } else {
                    // the peer's chunk: its copy's bytes complete this phase
                    if (na == nr) {
                        tc::mbar_arrive_expect_tx(&a2_full[g], L::kA2);
                        ++na;
                    }
                    if (!tc::mbar_wait_cluster(&a2_full[g], (uint32_t)(nr & 1), a.spin)) {
                        atomicExch(err, tc::kErrTimeoutFull);
                        return false;
                    }
                    ++nr;
                }
                if (!tc::mbar_wait(&w2_full[s2], (uint32_t)(w2i / kF12W2Stages) & 1u, a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    return false;
                }
                tc::tc_fence_after();
                const uint32_t aa = tc::smem_u32(sA2 + g * L::kA2), wb = tc::smem_u32(sW2 + s2 * L::kW2);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = tc::sdesc_kmajor_sw128(aa + kk * 32);
                    const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                    tc::umma_f16(tmem, ad, tc::sdesc_kmajor_sw128(wb + kk * 32), idescA, acc);
                    if (kNB > 0)
                        tc::umma_f16(tmem + kNA, ad, tc::sdesc_kmajor_sw128(wb + kNA * 128 + kk * 32), idescB, acc);
                }
                tc::umma_commit(&w2_empty[s2]);
                tc::umma_commit_multicast(&a2_empty[g], (uint16_t)(1u << g));   // stage g's maker
                ++w2i;
                ++q;
                return true;
            };
            for (int tile = cluster; tile < m_tiles && ok; tile += nclusters, ++xi) {
                if (!tc::mbar_wait(&x_full[xi % kF12XStages], (uint32_t)((xi / kF12XStages) & 1), a.spin)) {
                    atomicExch(err, tc::kErrTimeoutFull);
                    break;
                }
                for (int p = 0; p < a.passes && ok; ++p, ++pi) {
                    // this CTA's chunks of the pass are c0, c0 + 2, ...; MMA1 runs one own chunk ahead
                    const int c0 = ((q & 1) == rank) ? 0 : 1;
                    if (c0 < chunks && !mma1()) { ok = false; break; }
                    for (int c = 0; c < chunks; ++c) {
                        if (((q & 1) == rank) && c + 2 < chunks && !mma1()) { ok = false; break; }
                        if (!mma2(c)) { ok = false; break; }
                    }
                    if (!ok) break;
                    tc::umma_commit(d2_full);
                }
                if (!ok) break;
                tc::umma_commit(&x_empty[xi % kF12XStages]);     // the tile's MMA1s are done with X
            }
            // every MMA issued by this thread completes before TMEM is released (full limit)
            tc::umma_commit(drain);
            if (!tc::mbar_wait(drain, 0)) atomicExch(err, tc::kErrTimeoutDrain);
            mma_nr = nr;
            mma_na = na;
        }
    } else if (warp == 3) {
        if (lane == 0) {
            // each own chunk, in order, once the 16 epilogue warps have written it: stage `rank` to
            // the same stage of the peer, completing on the peer's a2_full[rank]
            const uint32_t peer_a2 = tc::mapa(sA2, (uint32_t)peer) + (uint32_t)(rank * L::kA2);
            const uint32_t peer_full = tc::mapa(&a2_full[rank], (uint32_t)peer);
            int q = 0, sent = 0;
            bool ok = true;
            for (int tile = cluster; tile < m_tiles && ok; tile += nclusters)
                for (int p = 0; p < a.passes && ok; ++p)
                    for (int c = 0; c < chunks; ++c, ++q) {
                        if ((q & 1) != rank) continue;
                        if (!tc::mbar_wait(&a2_ready[rank], (uint32_t)(sent & 1), a.spin)) {
                            atomicExch(err, tc::kErrTimeoutFull);
                            ok = false;
                            break;
                        }
                        tc::bulk_copy_to_peer(peer_a2, sA2 + rank * L::kA2, L::kA2, peer_full);
                        ++sent;
                    }
            // tell the peer how many chunks this CTA sent it (read after the first cluster barrier)
            tc::st_cluster_u32(tc::mapa(peer_sent, (uint32_t)peer), (uint32_t)sent);
        }
    } else {
        const int e = warp - 4;                     // 0..15
        const int quad = warp & 3;                  // TMEM lane quadrant = rows 32 quad .. + 31 of the tile
        const int grp = e >> 2;                     // h1: columns 16 grp .. + 15 of a chunk; h2: first slice
        const int r = quad * 32 + lane;             // this thread's row of the tile
        uint8_t *my_stage = staging + (size_t)e * 2 * kStageBytesPerWarp;
        // A2 row r, 16-byte units 2 grp and 2 grp + 1 of the 128-byte k-block, at the 128-byte
        // swizzle positions unit ^ (r % 8)
        const uint32_t off0 = (uint32_t)(r * 128 + (((2 * grp) ^ (r & 7)) << 4));
        const uint32_t off1 = (uint32_t)(r * 128 + (((2 * grp + 1) ^ (r & 7)) << 4));
        uint8_t *my_a2 = sA2 + rank * L::kA2;
        int nstore = 0, q = 0, nl = 0, pi = 0;
        bool ok = true;
        if (lane == 0) tc::tma_prefetch_desc(&tmH2);
        const uint32_t tq = (uint32_t)(quad * 32) << 16;
        for (int tile = cluster; tile < m_tiles && ok; tile += nclusters) {
            const int row0 = tile * kBM + quad * 32;
            for (int p = 0; p < a.passes && ok; ++p, ++pi) {
                for (int c = 0; c < chunks; ++c, ++q) {
                    if ((q & 1) != rank) continue;           // the peer makes this chunk
                    float b[16];
                    {
                        const float4 *bp = reinterpret_cast<const float4 *>(a.b1 + c * kF12Chunk + grp * 16);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 v = __ldg(bp + i);
                            b[4 * i] = v.x; b[4 * i + 1] = v.y; b[4 * i + 2] = v.z; b[4 * i + 3] = v.w;
                        }
                    }
                    const uint32_t par = (uint32_t)(nl & 1);
                    if (!__all_sync(0xffffffffu, tc::mbar_wait(d1_full, par, a.spin))) {
                        if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    float v[16];
                    tc::tmem_ld16(tmem + tq + kF12D1Col + (uint32_t)(grp * 16), v);
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(d1_empty);
                    uint32_t w[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float g0, g1;
                        gelu_pair(v[2 * i], v[2 * i + 1], b[2 * i], b[2 * i + 1], g0, g1);
                        __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
                        w[i] = *reinterpret_cast<uint32_t *>(&h);
                    }
                    // both CTAs' layer-2 MMAs are done with this CTA's stage (its previous chunk)
                    if (!__all_sync(0xffffffffu, tc::mbar_wait_cluster(&a2_empty[rank], par ^ 1u, a.spin))) {
                        if (lane == 0) atomicExch(err, tc::kErrTimeoutEmpty);
                        ok = false;
                        break;
                    }
                    *reinterpret_cast<uint4 *>(my_a2 + off0) = make_uint4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<uint4 *>(my_a2 + off1) = make_uint4(w[4], w[5], w[6], w[7]);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&a2_ready[rank]);
                    ++nl;
                }
                if (!ok) break;
                // the pass's h2 columns (2p + rank) NP .. + NP - 1: GELU(D2 + b2), BF16, TMA stores
                if (!__all_sync(0xffffffffu, tc::mbar_wait(d2_full, (uint32_t)(pi & 1), a.spin))) {
                    if (lane == 0) atomicExch(err, tc::kErrTimeoutTmemFull);
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const int colp = (2 * p + rank) * NP;
#pragma unroll 1
                for (int j = grp; j < NP / 16; j += kF12EpiWarps / 4) {
                    const int col0 = colp + j * 16;
                    if (col0 >= a.N2) break;             // warp-uniform
                    float v[16];
                    tc::tmem_ld16(tmem + tq + (uint32_t)(j * 16), v);
                    if (row0 >= a.M) continue;           // warp-uniform: no row of this slice is in range
                    float b[16];
                    const float4 *bp = reinterpret_cast<const float4 *>(a.b2 + col0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 t4 = __ldg(bp + i);
                        b[4 * i] = t4.x; b[4 * i + 1] = t4.y; b[4 * i + 2] = t4.z; b[4 * i + 3] = t4.w;
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
    // neither CTA leaves while a copy or a commit of its peer may still reach its shared memory
    // (every wait above is bounded, so every thread of both CTAs gets here). After the first
    // cluster barrier each MMA thread knows how many chunks its peer sent; one that stopped early
    // (a wait that ran out) may have one copy still in flight, at most: the peer sends its next
    // chunk only after both CTAs' MMAs have read the previous one. It waits for that copy's bytes
    // (full limit) before the second barrier lets both CTAs leave.
    tc::tc_fence_before();
    __syncwarp();
    tc::cluster_sync();
    if (warp == 1 && lane == 0) {
        const int sent = (int)*peer_sent;
        uint64_t *full = &a2_full[peer];
        for (; mma_nr < sent; ++mma_nr) {
            if (mma_na == mma_nr) {
                tc::mbar_arrive_expect_tx(full, L::kA2);
                ++mma_na;
            }
            if (!tc::mbar_wait_cluster(full, (uint32_t)(mma_nr & 1))) {
                atomicExch(err, tc::kErrTimeoutDrain);
                break;
            }
        }
    }
    __syncwarp();
    tc::cluster_sync();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace chemgb
