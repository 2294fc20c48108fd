// gemm_launch.cuh -- host-side launch of gemm_tn_kernel: TMA descriptors,
// tile-width dispatch and the persistent grid. Included by the translation
// units that instantiate the kernel for their epilogue.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <string>

#include "gemm.cuh"
#include "internal.cuh"

namespace chemgb {

// cuTensorMapEncodeTiled resolved through the runtime (no link-time libcuda dependency).
inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D operand tensor map over a row-major [rows][cols] matrix of BF16 (esize 2)
// or E4M3 (esize 1) with row stride ld (elements): box = box_rows x 128 bytes,
// 128-byte swizzle, zero fill outside.
inline int make_tmap_operand(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                             int esize) {
    if (!aligned16(ptr) || (ld * esize) % 16 != 0)
        return set_error(CHEM_EINVAL, "GEMM operand: base must be 16-byte aligned and rows a multiple of 16 bytes");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled_fn();
    if (!enc) return set_error(CHEM_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(CHEM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return CHEM_OK;
}

inline int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

// Output tensor map for the TMA-store epilogue: [rows][cols] of BF16 (esize 2)
// or E4M3 (esize 1), box 32 rows x 16 columns, no swizzle.
inline int make_tmap_out(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int esize) {
    if (!aligned16(ptr) || (ld * esize) % 16 != 0)
        return set_error(CHEM_EINVAL, "GEMM output: base must be 16-byte aligned and rows a multiple of 16 bytes");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {16, 32};
    cuuint32_t estr[2] = {1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled_fn();
    if (!enc) return set_error(CHEM_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(CHEM_ECUDA, "cuTensorMapEncodeTiled (output) failed (" + std::to_string((int)r) + ")");
    return CHEM_OK;
}

template <int BN, int STAGES, class Epi>
int launch_gemm_bn(const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K, const Epi &epi,
                   int *err, cudaStream_t st, int max_ctas) {
    using L = GemmSmem<BN, STAGES>;
    static bool configured = false;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(gemm_tn_kernel<BN, STAGES, Epi>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kTotal),
                            "GEMM smem attribute");
        if (rc) return rc;
        configured = true;
    }
    CUtensorMap ta, tb;
    const int esize = Epi::kF8 ? 1 : 2;
    int rc = make_tmap_operand(&ta, X, M, K, ldx, kBM, esize);
    if (rc) return rc;
    rc = make_tmap_operand(&tb, W, N, K, ldw, BN, esize);
    if (rc) return rc;
    CUtensorMap tc;
    std::memset(&tc, 0, sizeof(tc));
    if (const void *op = epi.tma_ptr()) {
        rc = make_tmap_out(&tc, op, M, N, epi.ldo, Epi::kOutBytes / 16);
        if (rc) return rc;
    }
    const int tiles = ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
    int grid = num_sms();
    if (max_ctas > 0 && max_ctas < grid) grid = max_ctas;
    if (tiles < grid) grid = tiles;
    void *pb = prof_begin(st);
    gemm_tn_kernel<BN, STAGES, Epi><<<grid, kGemmThreads, L::kTotal, st>>>(ta, tb, tc, M, N, K, epi, err);
    if (pb)
        prof_end(pb, st, "gemm_tn_kernel<" + std::to_string(BN) + (Epi::kF8 ? ",e4m3> " : "> ") + std::to_string(N) +
                             "x" + std::to_string(K),
                 2.0 * M * N * K, (double)esize * ((double)M * K + (double)N * K));
    return check_cuda(cudaGetLastError(), "GEMM launch");
}

// Two-CTA variant (clusters of two, M = 256 per MMA); grid = 2 x pairs.
template <int BN, int STAGES, class Epi>
int launch_gemm_pair_bn(const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K, const Epi &epi,
                        int *err, cudaStream_t st, int max_ctas) {
    using L = GemmPairSmem<BN, STAGES>;
    static bool configured = false;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(gemm_tn_pair_kernel<BN, STAGES, Epi>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kTotal),
                            "GEMM (pair) smem attribute");
        if (rc) return rc;
        configured = true;
    }
    CUtensorMap ta, tb;
    const int esize = Epi::kF8 ? 1 : 2;
    int rc = make_tmap_operand(&ta, X, M, K, ldx, kBM, esize);
    if (rc) return rc;
    rc = make_tmap_operand(&tb, W, N, K, ldw, BN / 2, esize);
    if (rc) return rc;
    CUtensorMap tc;
    std::memset(&tc, 0, sizeof(tc));
    if (const void *op = epi.tma_ptr()) {
        rc = make_tmap_out(&tc, op, M, N, epi.ldo, Epi::kOutBytes / 16);
        if (rc) return rc;
    }
    const int tiles = ((M + 2 * kBM - 1) / (2 * kBM)) * ((N + BN - 1) / BN);
    int pairs = num_sms() / 2;
    if (max_ctas > 0 && max_ctas / 2 < pairs) pairs = max_ctas / 2 > 0 ? max_ctas / 2 : 1;
    if (tiles < pairs) pairs = tiles;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(kGemmThreads, 1, 1);
    cfg.dynamicSmemBytes = L::kTotal;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *pb = prof_begin(st);
    rc = check_cuda(cudaLaunchKernelEx(&cfg, gemm_tn_pair_kernel<BN, STAGES, Epi>, ta, tb, tc, M, N, K, epi, err),
                    "GEMM (pair) launch");
    if (pb)
        prof_end(pb, st, "gemm_tn_pair_kernel<" + std::to_string(BN) + (Epi::kF8 ? ",e4m3> " : "> ") +
                             std::to_string(N) + "x" + std::to_string(K),
                 2.0 * M * N * K, (double)esize * ((double)M * K + (double)N * K));
    return rc;
}

// Tile widths the library is built with (the autotuner picks among them). A tile code is the
// width, plus kPairTile for the two-CTA variant (widths 128, 160, 208, 256).
constexpr int kTileWidths[] = {32, 64, 128, 160, 208, 256};
constexpr int kPairTile = 0x10000;
constexpr int kPairWidths[] = {128, 160, 208, 256};

template <class Epi>
int launch_gemm(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                const Epi &epi, int *err, cudaStream_t st, int max_ctas = 0) {
    if (M <= 0 || N <= 0 || K <= 0) return CHEM_OK;
    if (bn & kPairTile) {
        switch (bn & 0xFFFF) {
            case 128: return launch_gemm_pair_bn<128, 8>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
            case 160: return launch_gemm_pair_bn<160, 7>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
            case 208: return launch_gemm_pair_bn<208, 6>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
            case 256: return launch_gemm_pair_bn<256, 6>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
            default: return set_error(CHEM_EINVAL, "GEMM: unsupported pair tile width " + std::to_string(bn & 0xFFFF));
        }
    }
    switch (bn) {
        case 32: return launch_gemm_bn<32, 8>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        case 64: return launch_gemm_bn<64, 8>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        case 128: return launch_gemm_bn<128, 6>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        case 160: return launch_gemm_bn<160, 5>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        case 208: return launch_gemm_bn<208, 4>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        case 256: return launch_gemm_bn<256, 4>(X, ldx, W, ldw, M, N, K, epi, err, st, max_ctas);
        default: return set_error(CHEM_EINVAL, "GEMM: unsupported tile width " + std::to_string(bn));
    }
}

// Default tile width for an output width N (fewest padded columns, then widest tile).
inline int default_tile_width(int N) {
    int best = 256;
    long best_pad = -1;
    for (int bn : kTileWidths) {
        if (bn < 64 && N > 64) continue;
        long pad = (long)((N + bn - 1) / bn) * bn - N;
        if (best_pad < 0 || pad < best_pad || (pad == best_pad && bn > best)) { best = bn; best_pad = pad; }
    }
    return best;
}

// Forward declarations of the per-epilogue launchers (one translation unit each).
int gemm_gelu(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K, const float *bias,
              void *out, int64_t ldo, float *pre, int64_t ldp, int *err, cudaStream_t st, int max_ctas = 0);
int gemm_linear(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                const float *bias, float *out, int64_t ldo, int *err, cudaStream_t st, int max_ctas = 0);
int gemm_gelu_grad(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *z, int64_t ldz, void *out, int64_t ldo, int *err, cudaStream_t st, int max_ctas = 0);
// Reduced-precision hidden layer (EpiGeluQ): f8in selects E4M3 operands (X, W) with the per-column
// scale cs, f8out an E4M3 output scaled by inv_so; otherwise BF16.
int gemm_gelu_q(bool f8in, bool f8out, int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N,
                int K, const float *bias, const float *cs, void *out, int64_t ldo, float inv_so, int *err,
                cudaStream_t st, int max_ctas = 0);

}  // namespace chemgb
