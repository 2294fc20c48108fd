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

// A GEMM operand: row-major rows of K elements with row stride ld; for a grouped launch its
// map kind and the elements between consecutive groups (rows x ld for stacked rows, the column
// offset for side-by-side columns).
struct GemmOperand {
    const void *ptr;
    int64_t ld;
    int kind;
    int64_t gstride;
};

// 3-D operand map of one of the grouped kinds: box = box_rows x 128 bytes of one group.
// Stacked rows: dims (K, rows, G), strides (ld, gstride); side-by-side columns: dims
// (K, G, rows), strides (gstride, ld). Zero fill outside, so K and rows clip per group.
inline int make_tmap_operand_grouped(CUtensorMap *map, const GemmOperand &op, int64_t rows, int64_t cols, int G,
                                     int box_rows, int esize) {
    if (!aligned16(op.ptr) || (op.ld * esize) % 16 != 0 || (op.gstride * esize) % 16 != 0 || op.gstride <= 0)
        return set_error(CHEM_EINVAL, "grouped GEMM operand: base, row and group strides must be 16-byte multiples");
    const bool rowg = op.kind == kMapRowGrp;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)(rowg ? rows : G), (cuuint64_t)(rowg ? G : rows)};
    cuuint64_t strides[2] = {(cuuint64_t)((rowg ? op.ld : op.gstride) * esize),
                             (cuuint64_t)((rowg ? op.gstride : op.ld) * esize)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esize), (cuuint32_t)(rowg ? box_rows : 1), (cuuint32_t)(rowg ? 1 : box_rows)};
    cuuint32_t estr[3] = {1, 1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled_fn();
    if (!enc) return set_error(CHEM_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                     const_cast<void *>(op.ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(CHEM_ECUDA, "cuTensorMapEncodeTiled (grouped) failed (" + std::to_string((int)r) + ")");
    return CHEM_OK;
}

inline int make_operand_map(CUtensorMap *map, const GemmOperand &op, int64_t rows, int64_t cols, int G, int box_rows,
                            int esize) {
    if (op.kind == kMap2D) return make_tmap_operand(map, op.ptr, rows, cols, op.ld, box_rows, esize);
    return make_tmap_operand_grouped(map, op, rows, cols, G, box_rows, esize);
}

// Tries of each pipeline wait of the GEMMs launched by this host thread (tc::kSpinLimit unless a
// network handle with a smaller limit is launching; see WaitLimitScope).
inline uint32_t &gemm_wait_limit() {
    static thread_local uint32_t limit = tc::kSpinLimit;
    return limit;
}
// Sets this thread's GEMM wait limit for the lifetime of the object, then restores it.
struct WaitLimitScope {
    uint32_t saved;
    explicit WaitLimitScope(uint32_t limit) : saved(gemm_wait_limit()) { gemm_wait_limit() = limit; }
    ~WaitLimitScope() { gemm_wait_limit() = saved; }
    WaitLimitScope(const WaitLimitScope &) = delete;
    WaitLimitScope &operator=(const WaitLimitScope &) = delete;
};

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

// Output map of a grouped TMA-store epilogue: box 32 rows x 16 columns of one group.
inline int make_tmap_out_grouped(CUtensorMap *map, const void *ptr, int kind, int64_t rows, int64_t cols, int G,
                                 int64_t ld, int64_t gstride, int esize) {
    if (kind == kMap2D) return make_tmap_out(map, ptr, rows, cols, ld, esize);
    if (!aligned16(ptr) || (ld * esize) % 16 != 0 || (gstride * esize) % 16 != 0 || gstride <= 0)
        return set_error(CHEM_EINVAL, "grouped GEMM output: base, row and group strides must be 16-byte multiples");
    const bool rowg = kind == kMapRowGrp;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)(rowg ? rows : G), (cuuint64_t)(rowg ? G : rows)};
    cuuint64_t strides[2] = {(cuuint64_t)((rowg ? ld : gstride) * esize), (cuuint64_t)((rowg ? gstride : ld) * esize)};
    cuuint32_t box[3] = {16, (cuuint32_t)(rowg ? 32 : 1), (cuuint32_t)(rowg ? 1 : 32)};
    cuuint32_t estr[3] = {1, 1, 1};
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled_fn();
    if (!enc) return set_error(CHEM_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                     const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(CHEM_ECUDA, "cuTensorMapEncodeTiled (grouped output) failed (" + std::to_string((int)r) + ")");
    return CHEM_OK;
}

// G products of M x N x K in one persistent launch; out_kind / out_gstride describe the
// TMA-store output (used when the epilogue stores by TMA; element stores use the functor's
// own group offsets, which must agree).
template <int BN, int STAGES, class Epi>
int launch_gemm_grouped_bn(const GemmOperand &A, const GemmOperand &B, int G, int out_kind, int64_t out_gstride, int M,
                           int N, int K, const Epi &epi, int *err, cudaStream_t st, int max_ctas) {
    using L = GemmSmem<BN, STAGES>;
    static bool configured = false;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(gemm_tn_kernel<BN, STAGES, Epi>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kTotal),
                            "GEMM smem attribute");
        if (rc) return rc;
        configured = true;
    }
    const int esize = Epi::kF8 ? 1 : 2;
    CUtensorMap ta, tb, tc;
    int rc = make_operand_map(&ta, A, M, K, G, kBM, esize);
    if (rc) return rc;
    rc = make_operand_map(&tb, B, N, K, G, BN, esize);
    if (rc) return rc;
    std::memset(&tc, 0, sizeof(tc));
    if (const void *op = epi.tma_ptr()) {
        rc = make_tmap_out_grouped(&tc, op, out_kind, M, N, G, epi.ldo, out_gstride, Epi::kOutBytes / 16);
        if (rc) return rc;
    }
    const int64_t tiles64 = (int64_t)((M + kBM - 1) / kBM) * ((N + BN - 1) / BN) * G;
    if (tiles64 > 0x7fffffff) return set_error(CHEM_EINVAL, "GEMM: too many tiles for one launch");
    const int tiles = (int)tiles64;
    int grid = num_sms();
    if (max_ctas > 0 && max_ctas < grid) grid = max_ctas;
    if (tiles < grid) grid = tiles;
    const GemmGroups grp{G, A.kind, B.kind, out_kind, gemm_wait_limit()};
    void *pb = prof_begin(st);
    gemm_tn_kernel<BN, STAGES, Epi><<<grid, kGemmThreads, L::kTotal, st>>>(ta, tb, tc, M, N, K, grp, epi, err);
    if (pb)
        prof_end(pb, st, "gemm_tn_kernel<" + std::to_string(BN) + (Epi::kF8 ? ",e4m3> " : "> ") +
                             (G > 1 ? std::to_string(G) + "x" : std::string()) + std::to_string(N) + "x" +
                             std::to_string(K),
                 2.0 * M * N * K * G, (double)esize * ((double)M * K + (double)N * K) * G);
    return check_cuda(cudaGetLastError(), "GEMM launch");
}

// Tile widths the library is built with (the autotuner picks among them).
constexpr int kTileWidths[] = {32, 64, 128, 160, 208, 256};

// G products in one launch (single-CTA tiles only).
template <class Epi>
int launch_gemm_grouped(int bn, const GemmOperand &A, const GemmOperand &B, int G, int out_kind, int64_t out_gstride,
                        int M, int N, int K, const Epi &epi, int *err, cudaStream_t st, int max_ctas = 0) {
    if (M <= 0 || N <= 0 || K <= 0 || G <= 0) return CHEM_OK;
    switch (bn) {
#define CHEMGB_GROUPED_CASE(W_, S_)                                                                                 \
    case W_:                                                                                                        \
        return launch_gemm_grouped_bn<W_, S_>(A, B, G, out_kind, out_gstride, M, N, K, epi, err, st, max_ctas);
        CHEMGB_GROUPED_CASE(32, 8)
        CHEMGB_GROUPED_CASE(64, 8)
        CHEMGB_GROUPED_CASE(128, 6)
        CHEMGB_GROUPED_CASE(160, 5)
        CHEMGB_GROUPED_CASE(208, 4)
        CHEMGB_GROUPED_CASE(256, 4)
#undef CHEMGB_GROUPED_CASE
        default: return set_error(CHEM_EINVAL, "GEMM: unsupported tile width " + std::to_string(bn));
    }
}

template <class Epi>
int launch_gemm(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                const Epi &epi, int *err, cudaStream_t st, int max_ctas = 0) {
    if (M <= 0 || N <= 0 || K <= 0) return CHEM_OK;
    return launch_gemm_grouped(bn, GemmOperand{X, ldx, kMap2D, 0}, GemmOperand{W, ldw, kMap2D, 0}, 1, kMap2D, 0, M, N,
                               K, epi, err, st, max_ctas);
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
// Grouped forms: G products of M x N x K in one launch (the per-species networks). Output
// groups sit side by side in each row (group g's columns start at g x g_out), except for
// gemm_linear_grouped, whose g_out is any element offset (stacked weight gradients: rows x ldo).
int gemm_gelu_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                      const float *bias, int64_t g_bias, void *out, int64_t ldo, int64_t g_out, float *pre,
                      int64_t ldp, int64_t g_pre, int *err, cudaStream_t st, int max_ctas = 0);
int gemm_linear_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                        const float *bias, int64_t g_bias, float *out, int64_t ldo, int64_t g_out, int *err,
                        cudaStream_t st, int max_ctas = 0);
int gemm_gelu_grad_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                           const float *z, int64_t ldz, int64_t g_z, void *out, int64_t ldo, int64_t g_out, int *err,
                           cudaStream_t st, int max_ctas = 0);
// The last hidden layer and the output layer in one launch, h3 kept on chip (gemm_fused34.cuh):
// u = bf16(GELU(X W3^T + b3)) W4^T + b4 in FP32, bitwise gemm_gelu (layer 3) then gemm_linear
// (layer 4). X [M][ldx] BF16 with K3 columns, W3 [N3][ldw3], W4 [N4][ldw4] (K = N3), u [M][ldu].
bool fused34_supported(int K3, int N3, int N4);
int gemm_fused34(const void *X, int64_t ldx, int K3, const void *W3, int64_t ldw3, const void *W4, int64_t ldw4, int M,
                 int N3, int N4, const float *b3, const float *b4, float *u, int64_t ldu, int *err, cudaStream_t st);
// Reduced-precision hidden layer (EpiGeluQ): f8in selects E4M3 operands (X, W) with the per-column
// scale cs, f8out an E4M3 output scaled by inv_so; otherwise BF16.
int gemm_gelu_q(bool f8in, bool f8out, int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N,
                int K, const float *bias, const float *cs, void *out, int64_t ldo, float inv_so, int *err,
                cudaStream_t st, int max_ctas = 0);

}  // namespace chemgb
