// dense.cu -- chem_dense_bf16: one dense layer of the Sec. 3.2 network on the
// tensor cores, exposed on its own (the building block of every MLP call).
#include "gemm_launch.cuh"

using namespace chemgb;

namespace {
__device__ int g_dense_err;   // error word used when the caller passes none
}

extern "C" int chem_dense_bf16(int64_t M, int N, int K, const void *x, int64_t ldx, const void *W, int64_t ldw,
                               const float *b, int act, void *y, int64_t ldy, int tile_n, int *err,
                               chem_stream_t stream) {
    if (M < 0 || N < 0 || K < 0 || M > 0x7fffffff) return set_error(CHEM_EINVAL, "chem_dense_bf16: bad sizes");
    if (M == 0 || N == 0) return CHEM_OK;
    if (K == 0) return set_error(CHEM_EINVAL, "chem_dense_bf16: K must be positive");
    if (!x || !W || !y) return set_error(CHEM_EINVAL, "chem_dense_bf16: null array");
    if (ldx < K || ldw < K || ldy < N) return set_error(CHEM_EINVAL, "chem_dense_bf16: leading dimension too small");
    if (act != 0 && act != 1) return set_error(CHEM_EINVAL, "chem_dense_bf16: act must be 0 (none) or 1 (GELU)");
    if (!aligned16(y) || (b && ((reinterpret_cast<uintptr_t>(b) & 3u) != 0)) || (err && !aligned16(err)))
        return set_error(CHEM_EINVAL, "chem_dense_bf16: y and err must be 16-byte aligned, b 4-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_dense_bf16: " + why);
    int *e = err;
    if (!e) {
        int rc = check_cuda(cudaGetSymbolAddress(reinterpret_cast<void **>(&e), g_dense_err), "chem_dense_bf16");
        if (rc) return rc;
    }
    int bn = tile_n > 0 ? tile_n : default_tile_width(N);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (act == 1) return gemm_gelu(bn, x, ldx, W, ldw, (int)M, N, K, b, y, ldy, nullptr, 0, e, st);
    return gemm_linear(bn, x, ldx, W, ldw, (int)M, N, K, b, static_cast<float *>(y), ldy, e, st);
}
