// gemm_q_8b.cu -- the last hidden layer of the reduced-precision forward
// (E4M3 operands, bias + GELU, BF16 output for the BF16 output layer), and
// the dispatcher over the three reduced-precision layer kinds.
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu_q_b8(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *bias, void *out, int64_t ldo, float inv_so, int *err, cudaStream_t st, int max_ctas);
int gemm_gelu_q_88(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *bias, const float *cs, void *out, int64_t ldo, float inv_so, int *err,
                   cudaStream_t st, int max_ctas);

int gemm_gelu_q(bool f8in, bool f8out, int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N,
                int K, const float *bias, const float *cs, void *out, int64_t ldo, float inv_so, int *err,
                cudaStream_t st, int max_ctas) {
    if (!f8in && f8out) return gemm_gelu_q_b8(bn, X, ldx, W, ldw, M, N, K, bias, out, ldo, inv_so, err, st, max_ctas);
    if (f8in && f8out) return gemm_gelu_q_88(bn, X, ldx, W, ldw, M, N, K, bias, cs, out, ldo, inv_so, err, st, max_ctas);
    if (f8in) {
        EpiGeluQ<true, false> e{M, N, bias, cs, out, ldo, 1.0f};
        return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
    }
    return set_error(CHEM_EINVAL, "gemm_gelu_q: BF16 in and out is gemm_gelu");
}
}  // namespace chemgb
