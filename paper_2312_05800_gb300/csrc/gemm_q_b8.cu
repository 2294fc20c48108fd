// gemm_q_b8.cu -- the first hidden layer of the reduced-precision forward:
// BF16 operands, bias + GELU, output quantised to E4M3 for the next layer.
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu_q_b8(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *bias, void *out, int64_t ldo, float inv_so, int *err, cudaStream_t st, int max_ctas) {
    EpiGeluQ<false, true> e{M, N, bias, nullptr, out, ldo, inv_so};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
