// gemm_q_88.cu -- a middle hidden layer of the reduced-precision forward:
// E4M3 operands with per-output-column scales, bias + GELU, E4M3 output.
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu_q_88(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *bias, const float *cs, void *out, int64_t ldo, float inv_so, int *err,
                   cudaStream_t st, int max_ctas) {
    EpiGeluQ<true, true> e{M, N, bias, cs, out, ldo, inv_so};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
