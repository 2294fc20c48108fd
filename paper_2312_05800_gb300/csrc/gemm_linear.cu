// gemm_linear.cu -- instantiations of the tensor-core GEMM with the FP32
// bias-only epilogue (output layer of the Sec. 3.2 network; weight gradients).
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_linear(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                const float *bias, float *out, int64_t ldo, int *err, cudaStream_t st, int max_ctas) {
    EpiLinear e{M, N, bias, out, ldo};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
int gemm_linear_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                        const float *bias, int64_t g_bias, float *out, int64_t ldo, int64_t g_out, int *err,
                        cudaStream_t st, int max_ctas) {
    EpiLinear e{M, N, bias, out, ldo, g_out, g_bias};
    return launch_gemm_grouped(bn, X, W, G, kMap2D, 0, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
