// gemm_gelu.cu -- instantiations of the tensor-core GEMM with the bias + GELU
// epilogue (hidden layers of the Sec. 3.2 network, forward).
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K, const float *bias,
              void *out, int64_t ldo, float *pre, int64_t ldp, int *err, cudaStream_t st, int max_ctas) {
    EpiGelu e{M, N, bias, static_cast<__nv_bfloat16 *>(out), ldo, pre, ldp};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
int gemm_gelu_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                      const float *bias, int64_t g_bias, void *out, int64_t ldo, int64_t g_out, float *pre,
                      int64_t ldp, int64_t g_pre, int *err, cudaStream_t st, int max_ctas) {
    EpiGelu e{M, N, bias, static_cast<__nv_bfloat16 *>(out), ldo, pre, ldp, g_out, g_bias, g_pre};
    return launch_gemm_grouped(bn, X, W, G, kMapColGrp, g_out, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
