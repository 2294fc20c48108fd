// gemm_grad.cu -- instantiations of the tensor-core GEMM whose epilogue
// multiplies by GELU'(z) (backward pass of the Sec. 3.2 network).
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu_grad(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *z, int64_t ldz, void *out, int64_t ldo, int *err, cudaStream_t st, int max_ctas) {
    EpiGeluGrad e{M, N, z, ldz, static_cast<__nv_bfloat16 *>(out), ldo};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
int gemm_gelu_grad_grouped(int bn, const GemmOperand &X, const GemmOperand &W, int G, int M, int N, int K,
                           const float *z, int64_t ldz, int64_t g_z, void *out, int64_t ldo, int64_t g_out, int *err,
                           cudaStream_t st, int max_ctas) {
    EpiGeluGrad e{M, N, z, ldz, static_cast<__nv_bfloat16 *>(out), ldo, g_z, g_out};
    return launch_gemm_grouped(bn, X, W, G, kMap2D, 0, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
