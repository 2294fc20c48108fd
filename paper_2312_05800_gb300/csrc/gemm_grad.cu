// gemm_grad.cu -- instantiations of the tensor-core GEMM whose epilogue
// multiplies by GELU'(z) (backward pass of the Sec. 3.2 network).
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu_grad(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K,
                   const float *z, int64_t ldz, void *out, int64_t ldo, int *err, cudaStream_t st, int max_ctas) {
    EpiGeluGrad e{M, N, z, ldz, static_cast<__nv_bfloat16 *>(out), ldo};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
