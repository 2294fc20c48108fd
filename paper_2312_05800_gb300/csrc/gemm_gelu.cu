// gemm_gelu.cu -- instantiations of the tensor-core GEMM with the bias + GELU
// epilogue (hidden layers of the Sec. 3.2 network, forward).
#include "gemm_launch.cuh"

namespace chemgb {
int gemm_gelu(int bn, const void *X, int64_t ldx, const void *W, int64_t ldw, int M, int N, int K, const float *bias,
              void *out, int64_t ldo, float *pre, int64_t ldp, int *err, cudaStream_t st, int max_ctas) {
    EpiGelu e{M, N, bias, static_cast<__nv_bfloat16 *>(out), ldo, pre, ldp};
    return launch_gemm(bn, X, ldx, W, ldw, M, N, K, e, err, st, max_ctas);
}
}  // namespace chemgb
