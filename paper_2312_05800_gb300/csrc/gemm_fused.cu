// gemm_fused.cu -- host launch of gemm_fused34_kernel: the last hidden layer and
// the output layer in one persistent launch, h3 kept on chip (gemm_fused34.cuh).
#include "gemm_fused34.cuh"
#include "gemm_launch.cuh"

namespace chemgb {
namespace {

template <int NA, int NB>
int launch_fused34_nb(const void *X, int64_t ldx, int K3, const void *W3, int64_t ldw3, const void *W4, int64_t ldw4,
                      int M, int N4, const float *b3, const float *b4, float *u, int64_t ldu, int *err,
                      cudaStream_t st) {
    using L = F34Smem<NA, NB>;
    static bool configured = false;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(gemm_fused34_kernel<NA, NB>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kTotal),
                            "fused output GEMM smem attribute");
        if (rc) return rc;
        configured = true;
    }
    CUtensorMap tx, t3a, t3b, t4;
    int rc = make_tmap_operand(&tx, X, M, K3, ldx, kBM, 2);
    if (!rc) rc = make_tmap_operand(&t3a, W3, NA + NB, K3, ldw3, NA, 2);
    if (!rc) rc = make_tmap_operand(&t3b, W3, NA + NB, K3, ldw3, NB, 2);
    if (!rc) rc = make_tmap_operand(&t4, W4, N4, NA + NB, ldw4, 32, 2);
    if (rc) return rc;
    const int m_tiles = (M + kBM - 1) / kBM;
    int grid = num_sms();
    if (m_tiles < grid) grid = m_tiles;
    const F34Args a{M, K3, NA + NB, N4, b3, b4, u, ldu, gemm_wait_limit()};
    void *pb = prof_begin(st);
    gemm_fused34_kernel<NA, NB><<<grid, kF34Threads, L::kTotal, st>>>(tx, t3a, t3b, t4, a, err);
    if (pb)
        prof_end(pb, st, "gemm_fused34_kernel " + std::to_string(NA + NB) + "x" + std::to_string(K3) + "+" +
                             std::to_string(N4) + "x" + std::to_string(NA + NB),
                 2.0 * M * ((double)(NA + NB) * K3 + (double)N4 * (NA + NB)),
                 2.0 * (double)M * K3 + 4.0 * (double)M * N4);
    return check_cuda(cudaGetLastError(), "fused output GEMM launch");
}

}  // namespace

bool fused34_supported(int K3, int N3, int N4) { return N3 == 400 && K3 >= 64 && N4 >= 1 && N4 <= 32; }

int gemm_fused34(const void *X, int64_t ldx, int K3, const void *W3, int64_t ldw3, const void *W4, int64_t ldw4, int M,
                 int N3, int N4, const float *b3, const float *b4, float *u, int64_t ldu, int *err, cudaStream_t st) {
    if (M <= 0) return CHEM_OK;
    if (!fused34_supported(K3, N3, N4))
        return set_error(CHEM_EINVAL, "fused output GEMM: needs 400 hidden units and at most 32 outputs");
    if (!aligned16(b3) || !aligned16(u) || (ldu & 3) != 0)
        return set_error(CHEM_EINVAL, "fused output GEMM: bias and output must be 16-byte aligned");
    return launch_fused34_nb<192, 208>(X, ldx, K3, W3, ldw3, W4, ldw4, M, N4, b3, b4, u, ldu, err, st);
}

}  // namespace chemgb
