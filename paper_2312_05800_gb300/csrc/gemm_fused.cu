// gemm_fused.cu -- host launches of the fused layer pairs: gemm_fused12_kernel
// (the network's first two layers in one persistent launch of CTA pairs, h1 kept
// on chip; gemm_fused.cuh) and gemm_fused34_kernel (the last hidden layer and the
// output layer, h3 kept on chip; gemm_fused34.cuh).
#include "gemm_fused.cuh"
#include "gemm_fused34.cuh"
#include "gemm_launch.cuh"

namespace chemgb {
namespace {

template <int NP>
int launch_fused12_np(const void *X, int64_t ldx, const void *W1, int64_t ldw1, const void *W2, int64_t ldw2, int M,
                      int N1, int N2, const float *b1, const float *b2, void *h2, int64_t ldh2, int *err,
                      cudaStream_t st) {
    using L = F12Smem<NP>;
    static bool configured = false;
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kF12Threads);
    cfg.dynamicSmemBytes = L::kTotal;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!configured) {
        int rc = check_cuda(cudaFuncSetAttribute(gemm_fused12_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)L::kTotal),
                            "fused GEMM smem attribute");
        if (rc) return rc;
        cfg.gridDim = dim3(2 * (num_sms() / 2));
        rc = check_cuda(cudaOccupancyMaxActiveClusters(&max_clusters, gemm_fused12_kernel<NP>, &cfg),
                        "fused GEMM cluster occupancy");
        if (rc) return rc;
        if (max_clusters < 1) return set_error(CHEM_EUNSUPPORTED, "fused GEMM: no CTA pair fits on the device");
        configured = true;
    }
    CUtensorMap tx, tw1, tw2, th2;
    int rc = make_tmap_operand(&tx, X, M, 64, ldx, kBM, 2);
    if (!rc) rc = make_tmap_operand(&tw1, W1, N1, 64, ldw1, kF12Chunk, 2);
    if (!rc) rc = make_tmap_operand(&tw2, W2, N2, N1, ldw2, NP / 2, 2);
    if (!rc) rc = make_tmap_out(&th2, h2, M, N2, ldh2, 2);
    if (rc) return rc;
    const int m_tiles = (M + kBM - 1) / kBM;
    const int clusters = m_tiles < max_clusters ? m_tiles : max_clusters;
    cfg.gridDim = dim3(2 * clusters);
    const F12Args a{M, N1, N2, (N2 + 2 * NP - 1) / (2 * NP), b1, b2, gemm_wait_limit()};
    void *pb = prof_begin(st);
    rc = check_cuda(cudaLaunchKernelEx(&cfg, gemm_fused12_kernel<NP>, tx, tw1, tw2, th2, a, err), "fused GEMM launch");
    if (pb)
        prof_end(pb, st, "gemm_fused12_kernel<" + std::to_string(NP) + "> " + std::to_string(N1) + "x" +
                             std::to_string(N2),
                 2.0 * M * ((double)N1 * 64 + (double)N2 * N1), 2.0 * ((double)M * 64 + (double)N2 * M));
    return rc;
}

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

bool fused12_supported(int K1, int N1, int N2) {
    return K1 == 64 && N1 >= kF12Chunk && N1 % kF12Chunk == 0 && N2 >= 16 && N2 % 16 == 0;
}

int gemm_fused12(const void *X, int64_t ldx, int K1, const void *W1, int64_t ldw1, const void *W2, int64_t ldw2, int M,
                 int N1, int N2, const float *b1, const float *b2, void *h2, int64_t ldh2, int *err, cudaStream_t st) {
    if (M <= 0) return CHEM_OK;
    if (!fused12_supported(K1, N1, N2))
        return set_error(CHEM_EINVAL, "fused GEMM: needs K1 = 64, h1 a multiple of 64 and h2 a multiple of 16");
    if (!aligned16(b1) || !aligned16(b2)) return set_error(CHEM_EINVAL, "fused GEMM: biases must be 16-byte aligned");
    // a pair of CTAs covers 2 NP columns of h2 per pass: the fewest passes with NP <= 400 (the widest
    // pass whose W2 ring fits in shared memory), then the narrowest compiled NP that covers them
    const int passes = (N2 + 799) / 800;
    const int need = (N2 + 2 * passes - 1) / (2 * passes);
    if (need <= 128) return launch_fused12_np<128>(X, ldx, W1, ldw1, W2, ldw2, M, N1, N2, b1, b2, h2, ldh2, err, st);
    if (need <= 256) return launch_fused12_np<256>(X, ldx, W1, ldw1, W2, ldw2, M, N1, N2, b1, b2, h2, ldh2, err, st);
    if (need <= 288) return launch_fused12_np<288>(X, ldx, W1, ldw1, W2, ldw2, M, N1, N2, b1, b2, h2, ldh2, err, st);
    return launch_fused12_np<400>(X, ldx, W1, ldw1, W2, ldw2, M, N1, N2, b1, b2, h2, ldh2, err, st);
}

}  // namespace chemgb
