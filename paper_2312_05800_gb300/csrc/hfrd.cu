// hfrd.cu -- the random training-data generation of Sec. 3.1 on the GPU.
//
// Each base composition (T, p, Y) yields a random composition by Eq. 1-4 with
// uniform random numbers c in [-1, 1] that the caller draws (they are inputs,
// one per equation and per species):
//   T'    = T + alpha c_T (T_max - T_min)                 (Eq. 1)
//   p'    = p + beta  c_p (p_max - p_min)                 (Eq. 2)
//   Y'_b  = Y_b + alpha c_b (Y_b,max - Y_b,min)           (Eq. 3, b the bath species N2)
//   Y'_j  = max(Y_j, 0)^(1 + gamma c_j), j != b           (Eq. 4)
// then the species other than the bath are scaled to sum to 1 - Y'_b. A state
// is kept when it is admissible (0 <= Y'_b < 1, T' > 0, p' > 0, some other
// species left) and its element ratios lie in Table 1: H/C, O/N and the
// equivalence ratio phi = (2 n_C + n_H / 2) / n_O from the element moles
// n_e = sum_k a_ek Y'_k / W_k. The lean-mixing states of Sec. 3.1 are linear
// blends, in T and every Y, between two endpoint states (the leanest mixture's
// adiabatic equilibrium and ambient air).
//
// One thread per state; species loops in ascending order with explicitly
// rounded FP64 operations (no contraction into FMA), so every value is the
// plain definition's.
#include <cmath>

#include "internal.cuh"

namespace chemgb {
namespace {

struct HfrdArgs {
    chem_hfrd_params p;
    int N, bath;
    int atoms[4][kMaxSpecies];     // counts of C, H, O, N per species
};

__global__ void hfrd_kernel(int64_t n, int64_t ld, HfrdArgs a, const double *__restrict__ W,
                            const double *__restrict__ T, const double *__restrict__ p, const double *__restrict__ Y,
                            const double *__restrict__ c, double *__restrict__ T2, double *__restrict__ p2,
                            double *__restrict__ Y2, uint8_t *__restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const chem_hfrd_params &q = a.p;
    const int N = a.N, b = a.bath;
    const double t2 = __dadd_rn(T[i], __dmul_rn(__dmul_rn(q.alpha, c[i]), __dsub_rn(q.T_max, q.T_min)));
    const double pp = __dadd_rn(p[i], __dmul_rn(__dmul_rn(q.beta, c[ld + i]), __dsub_rn(q.p_max, q.p_min)));
    const double yb = __dadd_rn(Y[(int64_t)b * ld + i],
                                __dmul_rn(__dmul_rn(q.alpha, c[2 * ld + i]), __dsub_rn(q.Yb_max, q.Yb_min)));
    T2[i] = t2;
    p2[i] = pp;
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
        if (k == b) continue;
        const double y = fmax(Y[(int64_t)k * ld + i], 0.0);
        const double v = pow(y, __dadd_rn(1.0, __dmul_rn(q.gamma, c[(int64_t)(3 + k) * ld + i])));
        Y2[(int64_t)k * ld + i] = v;
        s = __dadd_rn(s, v);
    }
    const bool ok = (yb >= 0.0 && yb < 1.0) && s > 0.0 && t2 > 0.0 && pp > 0.0;
    if (!ok) {
        Y2[(int64_t)b * ld + i] = 0.0;
        keep[i] = 0;
        return;
    }
    const double f = __ddiv_rn(__dsub_rn(1.0, yb), s);
    double ne[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < N; ++k) {
        double v;
        if (k == b) {
            v = yb;
        } else {
            v = __dmul_rn(Y2[(int64_t)k * ld + i], f);
        }
        Y2[(int64_t)k * ld + i] = v;
        const double yw = __ddiv_rn(v, W[k]);
#pragma unroll
        for (int e = 0; e < 4; ++e) ne[e] = __dadd_rn(ne[e], __dmul_rn((double)a.atoms[e][k], yw));
    }
    const double hc = __ddiv_rn(ne[1], ne[0]);
    const double on = __ddiv_rn(ne[2], ne[3]);
    const double phi = __ddiv_rn(__dadd_rn(__dmul_rn(2.0, ne[0]), __dmul_rn(0.5, ne[1])), ne[2]);
    const bool in = hc >= q.hc_lo && hc <= q.hc_hi && on >= q.on_lo && on <= q.on_hi && phi >= q.phi_lo &&
                    phi <= q.phi_hi;
    keep[i] = in ? 1 : 0;
}

struct BlendArgs {
    int N;
    double Ta, Tb;
    double Ya[kMaxSpecies], Yb[kMaxSpecies];
};

__global__ void blend_kernel(int64_t n, int64_t ld, BlendArgs a, const double *__restrict__ s,
                             double *__restrict__ T, double *__restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = s[i], u = __dsub_rn(1.0, t);
    T[i] = __dadd_rn(__dmul_rn(u, a.Ta), __dmul_rn(t, a.Tb));
    for (int k = 0; k < a.N; ++k) Y[(int64_t)k * ld + i] = __dadd_rn(__dmul_rn(u, a.Ya[k]), __dmul_rn(t, a.Yb[k]));
}

}  // namespace
}  // namespace chemgb

using namespace chemgb;

extern "C" void chem_hfrd_params_default(chem_hfrd_params *q) {
    if (!q) return;
    *q = chem_hfrd_params{};
    q->alpha = 0.125;
    q->beta = 10.0;
    q->gamma = 0.1;
    q->hc_lo = 2.65;
    q->hc_hi = 4.67;
    q->on_lo = 0.254;
    q->on_hi = 0.32;
    q->phi_lo = 0.20;
    q->phi_hi = 1.15;
}

extern "C" int chem_hfrd_perturb(const chem_mech *m, const chem_hfrd_params *prm, const int32_t *chon, int64_t n,
                                 int64_t ld, const double *T, const double *p, const double *Y, const double *c,
                                 double *T2, double *p2, double *Y2, uint8_t *keep, chem_stream_t stream) {
    if (!m || !prm || !chon) return set_error(CHEM_EINVAL, "chem_hfrd_perturb: null handle, parameters or atom table");
    if (n < 0 || ld < n || (ld & 3) != 0) return set_error(CHEM_EINVAL, "chem_hfrd_perturb: need 0 <= n <= ld, ld % 4 == 0");
    if (n == 0) return CHEM_OK;
    if (!T || !p || !Y || !c || !T2 || !p2 || !Y2 || !keep) return set_error(CHEM_EINVAL, "chem_hfrd_perturb: null array");
    const void *ptrs[] = {T, p, Y, c, T2, p2, Y2, keep};
    for (const void *q : ptrs)
        if (!aligned16(q)) return set_error(CHEM_EINVAL, "chem_hfrd_perturb: arrays must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_hfrd_perturb: " + why);
    HfrdArgs a;
    a.p = *prm;
    a.N = m->N;
    a.bath = m->bath;
    for (int e = 0; e < 4; ++e)
        for (int k = 0; k < kMaxSpecies; ++k) a.atoms[e][k] = k < m->N ? chon[e * m->N + k] : 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *pb = prof_begin(st);
    hfrd_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, ld, a, m->dev.W, T, p, Y, c, T2, p2, Y2, keep);
    // algorithmic bytes: reads T, p, Y and the 3 + N draws; writes T', p', Y' and the keep byte
    prof_end(pb, st, "hfrd_kernel", 0.0, (double)n * (8.0 * ((2 * m->N + 5) + (m->N + 2)) + 1.0));
    return check_cuda(cudaGetLastError(), "chem_hfrd_perturb launch");
}

extern "C" int chem_hfrd_blend(int N, int64_t n, int64_t ld, const double *s, double Ta, const double *Ya, double Tb,
                               const double *Yb, double *T, double *Y, chem_stream_t stream) {
    if (N < 1 || N > kMaxSpecies || n < 0 || ld < n || (ld & 3) != 0)
        return set_error(CHEM_EINVAL, "chem_hfrd_blend: need 1 <= N <= 64, 0 <= n <= ld, ld % 4 == 0");
    if (n == 0) return CHEM_OK;
    if (!s || !Ya || !Yb || !T || !Y) return set_error(CHEM_EINVAL, "chem_hfrd_blend: null array");
    if (!aligned16(s) || !aligned16(T) || !aligned16(Y))
        return set_error(CHEM_EINVAL, "chem_hfrd_blend: device arrays must be 16-byte aligned");
    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_hfrd_blend: " + why);
    BlendArgs a;
    a.N = N;
    a.Ta = Ta;
    a.Tb = Tb;
    for (int k = 0; k < kMaxSpecies; ++k) {
        a.Ya[k] = k < N ? Ya[k] : 0.0;
        a.Yb[k] = k < N ? Yb[k] : 0.0;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    blend_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, ld, a, s, T, Y);
    return check_cuda(cudaGetLastError(), "chem_hfrd_blend launch");
}
