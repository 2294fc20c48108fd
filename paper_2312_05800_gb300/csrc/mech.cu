// mech.cu -- mechanism loading (host parse, derived tables, one device blob),
// error reporting and option defaults of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "internal.cuh"

namespace chemgb {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CHEM_OK;
    return set_error(CHEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool device_ok(std::string *why) {
    // cached per device: 1 = sm_103, 2 = other architecture
    static int state[64] = {0};
    static int cc[64] = {0};
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        if (why) *why = "no CUDA device";
        return false;
    }
    if (dev < 64 && state[dev] == 0) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
            cudaGetLastError();
            if (why) *why = "cannot query the device";
            return false;
        }
        cc[dev] = major * 10 + minor;
        state[dev] = (major == 10 && minor == 3) ? 1 : 2;
    }
    if (dev >= 64 || state[dev] != 1) {
        if (why) *why = "device is sm_" + std::to_string(dev < 64 ? cc[dev] : 0) +
                        "; this library is built for sm_103a only";
        return false;
    }
    return true;
}

namespace {

struct Reader {
    const uint8_t *p, *end;
    bool ok = true;
    template <typename T>
    void read(T *dst, size_t n) {
        size_t b = sizeof(T) * n;
        if (!ok || (size_t)(end - p) < b) { ok = false; return; }
        std::memcpy(dst, p, b);
        p += b;
    }
};

// Appends a typed array to the host image of the device blob (256-byte aligned).
struct BlobBuilder {
    std::vector<uint8_t> bytes;
    template <typename T>
    size_t add(const std::vector<T> &v) {
        size_t off = (bytes.size() + 255) & ~size_t(255);
        bytes.resize(off + sizeof(T) * v.size());
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), sizeof(T) * v.size());
        return off;
    }
};

template <typename real>
struct PropOffsets { size_t invW, nasa_cp, nasa_h, visc, wilke, diff; };

template <typename real>
PropOffsets<real> add_prop_tables(BlobBuilder &bb, int N, int Np, const std::vector<double> &W,
                                  const std::vector<double> &lo, const std::vector<double> &hi,
                                  const std::vector<double> &visc, const std::vector<double> &diff) {
    std::vector<real> invW(N), cp(2 * N * 5), h(2 * N * 6), vis(N * 5);
    std::vector<real> wil((size_t)3 * N * Np, real(0)), dif((size_t)5 * N * Np, real(0));
    for (int k = 0; k < N; ++k) {
        invW[k] = real(1.0 / W[k]);
        for (int r = 0; r < 2; ++r) {
            const double *a = (r == 0 ? lo.data() : hi.data()) + 7 * k;
            for (int i = 0; i < 5; ++i) cp[(r * N + k) * 5 + i] = real(a[i]);
            h[(r * N + k) * 6 + 0] = real(a[0]);
            h[(r * N + k) * 6 + 1] = real(a[1] / 2.0);
            h[(r * N + k) * 6 + 2] = real(a[2] / 3.0);
            h[(r * N + k) * 6 + 3] = real(a[3] / 4.0);
            h[(r * N + k) * 6 + 4] = real(a[4] / 5.0);
            h[(r * N + k) * 6 + 5] = real(a[5]);
        }
        for (int i = 0; i < 5; ++i) vis[k * 5 + i] = real(visc[k * 5 + i]);
        for (int j = 0; j < N; ++j) {
            // Wilke weights: Phi_kj = c_kj (1 + w_jk r_k / r_j)^2, r = sqrt(mu)
            double c = 1.0 / std::sqrt(8.0 * (1.0 + W[k] / W[j]));
            double w = std::pow(W[j] / W[k], 0.25);
            wil[(0 * (size_t)N + k) * Np + j] = real(c);
            wil[(1 * (size_t)N + k) * Np + j] = real(2.0 * c * w);
            wil[(2 * (size_t)N + k) * Np + j] = real(c * w * w);
            for (int n = 0; n < 5; ++n)
                dif[((size_t)n * N + k) * Np + j] = (j == k) ? real(0) : real(diff[((size_t)j * N + k) * 5 + n]);
        }
    }
    PropOffsets<real> o;
    o.invW = bb.add(invW);
    o.nasa_cp = bb.add(cp);
    o.nasa_h = bb.add(h);
    o.visc = bb.add(vis);
    o.wilke = bb.add(wil);
    o.diff = bb.add(dif);
    return o;
}

template <typename real>
PropTables<real> resolve(const PropOffsets<real> &o, uint8_t *base) {
    PropTables<real> t;
    t.invW = reinterpret_cast<const real *>(base + o.invW);
    t.nasa_cp = reinterpret_cast<const real *>(base + o.nasa_cp);
    t.nasa_h = reinterpret_cast<const real *>(base + o.nasa_h);
    t.visc = reinterpret_cast<const real *>(base + o.visc);
    t.wilke = reinterpret_cast<const real *>(base + o.wilke);
    t.diff = reinterpret_cast<const real *>(base + o.diff);
    return t;
}

}  // namespace
}  // namespace chemgb

using namespace chemgb;

extern "C" int chem_mech_load_bytes(const void *data, size_t nbytes, chem_mech **out) {
    if (!data || !out) return set_error(CHEM_EINVAL, "chem_mech_load_bytes: null argument");
    *out = nullptr;
    Reader rd{static_cast<const uint8_t *>(data), static_cast<const uint8_t *>(data) + nbytes};
    char magic[8];
    rd.read(magic, 8);
    if (!rd.ok || std::memcmp(magic, "CHMECH01", 8) != 0) return set_error(CHEM_EIO, "mechanism: bad magic");
    int32_t hdr[4];
    double th[4];
    rd.read(hdr, 4);
    rd.read(th, 4);
    int N = hdr[0], R = hdr[1], E = hdr[2], bath = hdr[3];
    if (!rd.ok) return set_error(CHEM_EIO, "mechanism: truncated header");
    if (N < 1 || N > kMaxSpecies || R < 1 || R > kMaxReactions || E < 1 || E > 16 || bath < 0 || bath >= N)
        return set_error(CHEM_EINVAL, "mechanism: sizes out of range (1 <= N <= 64, 1 <= R <= 4096)");
    std::vector<double> W(N), lo(7 * N), hi(7 * N), sigma(N), eps(N), visc(5 * N), diff((size_t)5 * N * N);
    std::vector<int32_t> elem(N * E), rtype(R), reac(3 * R), prod(3 * R);
    std::vector<double> A(R), beta(R), Ea(R), A0(R), beta0(R), Ea0(R), troe(4 * R), eff((size_t)R * N);
    rd.read(W.data(), N); rd.read(lo.data(), 7 * N); rd.read(hi.data(), 7 * N); rd.read(elem.data(), N * E);
    rd.read(sigma.data(), N); rd.read(eps.data(), N); rd.read(visc.data(), 5 * N); rd.read(diff.data(), diff.size());
    rd.read(rtype.data(), R); rd.read(reac.data(), 3 * R); rd.read(prod.data(), 3 * R);
    rd.read(A.data(), R); rd.read(beta.data(), R); rd.read(Ea.data(), R);
    rd.read(A0.data(), R); rd.read(beta0.data(), R); rd.read(Ea0.data(), R);
    rd.read(troe.data(), 4 * R); rd.read(eff.data(), eff.size());
    if (!rd.ok) return set_error(CHEM_EIO, "mechanism: truncated body");
    for (int k = 0; k < N; ++k)
        if (!(W[k] > 0.0)) return set_error(CHEM_EIO, "mechanism: non-positive molar mass");
    for (int j = 0; j < R; ++j) {
        if (rtype[j] < 0 || rtype[j] > 2) return set_error(CHEM_EIO, "mechanism: bad reaction type");
        for (int i = 0; i < 3; ++i)
            if (reac[3 * j + i] < -1 || reac[3 * j + i] >= N || prod[3 * j + i] < -1 || prod[3 * j + i] >= N)
                return set_error(CHEM_EIO, "mechanism: species index out of range");
        if (reac[3 * j] < 0 || prod[3 * j] < 0) return set_error(CHEM_EIO, "mechanism: empty reaction side");
        if (!(A[j] > 0.0) || (rtype[j] == 2 && !(A0[j] > 0.0)))
            return set_error(CHEM_EIO, "mechanism: non-positive pre-exponential factor");
    }
    int Np = (N + 3) & ~3;

    // Device order of the reactions: Troe fall-off first, then three-body, then
    // elementary (stable within each type). Lanes of a warp take consecutive
    // reactions, so the long fall-off and third-body code paths then occupy
    // few warp iterations; sums over reactions only change their order.
    {
        std::vector<int> order;
        for (int t : {2, 1, 0})
            for (int j = 0; j < R; ++j)
                if (rtype[j] == t) order.push_back(j);
        auto perm_d = [&](std::vector<double> &v, int w) {
            std::vector<double> o(v.size());
            for (int j = 0; j < R; ++j)
                for (int i = 0; i < w; ++i) o[(size_t)j * w + i] = v[(size_t)order[j] * w + i];
            v.swap(o);
        };
        auto perm_i = [&](std::vector<int32_t> &v, int w) {
            std::vector<int32_t> o(v.size());
            for (int j = 0; j < R; ++j)
                for (int i = 0; i < w; ++i) o[(size_t)j * w + i] = v[(size_t)order[j] * w + i];
            v.swap(o);
        };
        perm_i(rtype, 1); perm_i(reac, 3); perm_i(prod, 3);
        perm_d(A, 1); perm_d(beta, 1); perm_d(Ea, 1); perm_d(A0, 1); perm_d(beta0, 1); perm_d(Ea0, 1);
        perm_d(troe, 4); perm_d(eff, N);
    }

    BlobBuilder bb;
    auto o32 = add_prop_tables<float>(bb, N, Np, W, lo, hi, visc, diff);
    auto o64 = add_prop_tables<double>(bb, N, Np, W, lo, hi, visc, diff);
    std::vector<double> nasa(2 * N * 7);
    for (int k = 0; k < N; ++k)
        for (int i = 0; i < 7; ++i) { nasa[k * 7 + i] = lo[k * 7 + i]; nasa[(N + k) * 7 + i] = hi[k * 7 + i]; }
    std::vector<double> lnA(R), EaR(R), lnA0(R), Ea0R(R);
    std::vector<int32_t> tb_row(R, -1), dnu(R, 0);
    std::vector<double> effc;
    int n_tb = 0;
    for (int j = 0; j < R; ++j) {
        lnA[j] = std::log(A[j]);
        EaR[j] = Ea[j] / kR;
        lnA0[j] = (A0[j] > 0.0) ? std::log(A0[j]) : 0.0;
        Ea0R[j] = Ea0[j] / kR;
        for (int i = 0; i < 3; ++i) dnu[j] += (prod[3 * j + i] >= 0) - (reac[3 * j + i] >= 0);
        if (rtype[j] != 0) {
            tb_row[j] = n_tb++;
            for (int k = 0; k < N; ++k) effc.push_back(eff[(size_t)j * N + k]);
        }
    }
    if (effc.empty()) effc.push_back(0.0);
    // species -> (reaction, signed nu) incidence, reactions in ascending order
    std::vector<int32_t> inc_ptr(N + 1, 0);
    std::vector<int2> inc;
    for (int k = 0; k < N; ++k) {
        inc_ptr[k] = (int)inc.size();
        for (int j = 0; j < R; ++j) {
            int nu = 0;
            for (int i = 0; i < 3; ++i) nu += (prod[3 * j + i] == k) - (reac[3 * j + i] == k);
            bool touches = false;
            for (int i = 0; i < 3; ++i) touches |= (prod[3 * j + i] == k) || (reac[3 * j + i] == k);
            if (touches && nu != 0) inc.push_back(make_int2(j, nu));
        }
    }
    inc_ptr[N] = (int)inc.size();
    if (inc.empty()) inc.push_back(make_int2(0, 0));
    std::vector<uint32_t> counters(kNumCounters, 0u);
    std::vector<double> nasa_s(2 * N * 6), troe_r(4 * R);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < N; ++k) {
            const double *a = (r == 0 ? lo.data() : hi.data()) + 7 * k;
            double *o = nasa_s.data() + (r * N + k) * 6;
            o[0] = a[0]; o[1] = a[1]; o[2] = a[2] / 2.0; o[3] = a[3] / 3.0; o[4] = a[4] / 4.0; o[5] = a[6];
        }
    for (int j = 0; j < R; ++j) {
        troe_r[4 * j + 0] = troe[4 * j + 0];
        troe_r[4 * j + 1] = (troe[4 * j + 1] != 0.0) ? 1.0 / troe[4 * j + 1] : 0.0;
        troe_r[4 * j + 2] = (troe[4 * j + 2] != 0.0) ? 1.0 / troe[4 * j + 2] : 0.0;
        troe_r[4 * j + 3] = troe[4 * j + 3];
    }
    std::vector<int32_t> rsp(6 * R, -1), rnu(6 * R, 0), tb_list;
    for (int j = 0; j < R; ++j) {
        int cnt = 0;
        for (int slot = 0; slot < 6; ++slot) {
            int sp = slot < 3 ? reac[3 * j + slot] : prod[3 * j + slot - 3];
            if (sp < 0) continue;
            bool seen = false;
            for (int u = 0; u < cnt; ++u) seen |= (rsp[6 * j + u] == sp);
            if (seen) continue;
            int nu = 0;
            for (int i = 0; i < 3; ++i) nu += (prod[3 * j + i] == sp) - (reac[3 * j + i] == sp);
            rsp[6 * j + cnt] = sp;
            rnu[6 * j + cnt] = nu;
            ++cnt;
        }
        if (rtype[j] != 0) tb_list.push_back(j);
    }
    if (tb_list.empty()) tb_list.push_back(0);

    size_t off_W = bb.add(W), off_nasa = bb.add(nasa), off_rtype = bb.add(rtype), off_reac = bb.add(reac),
           off_prod = bb.add(prod), off_lnA = bb.add(lnA), off_beta = bb.add(beta), off_EaR = bb.add(EaR),
           off_lnA0 = bb.add(lnA0), off_beta0 = bb.add(beta0), off_Ea0R = bb.add(Ea0R), off_troe = bb.add(troe),
           off_tb = bb.add(tb_row), off_eff = bb.add(effc), off_incp = bb.add(inc_ptr), off_inc = bb.add(inc),
           off_dnu = bb.add(dnu), off_cnt = bb.add(counters), off_nasa_s = bb.add(nasa_s),
           off_troe_r = bb.add(troe_r), off_rsp = bb.add(rsp), off_rnu = bb.add(rnu), off_tbl = bb.add(tb_list);

    std::string why;
    if (!device_ok(&why)) return set_error(CHEM_EUNSUPPORTED, "chem_mech_load: " + why);
    void *blob = nullptr;
    int rc = check_cuda(cudaMalloc(&blob, bb.bytes.size()), "chem_mech_load: cudaMalloc");
    if (rc) return rc;
    rc = check_cuda(cudaMemcpy(blob, bb.bytes.data(), bb.bytes.size(), cudaMemcpyHostToDevice),
                    "chem_mech_load: cudaMemcpy");
    if (rc) { cudaFree(blob); return rc; }

    chem_mech *m = new chem_mech();
    m->N = N; m->R = R; m->E = E; m->bath = bath;
    m->P_std = th[0]; m->T_lo = th[1]; m->T_mid = th[2]; m->T_hi = th[3];
    m->blob = blob;
    m->blob_bytes = bb.bytes.size();
    cudaGetDevice(&m->device);
    uint8_t *base = static_cast<uint8_t *>(blob);
    DevMech &d = m->dev;
    d.N = N; d.R = R; d.Np = Np; d.n_tb = n_tb; d.P_std = th[0]; d.T_mid = th[2];
    d.f32 = resolve(o32, base);
    d.f64 = resolve(o64, base);
    d.W = reinterpret_cast<const double *>(base + off_W);
    d.nasa = reinterpret_cast<const double *>(base + off_nasa);
    d.rtype = reinterpret_cast<const int *>(base + off_rtype);
    d.reac = reinterpret_cast<const int *>(base + off_reac);
    d.prod = reinterpret_cast<const int *>(base + off_prod);
    d.lnA = reinterpret_cast<const double *>(base + off_lnA);
    d.beta = reinterpret_cast<const double *>(base + off_beta);
    d.EaR = reinterpret_cast<const double *>(base + off_EaR);
    d.lnA0 = reinterpret_cast<const double *>(base + off_lnA0);
    d.beta0 = reinterpret_cast<const double *>(base + off_beta0);
    d.Ea0R = reinterpret_cast<const double *>(base + off_Ea0R);
    d.troe = reinterpret_cast<const double *>(base + off_troe);
    d.tb_row = reinterpret_cast<const int *>(base + off_tb);
    d.eff = reinterpret_cast<const double *>(base + off_eff);
    d.inc_ptr = reinterpret_cast<const int *>(base + off_incp);
    d.inc = reinterpret_cast<const int2 *>(base + off_inc);
    d.dnu = reinterpret_cast<const int *>(base + off_dnu);
    d.counters = reinterpret_cast<unsigned int *>(base + off_cnt);
    d.nasa_s = reinterpret_cast<const double *>(base + off_nasa_s);
    d.troe_r = reinterpret_cast<const double *>(base + off_troe_r);
    d.rsp = reinterpret_cast<const int *>(base + off_rsp);
    d.rnu = reinterpret_cast<const int *>(base + off_rnu);
    d.tb_list = reinterpret_cast<const int *>(base + off_tbl);
    d.lnPR = std::log(th[0] / kR);
    *out = m;
    return CHEM_OK;
}

extern "C" int chem_mech_load(const char *path, chem_mech **out) {
    if (!path || !out) return set_error(CHEM_EINVAL, "chem_mech_load: null argument");
    std::ifstream f(path, std::ios::binary);
    if (!f) return set_error(CHEM_EIO, std::string("chem_mech_load: cannot open ") + path);
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    return chem_mech_load_bytes(s.data(), s.size(), out);
}

extern "C" int chem_mech_free(chem_mech *m) {
    if (!m) return set_error(CHEM_EINVAL, "chem_mech_free: null handle");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->blob);
    if (prev >= 0) cudaSetDevice(prev);
    delete m;
    return CHEM_OK;
}

extern "C" int chem_mech_nspecies(const chem_mech *m) { return m ? m->N : -1; }
extern "C" int chem_mech_nreactions(const chem_mech *m) { return m ? m->R : -1; }

extern "C" void chem_ode_opts_default(chem_ode_opts *o) {
    if (!o) return;
    o->rtol = 1e-6;
    o->atol_Y = 1e-12;
    o->atol_T = 1e-6;
    o->h0 = 1e-9;
    o->max_steps = 10000;
    o->mode = CHEM_ODE_FP64;
}

extern "C" const char *chem_last_error(void) { return chemgb::g_last_error.c_str(); }

extern "C" const char *chem_version(void) {
    return "chemgb 0.1 (CUDA " CHEMGB_STR(__CUDACC_VER_MAJOR__) "." CHEMGB_STR(__CUDACC_VER_MINOR__) ", sm_103a)";
}
