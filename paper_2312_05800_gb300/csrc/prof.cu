// prof.cu -- opt-in per-kernel timing: CUDA events recorded on the launch
// stream around each tagged kernel, accumulated per tag (kernel and shape).
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace chemgb {
namespace {

struct Pending {
    std::string tag;
    double flops, bytes;
    cudaEvent_t a, b;
};
struct Acc {
    int launches = 0;
    double ms = 0, flops = 0, bytes = 0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::map<std::string, Acc> g_acc;

void drain_locked() {
    for (auto &p : g_pending) {
        float ms = 0.0f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        Acc &a = g_acc[p.tag];
        a.launches += 1;
        a.ms += ms;
        a.flops += p.flops;
        a.bytes += p.bytes;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
}

}  // namespace

bool prof_on() { return g_on; }

void *prof_begin(cudaStream_t st) {
    if (!g_on) return nullptr;
    cudaEvent_t a;
    if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
    cudaEventRecord(a, st);
    return a;
}

void prof_end(void *begin, cudaStream_t st, const std::string &tag, double flops, double bytes) {
    if (!begin) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> l(g_mu);
    g_pending.push_back({tag, flops, bytes, static_cast<cudaEvent_t>(begin), b});
}

}  // namespace chemgb

using namespace chemgb;

extern "C" int chem_prof_enable(int on) {
    std::lock_guard<std::mutex> l(g_mu);
    drain_locked();
    g_acc.clear();
    g_on = (on != 0);
    return CHEM_OK;
}

extern "C" int chem_prof_read(char *buf, int64_t buflen) {
    if (!buf || buflen < 1) return set_error(CHEM_EINVAL, "chem_prof_read: null buffer");
    std::lock_guard<std::mutex> l(g_mu);
    drain_locked();
    std::string out;
    char line[512];
    for (auto &kv : g_acc) {
        snprintf(line, sizeof(line), "%s\t%d\t%.6f\t%.6e\t%.6e\n", kv.first.c_str(), kv.second.launches, kv.second.ms,
                 kv.second.flops, kv.second.bytes);
        out += line;
    }
    if ((int64_t)out.size() + 1 > buflen) return set_error(CHEM_EINVAL, "chem_prof_read: buffer too small");
    memcpy(buf, out.c_str(), out.size() + 1);
    return CHEM_OK;
}
