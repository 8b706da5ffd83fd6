// Optional per-kernel timing: when enabled, every kernel launch of the
// library is bracketed by CUDA events recorded on its own launch stream.
// svlf_profile_report() waits for the device, sums the elapsed times per
// kernel name and clears the record.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "svlf_internal.cuh"

namespace svlf {

namespace {
struct Rec {
    const char *name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_pending;
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_open;  // begun, not yet ended (one per stream at most in practice)

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void prof_begin(const char *name, cudaStream_t s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{name, get_event(), get_event()};
    cudaEventRecord(r.a, s);
    g_open.push_back(r);
}

void prof_end(cudaStream_t s) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_open.empty()) return;
    Rec r = g_open.back();
    g_open.pop_back();
    cudaEventRecord(r.b, s);
    g_pending.push_back(r);
}

}  // namespace svlf

using namespace svlf;

extern "C" int svlf_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return SVLF_OK;
}

extern "C" int svlf_profile_report(svlf_kernel_stat *out, int max_entries, int *n_entries) {
    if (!n_entries || (max_entries > 0 && !out)) return SVLF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return SVLF_ERR_CUDA;
    std::vector<svlf_kernel_stat> acc;
    for (const Rec &r : g_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        bool found = false;
        for (auto &s : acc)
            if (std::strncmp(s.name, r.name, sizeof(s.name)) == 0) {
                s.launches += 1;
                s.total_ms += ms;
                found = true;
                break;
            }
        if (!found) {
            svlf_kernel_stat s;
            std::memset(&s, 0, sizeof(s));
            std::strncpy(s.name, r.name, sizeof(s.name) - 1);
            s.launches = 1;
            s.total_ms = ms;
            acc.push_back(s);
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
    const int n = (int)acc.size();
    for (int i = 0; i < n && i < max_entries; ++i) out[i] = acc[i];
    *n_entries = n;
    return SVLF_OK;
}
