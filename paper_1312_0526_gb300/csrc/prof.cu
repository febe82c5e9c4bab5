// prof.cu -- launch counting and per-step CUDA-event timing.
//
// Every launcher counts the kernels it launches (hpeel_kernel_launches).
// With hpeel_profile_enable(1), each instrumented step records a pair of
// CUDA events on the stream it launches on; after the API call has
// synchronised the stream, the elapsed times are added to per-step totals
// (hpeel_profile_read).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace hp {
namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
struct Total {
    uint64_t count = 0;
    double ms = 0.0;
};
std::map<std::string, Total> g_totals;
std::vector<cudaEvent_t> g_pool;
struct Pending {
    const char *name;
    cudaEvent_t a, b;
};
thread_local std::vector<Pending> t_pending;

cudaEvent_t get_event() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

// Launches recorded into a CUDA graph while it is captured are counted when
// the graph runs, not at capture time.
thread_local int t_count_pause = 0;
LaunchCountPause::LaunchCountPause() { t_count_pause++; }
LaunchCountPause::~LaunchCountPause() { t_count_pause--; }

void smem_optin(const void *fn) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess) {
        cudaGetLastError();
        return;
    }
    // the kernel's static shared memory counts against the same limit
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) optin -= (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) ==
        cudaSuccess)
        done[{dev, fn}] = true;
    cudaGetLastError();
}

void count_launch(uint32_t kernels) {
    if (t_count_pause == 0) g_launches.fetch_add(kernels, std::memory_order_relaxed);
}

ProfScope::ProfScope(const Launch &L_, const char *name_) : L(L_), name(name_), a(nullptr) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    cudaEvent_t e = get_event();
    if (e && cudaEventRecord(e, L.stream) == cudaSuccess) a = e;
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = get_event();
    if (b && cudaEventRecord(b, L.stream) == cudaSuccess)
        t_pending.push_back({name, (cudaEvent_t)a, b});
}

void prof_flush() {
    if (t_pending.empty()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending &p : t_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Total &t = g_totals[p.name];
            t.count += 1;
            t.ms += ms;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    t_pending.clear();
}

}  // namespace hp

extern "C" {

uint64_t hpeel_kernel_launches(void) { return hp::g_launches.load(); }

void hpeel_profile_enable(int on) { hp::g_enabled.store(on ? 1 : 0); }

void hpeel_profile_reset(void) {
    std::lock_guard<std::mutex> lk(hp::g_mu);
    hp::g_totals.clear();
}

size_t hpeel_profile_read(char *buf, size_t len) {
    std::string out;
    {
        std::lock_guard<std::mutex> lk(hp::g_mu);
        char line[256];
        for (const auto &kv : hp::g_totals) {
            snprintf(line, sizeof line, "%s %llu %.6f\n", kv.first.c_str(),
                     (unsigned long long)kv.second.count, kv.second.ms);
            out += line;
        }
    }
    if (buf && len) {
        size_t k = out.size() < len - 1 ? out.size() : len - 1;
        memcpy(buf, out.data(), k);
        buf[k] = 0;
    }
    return out.size() + 1;
}

}  // extern "C"
