// Launch counting and optional per-kernel CUDA-event timing (host side only).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/flexproofs.h"
#include "kernels.h"

namespace fpk {
namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
struct Rec { const char* name; cudaEvent_t a, b; };
std::vector<Rec> g_open;
std::vector<cudaEvent_t> g_pool;
thread_local Rec t_cur{nullptr, nullptr, nullptr};

cudaEvent_t get_event() {
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e; cudaEventCreate(&e); return e;
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) { t_cur.name = nullptr; return; }
    std::lock_guard<std::mutex> lk(g_mu);
    t_cur = Rec{name, get_event(), get_event()};
    cudaEventRecord(t_cur.a, s);
}
void prof_end(cudaStream_t s) {
    if (!t_cur.name) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(t_cur.b, s);
    g_open.push_back(t_cur);
    t_cur.name = nullptr;
}
}  // namespace fpk

extern "C" {
uint64_t fp_launch_count(void) { return fpk::g_launches.load(); }
void fp_profile_enable(int on) { fpk::g_enabled.store(on ? 1 : 0); }
// Synchronises the recorded events and writes one line per kernel name,
// "name launches total_ms", then clears the records.  Returns the bytes needed.
size_t fp_profile_report(char* out, size_t cap) {
    using namespace fpk;
    std::lock_guard<std::mutex> lk(g_mu);
    static std::map<std::string, std::pair<uint64_t, double>> agg;   // kept until a report is written out
    for (auto& r : g_open) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto& e = agg[r.name];
        e.first++;
        e.second += ms;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_open.clear();
    std::string txt;
    char line[256];
    for (auto& kv : agg) {
        snprintf(line, sizeof line, "%s %llu %.6f\n", kv.first.c_str(), (unsigned long long)kv.second.first,
                 kv.second.second);
        txt += line;
    }
    if (out && cap) {
        size_t n = txt.size() < cap - 1 ? txt.size() : cap - 1;
        memcpy(out, txt.data(), n);
        out[n] = 0;
        agg.clear();
    }
    return txt.size() + 1;
}
}
