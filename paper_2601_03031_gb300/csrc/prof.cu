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
#include "fp.cuh"
#include "kernels.h"
#include "fq_split.cuh"

namespace fpk {
namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
struct Rec { const char* name; cudaEvent_t a, b; };
std::vector<Rec> g_open;
std::vector<cudaEvent_t> g_pool;
thread_local Rec t_cur{nullptr, nullptr, nullptr};
struct Each { const char* name; float start_ms, ms; };
std::vector<Each> g_each;    // every timed launch in issue order, until listed
cudaEvent_t g_origin = nullptr;   // the first timed launch's start since the list was last cleared

cudaEvent_t get_event() {
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e; cudaEventCreate(&e); return e;
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_enabled.load(std::memory_order_relaxed)) { t_cur.name = nullptr; return; }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        t_cur.name = nullptr;                   // launches recorded into a graph are not timed
        return;
    }
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
        float start = 0.f;
        if (!g_origin) {
            g_origin = r.a;
        } else {
            cudaEventElapsedTime(&start, g_origin, r.a);
        }
        g_each.push_back({r.name, start, ms});
        if (r.a != g_origin) g_pool.push_back(r.a);
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
// One line per timed launch, "name start_ms ms" (start relative to the first listed launch's start),
// in the order the launches were issued, for the launches that fp_profile_report has synchronised;
// cleared by a call that writes them out.
size_t fp_profile_launches(char* out, size_t cap) {
    using namespace fpk;
    std::lock_guard<std::mutex> lk(g_mu);
    std::string txt;
    char line[256];
    for (auto& e : g_each) {
        snprintf(line, sizeof line, "%s %.6f %.6f\n", e.name, (double)e.start_ms, (double)e.ms);
        txt += line;
    }
    if (out && cap) {
        size_t n = txt.size() < cap - 1 ? txt.size() : cap - 1;
        memcpy(out, txt.data(), n);
        out[n] = 0;
        g_each.clear();
        if (g_origin) g_pool.push_back(g_origin);
        g_origin = nullptr;
    }
    return txt.size() + 1;
}
}

// ---------------------------------------------------------------------------------------
// Peak of the integer multiply-add pipe: every thread runs 8 independent chains of 32-bit
// multiply-adds (alternating low and high halves, the two kinds every Montgomery product issues),
// so the pipe, not latency, bounds the rate.  ops = lanes x iterations x 8.
// ---------------------------------------------------------------------------------------
__global__ void k_imad_probe(uint32_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[8];
    for (int k = 0; k < 8; k++) a[k] = seed + threadIdx.x * 8 + k;
    const uint32_t m = 0x9e3779b9u + blockIdx.x, c = 0x7f4a7c15u;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(c));
            asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k + 1]) : "r"(m), "r"(c));
        }
    }
    uint32_t x = 0;
    for (int k = 0; k < 8; k++) x ^= a[k];
    if (x == 0x12345678u) sink[0] = x;
}

extern "C" int fp_imad_probe(double* ops_per_s, double* ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) return 2;
    const uint32_t iters = 4096, threads = 256, blocks = (uint32_t)sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    k_imad_probe<<<blocks, threads>>>(64, 1, sink);      // warm-up
    cudaEventRecord(a);
    k_imad_probe<<<blocks, threads>>>(iters, 2, sink);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b); cudaFree(sink);
    if (e != cudaSuccess) return 3;
    *ops_per_s = (double)blocks * threads * iters * 8 / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return 0;
}

// one lane, n dependent Montgomery products in Fq: the latency that bounds the lane-parallel engines
// (every round of a Miller step, cyclotomic squaring or group formula waits for one such product)
__global__ void k_fq_mul_chain(uint32_t n, uint32_t* sink) {
    if (threadIdx.x != 0) return;
    fq a, b;
    fq_from_const(a, FQ_R2);
    fq_from_const(b, FQ_R3);
    for (uint32_t i = 0; i < n; i++) a = fq_mul(a, b);
    if (a.v[0] == 0x12345678u) sink[0] = a.v[1];
}

// the same chain with each product split over the four warps of a 128-thread block (fq_split.cuh):
// the unit of the block engine's cyclotomic squarings
__global__ void __launch_bounds__(128) k_fq_mul_split_chain(uint32_t n, uint32_t* sink) {
    fq a, b;
    fq_from_const(a, FQ_R2);
    fq_from_const(b, FQ_R3);
    for (uint32_t i = 0; i < n; i++) a = fq_mul_split(a, b);
    if (a.v[0] == 0x12345678u) sink[0] = a.v[1];
}

extern "C" int fp_fq_mul_split_latency(double* ns_per_product) {
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) return 2;
    const uint32_t n = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    k_fq_mul_split_chain<<<1, 128>>>(64, sink);          // warm-up
    cudaEventRecord(a);
    k_fq_mul_split_chain<<<1, 128>>>(n, sink);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b); cudaFree(sink);
    if (e != cudaSuccess) return 3;
    *ns_per_product = (double)ms * 1e6 / n;
    return 0;
}

extern "C" int fp_fq_mul_latency(double* ns_per_product) {
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) return 2;
    const uint32_t n = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    k_fq_mul_chain<<<1, 32>>>(64, sink);                 // warm-up
    cudaEventRecord(a);
    k_fq_mul_chain<<<1, 32>>>(n, sink);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a); cudaEventDestroy(b); cudaFree(sink);
    if (e != cudaSuccess) return 3;
    *ns_per_product = (double)ms * 1e6 / n;
    return 0;
}
