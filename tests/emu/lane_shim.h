// Host build of the device arithmetic headers, for CPU tests of the lane-parallel engines: each
// lane of a warp (or block) is a host thread, __syncwarp / __syncthreads are a barrier over all of
// them, and the PTX carry-chain primitives are written with 64-bit host arithmetic (one carry flag
// per thread).  Test infrastructure only; the library never uses it.
#pragma once
#include <barrier>
#include <cstdint>
#include <cstring>
#include <thread>

#define __device__
#define __forceinline__ inline
#define __noinline__
#define __constant__ static const
#define __global__
#define FPG_PRIMITIVES_EXTERNAL 1
#define FPG_DEV static inline
#define FPG_NOINL static

static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }

namespace ptx {
static thread_local uint32_t cc;   // the carry flag of the calling lane
static inline uint32_t add_cc(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a + b;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
static inline uint32_t addc_cc(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a + b + cc;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
static inline uint32_t addc(uint32_t a, uint32_t b) { return (uint32_t)((uint64_t)a + b + cc); }
static inline uint32_t sub_cc(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a - b;
    cc = (uint32_t)(s >> 32) & 1;
    return (uint32_t)s;
}
static inline uint32_t subc_cc(uint32_t a, uint32_t b) {
    const uint64_t s = (uint64_t)a - b - cc;
    cc = (uint32_t)(s >> 32) & 1;
    return (uint32_t)s;
}
static inline uint32_t subc(uint32_t a, uint32_t b) { return (uint32_t)((uint64_t)a - b - cc); }
static inline uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
    const uint64_t s = (uint64_t)(uint32_t)((uint64_t)a * b) + c;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
static inline uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) {
    const uint64_t s = (uint64_t)(uint32_t)((uint64_t)a * b) + c + cc;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
static inline uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
    const uint64_t s = (((uint64_t)a * b) >> 32) + c;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
static inline uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) {
    const uint64_t s = (((uint64_t)a * b) >> 32) + c + cc;
    cc = (uint32_t)(s >> 32);
    return (uint32_t)s;
}
}  // namespace ptx

static inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, unsigned s) {
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> (s & 31));
}
static inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
// byte i of the result is byte (s >> 4 i) & 7 of the 8 bytes y:x
static inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
    const uint64_t v = ((uint64_t)y << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; i++) r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7))) & 0xff) << (8 * i);
    return r;
}

// kernels: one block at a time, its shared variables as statics, blockIdx per lane thread
#define __shared__ static
#define __launch_bounds__(...)
static inline uint32_t min(uint32_t a, uint32_t b) { return a < b ? a : b; }

static std::barrier<>* g_lanes = nullptr;   // all lanes of the emulated launch
static inline void __syncwarp(unsigned = 0xffffffffu) { g_lanes->arrive_and_wait(); }
static inline void __syncthreads() { g_lanes->arrive_and_wait(); }
struct LaneIdx { unsigned x; };
static thread_local LaneIdx threadIdx;
static thread_local LaneIdx blockIdx;
static const LaneIdx blockDim{128};

// __shfl_sync / __shfl_xor_sync for the quads of four lanes (mask 0xf << 4m, the only form the device
// code uses): each quad has a barrier of its own and the values pass through a shared array; any
// other mask or a source outside the quad aborts the test
#include <cstdlib>
static std::barrier<>* g_quad[256] = {};
static uint32_t g_xchg[1024];
static inline void emu_setup_quads(int n) {
    for (int i = 0; i < 256; i++) {
        delete g_quad[i];
        g_quad[i] = i < (n + 3) / 4 ? new std::barrier<>(4) : nullptr;
    }
}
static inline uint32_t emu_quad_xchg(unsigned mask, uint32_t v, unsigned src) {
    const unsigned L = threadIdx.x;
    if (mask != (0xfu << (L & 28)) || (src & 28) != (L & 28) || !g_quad[L >> 2]) std::abort();
    g_xchg[L] = v;
    g_quad[L >> 2]->arrive_and_wait();
    const uint32_t r = g_xchg[(L & ~31u) | src];
    g_quad[L >> 2]->arrive_and_wait();
    return r;
}
static inline uint32_t __shfl_sync(unsigned mask, uint32_t v, int src) {
    return emu_quad_xchg(mask, v, (unsigned)src & 31);
}
static inline int __shfl_sync(unsigned mask, int v, int src) {
    return (int)emu_quad_xchg(mask, (uint32_t)v, (unsigned)src & 31);
}
static inline uint32_t __shfl_xor_sync(unsigned mask, uint32_t v, int m) {
    return emu_quad_xchg(mask, v, (threadIdx.x & 31) ^ (unsigned)m);
}
