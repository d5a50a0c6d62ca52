// Host build of the field inverse of the CUDA path (mp::inv_ds in fp.cuh, batched division steps) for
// a CPU test: plain canonical integers in and out, little-endian 32-bit words.
#include "lane_shim.h"
#include "fp.cuh"

#include <vector>

extern "C" {
void emu_inv_fq(const uint32_t* x, uint32_t* r) { mp::inv_ds<12>(r, x, FQ_P, FQ_PINV); }
void emu_inv_fr(const uint32_t* x, uint32_t* r) { mp::inv_ds<8>(r, x, FR_P, FR_PINV); }
// the quad inverse (mp::inv_ds_quad) on four host threads as the lanes of one quad: lane q starts
// from x + q n (only lane 0's value is inverted), r + q n receives lane q's result
static void quad(const uint32_t* x, uint32_t* r, int n, void (*fn)(const uint32_t*, uint32_t*), int lanes = 4) {
    std::barrier<> bar(lanes);
    g_lanes = &bar;
    emu_setup_quads(lanes);
    std::vector<std::thread> th;
    for (int lane = 0; lane < lanes; lane++)
        th.emplace_back([=] {
            threadIdx.x = (unsigned)lane;
            fn(x + lane * n, r + lane * n);
        });
    for (auto& t : th) t.join();
}
void emu_inv_fq_quad(const uint32_t* x, uint32_t* r) {
    quad(x, r, 12, [](const uint32_t* a, uint32_t* b) { mp::inv_ds_quad<12>(b, a, FQ_P, FQ_PINV); });
}
void emu_inv_fr_quad(const uint32_t* x, uint32_t* r) {
    quad(x, r, 8, [](const uint32_t* a, uint32_t* b) { mp::inv_ds_quad<8>(b, a, FR_P, FR_PINV); });
}
// a whole warp: eight quads inverting eight values at once (each quad runs its own number of batches)
void emu_inv_fq_warp(const uint32_t* x, uint32_t* r) {
    quad(x, r, 12, [](const uint32_t* a, uint32_t* b) { mp::inv_ds_quad<12>(b, a, FQ_P, FQ_PINV); }, 32);
}
}
