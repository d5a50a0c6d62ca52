// Host build of the field inverse of the CUDA path (mp::inv_ds in fp.cuh, batched division steps) for
// a CPU test: plain canonical integers in and out, little-endian 32-bit words.
#include "lane_shim.h"
#include "fp.cuh"

extern "C" {
void emu_inv_fq(const uint32_t* x, uint32_t* r) { mp::inv_ds<12>(r, x, FQ_P, FQ_PINV); }
void emu_inv_fr(const uint32_t* x, uint32_t* r) { mp::inv_ds<8>(r, x, FR_P, FR_PINV); }
}
