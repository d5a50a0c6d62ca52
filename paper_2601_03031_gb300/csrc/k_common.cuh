// Shared helpers of the kernel translation units.
#pragma once
#include "kernels.h"
#include "pairing.cuh"
#include "sha256.cuh"

namespace fpk {

constexpr int TPB = 128;                    // threads per block of the per-element kernels
inline unsigned grid_for(uint64_t n, int tpb = TPB) { return (unsigned)((n + tpb - 1) / tpb); }

FPG_DEV uint64_t gtid() { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }

FPG_DEV void put_be32(uint8_t* o, uint32_t x) {
    o[0] = (uint8_t)(x >> 24); o[1] = (uint8_t)(x >> 16); o[2] = (uint8_t)(x >> 8); o[3] = (uint8_t)x;
}
FPG_DEV void put_be64(uint8_t* o, uint64_t x) {
    for (int i = 0; i < 8; i++) o[i] = (uint8_t)(x >> (56 - 8 * i));
}
// canonical little-endian words of a Montgomery Fr residue (scalar for double-and-add)
FPG_DEV void fr_canon_words(uint32_t* k, const fr& a) {
    fr c = fr_from_mont(a);
#pragma unroll
    for (int j = 0; j < 8; j++) k[j] = c.v[j];
}
FPG_DEV fr fr_load(const void* base, uint64_t i) { return reinterpret_cast<const fr*>(base)[i]; }

// offset of level l in a stored binary tree with `leaves` leaves (leaves first, then parents)
FPG_DEV uint64_t tree_off(uint64_t leaves, int l) { return 2 * leaves - 2 * (leaves >> l); }

}  // namespace fpk
