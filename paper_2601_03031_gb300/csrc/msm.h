// Shape of the batched multi-scalar multiplications (host and device).
//
// Each scalar is reduced mod r and split by the endomorphism: on G1 (GLV) into two parts below
// 2^128, on G2 (GLS) into four parts below 2^64.  The bits of a part plus one spare bit for the
// carry of the signed digits (129 or 65) are cut into W windows of nearly equal width: the first n_hi windows have c bits, the others c - 1, so no window is left with a few
// high bits whose digits crowd into a few buckets.  Window w has B_w = 2^(c_w - 1) buckets, and
// the buckets of one batch are laid out window after window (KW keys per batch).
#pragma once
#include <cstdint>

namespace fpk {

struct MsmShape {
    uint64_t n;         // terms per batch
    uint32_t nbatch;    // independent sums
    uint64_t npts;      // term i of batch j uses base (j n + i) mod npts
    int H;              // endomorphism parts per scalar (2 on G1, 4 on G2): bases table [H][npts]
    int c, W, n_hi;     // widest window, windows per part, windows of width c
    uint32_t KW;        // buckets per batch, all windows
    uint32_t S;         // segments per window in the bucket reduction
    uint32_t T;         // sorted bucket entries per chunk of the bucket pass (one thread each)
    __host__ __device__ int bits(int w) const { return w < n_hi ? c : c - 1; }
    __host__ __device__ int lo(int w) const { return w <= n_hi ? w * c : n_hi * c + (w - n_hi) * (c - 1); }
    __host__ __device__ uint32_t buckets(int w) const { return 1u << (bits(w) - 1); }
    __host__ __device__ uint32_t off(int w) const {
        return w <= n_hi ? (uint32_t)w << (c - 1) : ((uint32_t)n_hi << (c - 1)) + ((uint32_t)(w - n_hi) << (c - 2));
    }
    __host__ __device__ uint64_t nkeys() const { return (uint64_t)nbatch * KW; }
    __host__ __device__ uint64_t nsegs() const { return (uint64_t)nbatch * W * S; }
    __host__ __device__ uint64_t entries_max() const { return (uint64_t)H * n * nbatch * W; }
};

}  // namespace fpk
