// Shapes of the batched G1 multi-scalar multiplication (host and device).
#pragma once
#include <cstdint>

namespace fpk {

struct MsmShape {
    uint64_t n;         // terms per batch
    uint32_t nbatch;    // independent sums
    uint64_t npts;      // term i of batch j uses base (j n + i) mod npts
    int c, W;           // window bits, windows per GLV half
    uint32_t B;         // buckets per window = 2^(c-1)
    uint32_t S;         // segments per window in the bucket reduction
    __host__ __device__ uint64_t nkeys() const { return (uint64_t)nbatch * W * B; }
    __host__ __device__ uint64_t nsegs() const { return (uint64_t)nbatch * W * S; }
    __host__ __device__ uint64_t entries_max() const { return 2ull * n * nbatch * W; }
};

}  // namespace fpk
