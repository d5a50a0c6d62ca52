// Host build of the streaming SHA-256 of the CUDA path (sha256.cuh) for a CPU test: the message is
// fed in pieces at the given cut points, so that every buffering path (whole blocks in place, word
// moves, byte moves) runs.  Test infrastructure only.
#include "lane_shim.h"
#include "sha256.cuh"

extern "C" {
void emu_sha256_pieces(const uint8_t* data, uint32_t n, const uint32_t* cuts, int ncuts, uint8_t* out) {
    sha256_ctx c;
    sha256_init(c);
    uint32_t at = 0;
    for (int i = 0; i <= ncuts; i++) {
        const uint32_t end = i < ncuts ? cuts[i] : n;
        sha256_update(c, data + at, end - at);
        at = end;
    }
    sha256_final(c, out);
}
}
