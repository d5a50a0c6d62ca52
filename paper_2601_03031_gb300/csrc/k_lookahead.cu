// Launchers of the look-ahead round kernels (lookahead.cuh).
#include "k_common.cuh"
#include "lookahead.cuh"

namespace fpk {

void la_miller(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h2, void* out, cudaStream_t s) {
    const uint64_t n = (uint64_t)K * 8 * h2;
    if (!n) return;
    FP_KERNEL("k_la_miller_c", s, k_la_miller_c<<<(unsigned)n, 128, 0, s>>>((const g1a*)A, (const g2a*)v, R, h2,
                                                                           (fq12*)out));
}
void la_sparse(const void* A, const void* bvec, uint32_t k0, uint32_t K, uint32_t R, uint32_t h2, uint32_t b,
               void* out, cudaStream_t s) {
    const uint32_t cmax = std::min(b, 4 * h2);     // out (K 6 4 h2 Jacobian) zeroed by the caller
    FP_KERNEL("k_la_sparse", s, k_la_sparse<<<(unsigned)(((uint64_t)2 * K * cmax + 15) / 16), 128, 0, s>>>(
                                    (const g1a*)A, (const fr*)bvec, k0, K, R, h2, b, cmax, (g1j*)out));
}
void la_pre(const void* fe, const void* acc, uint32_t K, void* gpre, void* acc2, cudaStream_t s) {
    FP_KERNEL("k_la_gt_pre", s, k_la_gt_pre<<<4 * K, 128, 0, s>>>((const fq12*)fe, (fq12*)gpre));
    FP_KERNEL("k_la_g1_pre", s, k_la_g1_pre<<<(4 * K + 15) / 16, 128, 0, s>>>((const g1a*)acc, K, (g1a*)acc2));
}
void la_gt(const void* fe, const void* gpre, const void* x_mont, const void* xinv_mont, uint32_t K, void* pwp,
           cudaStream_t s) {
    FP_KERNEL("k_la_gt_c", s, k_la_gt_c<<<16 * K, 128, 0, s>>>((const fq12*)fe, (const fq12*)gpre,
                                                              (const fr*)x_mont, (const fr*)xinv_mont, (fq12*)pwp));
}
void la_out(const void* fe, const void* pwp, const void* acc, const void* acc2, const void* x_mont,
            const void* xinv_mont, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s) {
    uint8_t* rec = (uint8_t*)blocks + (size_t)(j - 1) * ROUND_BYTES;
    FP_KERNEL("k_la_gt_out", s, k_la_gt_out<<<2 * K, 128, 0, s>>>((const fq12*)fe, (const fq12*)pwp, rec, bopen_len,
                                                                 GT_SER + G1_SER));
    FP_KERNEL("k_la_g1_out", s, k_la_g1_out<<<K, 128, 0, s>>>((const g1a*)acc, (const g1a*)acc2, (const fr*)x_mont,
                                                             (const fr*)xinv_mont, K, rec + GT_SER, bopen_len,
                                                             GT_SER + G1_SER));
}

}  // namespace fpk
