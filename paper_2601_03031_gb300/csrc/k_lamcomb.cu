// Commit's row commitments C_j = sum_a m[j M + a] Lambda_a by fixed-base combs of the setup's bases.
//
// The bases Lambda_a (a < M) are fixed by the setup, so their multiples can be tabulated once: with
// the GLV split k = k0 + k1 |x|^2 (k0, k1 < 2^128; phi(x, y) = (omega x, y) acts as -|x|^2, so
// k P = k0 P + k1 (-phi(P)), as in msm.cu) and 4-bit windows w < 32 of both halves,
//     T[a][w][d0 + 16 d1] = d0 16^w Lambda_a + d1 16^w (-phi(Lambda_a))      (d0, d1 < 16, affine)
// and k Lambda_a = sum_w T[a][w][nibble_w(k0) + 16 nibble_w(k1)]: 32 mixed additions per term and no
// bucket reduction or window combination, at the price of 256 entries (24 KB) per base and window.
// The tables are built at setup (k_lamc_chain: 16^w Lambda_a; k_lamc_row0: d B and -phi(d B);
// k_lamc_rows: the other rows), the commit sums them (k_lamc_sum: a thread per (row, base, quarter
// of the windows)), and the partial sums per row are reduced pairwise and by block trees.
#include "k_common.cuh"

namespace fpk {

constexpr int LAMC_W = 32, LAMC_E = 256, LAMC_Q = 4;   // windows, entries per window, window quarters

size_t lam_comb_bytes(uint32_t M) { return (size_t)M * LAMC_W * LAMC_E * G1A_BYTES; }
size_t lam_comb_scratch_bytes(uint32_t M) { return (size_t)M * LAMC_W * G1J_BYTES; }

// -phi(P) = (omega x, -y) of an affine P (the identity stays the identity)
FPG_DEV g1a g1a_mphi(const g1a& P) {
    if (g1a_is_inf(P)) return P;
    fq om;
    fq_from_const(om, GLV_OMEGA);
    return {fq_mul(P.x, om), fq_neg(P.y)};
}

// affine forms of n <= 16 Jacobian points (none the identity) with one inversion (Montgomery's trick)
FPG_DEV void g1j_batch_affine(const g1j* p, int n, g1a* out) {
    fq pre[16];
    pre[0] = p[0].Z;
    for (int i = 1; i < n; i++) pre[i] = fq_mul(pre[i - 1], p[i].Z);
    fq inv = fq_inv(pre[n - 1]);
    for (int i = n - 1; i >= 0; i--) {
        const fq zi = i ? fq_mul(inv, pre[i - 1]) : inv;
        if (i) inv = fq_mul(inv, p[i].Z);
        const fq zi2 = fq_sqr(zi);
        out[i].x = fq_mul(p[i].X, zi2);
        out[i].y = fq_mul(p[i].Y, fq_mul(zi2, zi));
    }
}

// chain[a 32 + w] = 16^w Lambda_a (Jacobian), one thread per base
__global__ void __launch_bounds__(64) k_lamc_chain(const g1a* bases, uint32_t M, g1j* chain) {
    const uint64_t a = gtid();
    if (a >= M) return;
    g1j acc = g1_from_affine(bases[a]);
    for (int w = 0; w < LAMC_W; w++) {
        if (w)
            for (int i = 0; i < 4; i++) acc = jac_dbl(acc);
        chain[a * LAMC_W + w] = acc;
    }
}

// row 0 and column 0 of table (a, w): d B and -phi(d B) for d < 16, B = 16^w Lambda_a; one thread
// per table.  A base that is the identity gives the identity everywhere.
__global__ void __launch_bounds__(64) k_lamc_row0(const g1j* chain, uint32_t M, g1a* tab) {
    const uint64_t t = gtid();
    if (t >= (uint64_t)M * LAMC_W) return;
    g1a* T = tab + t * LAMC_E;
    g1a zero;
    fq_zero(zero.x);
    fq_zero(zero.y);
    T[0] = zero;
    const g1j B = chain[t];
    if (jac_is_inf(B)) {
        for (int e = 1; e < LAMC_E; e++) T[e] = zero;
        return;
    }
    g1j m[15];
    m[0] = B;
    m[1] = jac_dbl(B);
    for (int d = 2; d < 15; d++) m[d] = jac_add(m[d - 1], B);
    g1a aff[15];
    g1j_batch_affine(m, 15, aff);
    for (int d = 1; d < 16; d++) {
        T[d] = aff[d - 1];
        T[16 * d] = g1a_mphi(aff[d - 1]);
    }
}

// row d1 >= 1 of table (a, w): d0 B + d1 (-phi(B)) for d0 = 1 .. 15, from T[16 d1] and T[1] = B;
// one thread per row
__global__ void __launch_bounds__(64) k_lamc_rows(uint32_t M, g1a* tab) {
    const uint64_t u = gtid();
    if (u >= (uint64_t)M * LAMC_W * 15) return;
    const uint64_t t = u / 15;
    const int d1 = 1 + (int)(u % 15);
    g1a* T = tab + t * LAMC_E;
    const g1a B = T[1], Q = T[16 * d1];
    if (g1a_is_inf(B)) return;                               // the whole table is the identity
    g1j m[15];
    g1j acc = g1_from_affine(Q);
    for (int d0 = 1; d0 < 16; d0++) {
        acc = jac_madd(acc, B.x, B.y);                         // d0 B + Q; never the identity or a doubling
        m[d0 - 1] = acc;
    }
    g1a aff[15];
    g1j_batch_affine(m, 15, aff);
    for (int d0 = 1; d0 < 16; d0++) T[16 * d1 + d0] = aff[d0 - 1];
}

void lam_comb_tables(const void* bases_g1a, uint32_t M, void* scratch, void* tab, cudaStream_t s) {
    FP_KERNEL("k_lamc_chain", s, k_lamc_chain<<<grid_for(M, 64), 64, 0, s>>>((const g1a*)bases_g1a, M, (g1j*)scratch));
    FP_KERNEL("k_lamc_row0", s, k_lamc_row0<<<grid_for((uint64_t)M * LAMC_W, 64), 64, 0, s>>>((const g1j*)scratch, M,
                                                                                              (g1a*)tab));
    FP_KERNEL("k_lamc_rows", s, k_lamc_rows<<<grid_for((uint64_t)M * LAMC_W * 15, 64), 64, 0, s>>>(M, (g1a*)tab));
}

// partial[(j M + a) Q + q] = sum over the windows w in [8 q, 8 q + 8) of T[a][w][digit_w(m[j M + a])],
// one thread per (j, a, q); an entry with digit 0 is the identity and is skipped
__global__ void __launch_bounds__(128) k_lamc_sum(const g1a* tab, const fr* m_canon, uint32_t R, uint32_t M,
                                                  g1j* partial) {
    const uint64_t u = gtid();
    if (u >= (uint64_t)R * M * LAMC_Q) return;
    const uint64_t ja = u / LAMC_Q;
    const int q = (int)(u % LAMC_Q);
    const uint32_t a = (uint32_t)(ja % M);
    uint32_t k1[5], k0[4];
    div_by_const<4, 5>(k1, k0, m_canon[ja].v, GLV_D, GLV_BARRETT);
    const g1a* T = tab + (uint64_t)a * LAMC_W * LAMC_E;
    g1j acc;
    jac_set_inf(acc);
    for (int w = 8 * q; w < 8 * q + 8; w++) {
        const int e = (int)(((k0[w >> 3] >> (4 * (w & 7))) & 15) | (((k1[w >> 3] >> (4 * (w & 7))) & 15) << 4));
        if (e) acc = g1_madd(acc, T[(uint64_t)w * LAMC_E + e]);
    }
    partial[u] = acc;
}

void lam_comb_partials(const void* tab, const void* m_canon, uint32_t R, uint32_t M, void* partial, cudaStream_t s) {
    FP_KERNEL("k_lamc_sum", s, k_lamc_sum<<<grid_for((uint64_t)R * M * LAMC_Q, 128), 128, 0, s>>>(
                                   (const g1a*)tab, (const fr*)m_canon, R, M, (g1j*)partial));
}
uint32_t lam_comb_parts() { return LAMC_Q; }

}  // namespace fpk
