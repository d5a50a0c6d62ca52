// Host run of the look-ahead round kernels (lookahead.cuh) on a small state, one 128-thread block
// at a time, with the reductions between them done by the device helpers on the host.  Inputs and
// outputs are canonical big-endian bytes (G1 96, G2 192, Fr 32), the challenge as 32 bytes.  Writes
// the round record L.T (576) L.1 (96) R.T (576) R.1 (96) of every block.  Test infrastructure only.
#include "lane_shim.h"
#include "lookahead.cuh"

#include <vector>

namespace {
fq be_fq(const uint8_t* b) {
    fq a;
    for (int j = 0; j < 12; j++) {
        const uint8_t* p = b + 44 - 4 * j;
        a.v[j] = ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | p[3];
    }
    return fq_to_mont(a);
}
fr be_fr(const uint8_t* b) {
    fr a;
    for (int j = 0; j < 8; j++) {
        const uint8_t* p = b + 28 - 4 * j;
        a.v[j] = ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | p[3];
    }
    return fr_to_mont(a);
}
template <typename Fn>
void grid(uint64_t nblocks, Fn fn) {
    for (uint64_t bx = 0; bx < nblocks; bx++) {
        std::barrier<> bar(128);
        g_lanes = &bar;
        std::vector<std::thread> th;
        for (int lane = 0; lane < 128; lane++)
            th.emplace_back([&, lane] { threadIdx.x = lane; blockIdx.x = (unsigned)bx; fn(); });
        for (auto& t : th) t.join();
    }
}
}  // namespace

// K blocks of stride R whose live state has length 2h = 4 h2 <= R: A (K R G1), v (K R G2), b (K R Fr);
// the support of block k's b follows from (k0, bsz) as in the protocol; x (K challenges)
extern "C" void emu_la_round(uint32_t K, uint32_t R, uint32_t h2, uint32_t k0, uint32_t bsz, const uint8_t* A_be,
                             const uint8_t* v_be, const uint8_t* b_be, const uint8_t* x_be, uint8_t* rec_out) {
    using namespace fpk;
    const uint32_t h = 2 * h2;
    std::vector<g1a> A(K * R);
    std::vector<g2a> v(K * R);
    std::vector<fr> bv(K * R), xm(K), xim(K);
    for (uint32_t t = 0; t < K * R; t++) {
        const uint8_t* a = A_be + 96 * t;
        bool zero = true;
        for (int j = 0; j < 96; j++) zero = zero && !a[j];
        if (zero) { fq_zero(A[t].x); fq_zero(A[t].y); } else { A[t].x = be_fq(a); A[t].y = be_fq(a + 48); }
        const uint8_t* q = v_be + 192 * t;
        v[t].x.c0 = be_fq(q); v[t].x.c1 = be_fq(q + 48); v[t].y.c0 = be_fq(q + 96); v[t].y.c1 = be_fq(q + 144);
        bv[t] = be_fr(b_be + 32 * t);
    }
    for (uint32_t k = 0; k < K; k++) { xm[k] = be_fr(x_be + 32 * k); xim[k] = fr_inv(xm[k]); }
    // pairings: Miller loops, products per class, final exponentiations
    std::vector<fq12> ml((size_t)K * 8 * h2), fe((size_t)K * 8);
    grid((uint64_t)K * 8 * h2, [&] { k_la_miller_c(A.data(), v.data(), R, h2, ml.data()); });
    for (uint32_t c = 0; c < K * 8; c++) {                 // (the engines' final exponentiation is
        fq12 prod = ml[(size_t)c * h2];                      // checked on its own elsewhere)
        for (uint32_t i = 1; i < h2; i++) prod = fq12_mul(prod, ml[(size_t)c * h2 + i]);
        fe[c] = final_exp(prod);
    }
    // the six G1 sums
    const uint32_t cmax = min(bsz, 2 * h);
    std::vector<g1j> terms((size_t)K * 6 * 2 * h);
    std::memset(terms.data(), 0, terms.size() * sizeof(g1j));
    grid(((uint64_t)2 * K * cmax + 15) / 16, [&] {
        k_la_sparse(A.data(), bv.data(), k0, K, R, h2, bsz, cmax, terms.data());
    });
    std::vector<g1a> acc((size_t)K * 6);
    for (uint32_t c = 0; c < K * 6; c++) {
        g1j s = terms[(size_t)c * 2 * h];
        for (uint32_t p = 1; p < 2 * h; p++) s = jac_add(s, terms[(size_t)c * 2 * h + p]);
        acc[c] = g1_affine(s);
    }
    // the shifted bases, then after the challenge the parts and the record
    std::vector<fq12> gpre((size_t)K * 12), pwp((size_t)K * 16);
    std::vector<g1a> acc2((size_t)K * 12);
    grid((uint64_t)K * 4, [&] { k_la_gt_pre(fe.data(), gpre.data()); });
    grid(((uint64_t)4 * K + 15) / 16, [&] { k_la_g1_pre(acc.data(), K, acc2.data()); });
    const size_t GT = 576, G1 = 96, stride_side = GT + G1, stride_k = 2 * (GT + G1);
    grid((uint64_t)K * 16, [&] { k_la_gt_c(fe.data(), gpre.data(), xm.data(), xim.data(), pwp.data()); });
    grid((uint64_t)K * 2, [&] { k_la_gt_out(fe.data(), pwp.data(), rec_out, stride_k, stride_side); });
    grid((uint64_t)K, [&] {
        k_la_g1_out(acc.data(), acc2.data(), xm.data(), xim.data(), K, rec_out + GT, stride_k, stride_side);
    });
}
