// Host entry points over the lane-parallel device engines (warp12.cuh: Miller loop and final
// exponentiation on a warp or a 128-thread block; gt_exp.cuh: exponentiation in GT; group_ec.cuh: G1 scalar multiplication on an
// 8-lane group, G2 on a warp, and the parts of the split folds).  Points and field elements cross as
// canonical big-endian bytes (G1 96, G2 192, Fq12 576 in the tower order of the serialisation),
// scalars as 8 little-endian 32-bit words.  Test infrastructure only.
#include "lane_shim.h"
#include "warp12.cuh"
#include "group_ec.cuh"
#include "gt_exp.cuh"

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
g1a be_g1(const uint8_t* b) { g1a p; p.x = be_fq(b); p.y = be_fq(b + 48); return p; }
g2a be_g2(const uint8_t* b) {
    g2a p;
    p.x.c0 = be_fq(b); p.x.c1 = be_fq(b + 48); p.y.c0 = be_fq(b + 96); p.y.c1 = be_fq(b + 144);
    return p;
}
fq12 be_fq12(const uint8_t* b) {
    fq12 a;
    fq2* c[6] = {&a.c0.c0, &a.c0.c1, &a.c0.c2, &a.c1.c0, &a.c1.c1, &a.c1.c2};
    for (int t = 0; t < 6; t++) { c[t]->c0 = be_fq(b + 96 * t); c[t]->c1 = be_fq(b + 96 * t + 48); }
    return a;
}
void to_tower(fq12& f, const fq* flat) {
    fq* c = reinterpret_cast<fq*>(&f);
    for (int o = 0; o < 12; o++) c[2 * w_tower_pos(o >> 1) + (o & 1)] = flat[o];
}
// run fn on n host threads, one per lane, with a barrier over all of them
template <typename Fn>
void lanes(int n, Fn fn) {
    std::barrier<> bar(n);
    g_lanes = &bar;
    emu_setup_quads(n);
    std::vector<std::thread> th;
    for (int lane = 0; lane < n; lane++) th.emplace_back([&, lane] { threadIdx.x = lane; fn(); });
    for (auto& t : th) t.join();
}
W12 g_w;
WMill g_m;
WGt g_gt;
GEc<fq> g_g1;
GEcW g_g2;
}  // namespace

extern "C" {
// the block-split Fq product (fq_split.cuh) of 32 operand pairs (canonical integers, 12 little-endian
// words each, below p; not Montgomery form): out[w 32 + t] = x_t y_t 2^-384 mod p as warp w's lane t
// holds it
void emu_fq_mul_split(const uint32_t* x, const uint32_t* y, uint32_t* out) {
    lanes(128, [&] {
        const int L = (int)threadIdx.x, t = L & 31;
        fq a, b;
        for (int j = 0; j < 12; j++) { a.v[j] = x[12 * t + j]; b.v[j] = y[12 * t + j]; }
        const fq r = fq_mul_split(a, b);
        for (int j = 0; j < 12; j++) out[12 * L + j] = r.v[j];
    });
}
void emu_miller(int nw, const uint8_t* p, const uint8_t* q, uint8_t* out) {
    const g1a P = be_g1(p);
    const g2a Q = be_g2(q);
    if (nw == 4) lanes(128, [&] { w_miller<4>(g_m, P, Q); });
    else lanes(32, [&] { w_miller<1>(g_m, P, Q); });
    fq12 f;
    to_tower(f, g_m.f);
    fq12_to_be(out, f);
}
void emu_final_exp(int nw, const uint8_t* f_be, uint8_t* out) {
    const fq12 in = be_fq12(f_be);
    if (nw == 4) lanes(128, [&] { w_from_tower<4>(g_w.s[0], in); w_final_exp<4>(g_w); });
    else lanes(32, [&] { w_from_tower<1>(g_w.s[0], in); w_final_exp<1>(g_w); });
    fq12 r;
    to_tower(r, g_w.s[2]);
    fq12_to_be(out, r);
}
// bits [i0, i0 + n) of the Frobenius split of g^c (g in GT, c < r as 8 little-endian words)
void emu_gt_pow(int nw, const uint8_t* g_be, const uint32_t* c, int i0, int n, uint8_t* out) {
    const fq12 in = be_fq12(g_be);
    if (nw == 4)
        lanes(128, [&] { w_from_tower<4>(g_gt.w.s[0], in); w_gt_pow_bits<4>(g_gt, g_gt.w.s[1], g_gt.w.s[0], c, i0, n); });
    else
        lanes(32, [&] { w_from_tower<1>(g_gt.w.s[0], in); w_gt_pow_bits<1>(g_gt, g_gt.w.s[1], g_gt.w.s[0], c, i0, n); });
    fq12 r;
    to_tower(r, g_gt.w.s[1]);
    fq12_to_be(out, r);
}
// k P on an 8-lane group: np = 1 the whole multiplication, else part `part` of np on the base P
void emu_g1_mul(const uint8_t* p, const uint32_t* k, int np, int part, uint8_t* out) {
    const g1a P = be_g1(p);
    GPt<fq> r;
    lanes(8, [&] {
        const int L = (int)threadIdx.x;
        const GPt<fq> x = np == 4 ? gec_g1_mul_part<4>(g_g1, L, P, k, part)
                          : np == 2 ? gec_g1_mul_part<2>(g_g1, L, P, k, part)
                                    : gec_g1_mul_proj_w2(g_g1, L, P, k);
        if (L == 0) r = x;
    });
    g1a a;
    gec_to_affine(a.x, a.y, r);
    g1a_to_be(out, a);
}
void emu_g1_dbl_n(const uint8_t* p, int n, uint8_t* out) {
    const g1a P = be_g1(p);
    GPt<fq> r;
    lanes(8, [&] {
        const GPt<fq> x = gec_g1_dbl_n(g_g1, (int)threadIdx.x, gec_from_affine_or_inf(P.x, P.y), n);
        if (threadIdx.x == 0) r = x;
    });
    g1a a;
    gec_to_affine(a.x, a.y, r);
    g1a_to_be(out, a);
}
void emu_g2_mul(const uint8_t* q, const uint32_t* k, int np, int part, uint8_t* out) {
    const g2a Q = be_g2(q);
    GPt<fq2> r;
    lanes(32, [&] {
        const int L = (int)threadIdx.x;
        const GPt<fq2> x = np == 4 ? gecw_g2_mul_part<4>(g_g2, L, Q, k, part)
                           : np == 2 ? gecw_g2_mul_part<2>(g_g2, L, Q, k, part)
                                     : gecw_g2_mul_proj(g_g2, L, Q, k);
        if (L == 0) r = x;
    });
    g2a a;
    gec_to_affine(a.x, a.y, r);
    g2a_to_be(out, a);
}
// k P through the fixed-base comb of Step 1's folds: the chain 2^i P (i < 128) and the sum of one
// entry per window on an 8-lane group, the 64 window tables (gpt_g1_comb_table) on one thread
void emu_g1_comb(const uint8_t* p, const uint32_t* k, uint8_t* out) {
    const g1a P = be_g1(p);
    static GPt<fq> chain[128], tab[64 * 16];
    GPt<fq> r;
    lanes(8, [&] {
        const int L = (int)threadIdx.x;
        GPt<fq> acc = gec_from_affine_or_inf(P.x, P.y);
        for (int i = 0; i < 128; i++) {
            if (i) acc = gec_dbl(g_g1, L, acc);
            if (L == 0) chain[i] = acc;
            __syncwarp();
        }
        if (L == 0)
            for (int w = 0; w < 64; w++) gpt_g1_comb_table(chain[2 * w], chain[2 * w + 1], tab + 16 * w);
        __syncwarp();
        uint32_t k1[5], k0[4];
        div_by_const<4, 5>(k1, k0, k, GLV_D, GLV_BARRETT);
        GPt<fq> s = gec_identity<fq>();
        for (int w = 0; w < 64; w++) s = gec_add(g_g1, L, s, tab[16 * w + glv_window(k0, k1, w)]);
        // to affine as k_fold_c does (the two quads of the group), and through Jacobian coordinates as
        // the quad conversion kernels do; a disagreement leaves the output zero
        g1a a, b;
        gec_to_affine_quad(a.x, a.y, s);
        jac_to_affine_quad(b.x, b.y, proj_to_jac(s));
        if (L == 0) {
            r = s;
            if (fq_eq(a.x, b.x) && fq_eq(a.y, b.y)) g1a_to_be(out, a);
            else memset(out, 0, 96);
        }
    });
}
// k Q through the comb on G2: the chain 2^i Q (i < 64) on one warp, the 64 position tables
// (gpt_g2_comb_table) on one thread, the sum of one entry per position on an 8-lane group
void emu_g2_comb(const uint8_t* q, const uint32_t* k, uint8_t* out) {
    const g2a Q = be_g2(q);
    static GPt<fq2> chain[64], tab[64 * 16];
    GPt<fq2> r;
    lanes(32, [&] {
        const int L = (int)threadIdx.x;
        GPt<fq2> acc = gec_from_affine_or_inf(Q.x, Q.y);
        for (int i = 0; i < 64; i++) {
            if (i) acc = gecw_dbl(g_g2, L, acc);
            if (L == 0) chain[i] = acc;
            __syncwarp();
        }
        if (L == 0)
            for (int i = 0; i < 64; i++) gpt_g2_comb_table(chain[i], tab + 16 * i);
        __syncwarp();
    });
    // the sum on an 8-lane group with Fq2 products on each lane (the engine of k_fold_c, k_w_comb)
    static GEcs<fq2> e2;
    lanes(8, [&] {
        const int L = (int)threadIdx.x;
        uint32_t d[4][2];
        gls_digits(d, k);
        GPt<fq2> s = gec_identity<fq2>();
        for (int i = 0; i < 64; i++) s = gec_add(e2, L, s, tab[16 * i + gls_position(d, i)]);
        g2a a, b;
        gec_to_affine_quad(a.x, a.y, s);
        jac_to_affine_quad(b.x, b.y, proj_to_jac(s));
        if (L == 0) {
            r = s;
            if (fq2_eq(a.x, b.x) && fq2_eq(a.y, b.y)) g2a_to_be(out, a);
            else memset(out, 0, 192);
        }
    });
}
void emu_g2_dbl_n(const uint8_t* q, int n, uint8_t* out) {
    const g2a Q = be_g2(q);
    GPt<fq2> r;
    lanes(32, [&] {
        const GPt<fq2> x = gecw_g2_dbl_n(g_g2, (int)threadIdx.x, gec_from_affine_or_inf(Q.x, Q.y), n);
        if (threadIdx.x == 0) r = x;
    });
    g2a a;
    gec_to_affine(a.x, a.y, r);
    g2a_to_be(out, a);
}
}  // extern "C"
