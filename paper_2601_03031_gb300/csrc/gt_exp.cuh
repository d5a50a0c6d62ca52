// Exponentiation in GT (the order-r subgroup of the cyclotomic subgroup of Fq12^*) by a scalar
// c < r on the lane-parallel Fq12 engine (warp12.cuh).  On elements of order r the p-power
// Frobenius is the exponentiation by p = x (mod r), x = -|x| the curve parameter, so
// g^{|x|^i} = conj^i(pi^i(g)) (the inverse of a unitary element is its conjugate).  With c split
// into base-|x| digits as on G2 (GLS, group_ec.cuh: c = sum_i d_i |x|^i, d_i < 2^64),
// g^c = prod_i B_i^{d_i}, B_i = conj^i(pi^i(g)): a joint square-and-multiply of 64 steps over the
// 16 subset products of the B_i, instead of 255 squarings.  A range of digit bits [i0, i0 + n) on
// the base g^{2^i0} gives one part of such a split chain.
#pragma once
#include "group_ec.cuh"
#include "warp12.cuh"

struct WGt {
    W12 w;
    fq tab[16][12];     // subset products of the B_i (flat order)
};

template <int NW>
FPG_DEV void w_set_one(fq* a) {
    const int L = w_lane<NW>();
    wsync<NW>();
    if (L < 12) {
        fq z;
        fq_zero(z);
        fq one;
        fq_one(one);
        a[L] = L == 0 ? one : z;
    }
    wsync<NW>();
}

// acc = prod_i B_i^{bits [i0, i0 + n) of d_i} with B_i = conj^i(pi^i(g)) (see above); g, c as above
template <int NW>
FPG_NOINL void w_gt_pow_bits(WGt& G, fq* acc, const fq* g, const uint32_t* c, int i0, int n) {
    uint32_t d[4][2];
    gls_digits(d, c);
    fq(*tab)[12] = G.tab;
    w_set_one<NW>(tab[0]);
    w_copy<NW>(tab[1], g);
    w_frob<NW>(G.w, tab[2], g);
    w_frob2<NW>(G.w, tab[4], g);
    w_frob<NW>(G.w, tab[8], tab[4]);
    w_conj<NW>(tab[2], tab[2]);
    w_conj<NW>(tab[8], tab[8]);
    for (int s = 3; s < 16; s++) {
        if (!(s & (s - 1))) continue;
        const int top = 31 - __clz(s);
        w_mul<NW>(G.w, tab[s], tab[s & ~(1 << top)], tab[1 << top]);
    }
    w_set_one<NW>(acc);
    for (int i = i0 + n - 1; i >= i0; i--) {
        w_cyc_sqr<NW>(G.w, acc, acc);
        const int s = bit_of(d[0], i) | (bit_of(d[1], i) << 1) | (bit_of(d[2], i) << 2) | (bit_of(d[3], i) << 3);
        if (s) w_mul<NW>(G.w, acc, acc, tab[s]);       // the same digits on every lane: uniform
    }
}
