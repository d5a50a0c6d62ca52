// Extension-field tower of BLS12-381 for the pairing:
//   Fq2  = Fq[u]/(u^2 + 1)
//   Fq6  = Fq2[v]/(v^3 - xi),  xi = 1 + u
//   Fq12 = Fq6[w]/(w^2 - v)
// Karatsuba products at every level, the complex squaring in Fq12, Frobenius maps with
// precomputed xi-powers, and the Granger-Scott squaring for the cyclotomic subgroup (Fq12 seen
// as Fq4[w]/(w^3 - s), Fq4 = Fq2[s]/(s^2 - xi), s = w^3).
#pragma once
#include "fp.cuh"

struct fq2 { fq c0, c1; };
struct fq6 { fq2 c0, c1, c2; };
struct fq12 { fq6 c0, c1; };

// ------------------------------------------------------------------------------ Fq2
FPG_DEV fq2 fq2_select(bool c, const fq2& a, const fq2& b) { return {fq_select(c, a.c0, b.c0), fq_select(c, a.c1, b.c1)}; }
FPG_DEV fq2 fq2_add(const fq2& a, const fq2& b) { return {fq_add(a.c0, b.c0), fq_add(a.c1, b.c1)}; }
FPG_DEV fq2 fq2_sub(const fq2& a, const fq2& b) { return {fq_sub(a.c0, b.c0), fq_sub(a.c1, b.c1)}; }
FPG_DEV fq2 fq2_dbl(const fq2& a) { return {fq_dbl(a.c0), fq_dbl(a.c1)}; }
FPG_DEV fq2 fq2_neg(const fq2& a) { return {fq_neg(a.c0), fq_neg(a.c1)}; }
FPG_DEV fq2 fq2_conj(const fq2& a) { return {a.c0, fq_neg(a.c1)}; }
FPG_DEV fq2 fq2_mul_fq(const fq2& a, const fq& b) { return {fq_mul(a.c0, b), fq_mul(a.c1, b)}; }
FPG_DEV void fq2_zero(fq2& a) { fq_zero(a.c0); fq_zero(a.c1); }
FPG_DEV void fq2_one(fq2& a) { fq_one(a.c0); fq_zero(a.c1); }
FPG_DEV bool fq2_is_zero(const fq2& a) { return fq_is_zero(a.c0) && fq_is_zero(a.c1); }
FPG_DEV bool fq2_eq(const fq2& a, const fq2& b) { return fq_eq(a.c0, b.c0) && fq_eq(a.c1, b.c1); }
FPG_NOINL fq2 fq2_mul(const fq2& a, const fq2& b) {
    fq t0 = fq_mul(a.c0, b.c0), t1 = fq_mul(a.c1, b.c1);
    fq s = fq_mul(fq_add(a.c0, a.c1), fq_add(b.c0, b.c1));
    return {fq_sub(t0, t1), fq_sub(fq_sub(s, t0), t1)};
}
FPG_NOINL fq2 fq2_sqr(const fq2& a) {
    fq t = fq_mul(a.c0, a.c1);
    return {fq_mul(fq_add(a.c0, a.c1), fq_sub(a.c0, a.c1)), fq_dbl(t)};
}
FPG_DEV fq2 fq2_mul_xi(const fq2& a) { return {fq_sub(a.c0, a.c1), fq_add(a.c0, a.c1)}; }
FPG_NOINL fq2 fq2_inv(const fq2& a) {
    fq n = fq_add(fq_sqr(a.c0), fq_sqr(a.c1));
    fq ni = fq_inv(n);
    return {fq_mul(a.c0, ni), fq_neg(fq_mul(a.c1, ni))};
}
// the same with the Fq inverse on the four lanes of a quad (fq_inv_quad)
FPG_NOINL fq2 fq2_inv_quad(const fq2& a) {
    fq n = fq_add(fq_sqr(a.c0), fq_sqr(a.c1));
    fq ni = fq_inv_quad(n);
    return {fq_mul(a.c0, ni), fq_neg(fq_mul(a.c1, ni))};
}

// ------------------------------------------------------------------------------ Fq6
FPG_DEV fq6 fq6_add(const fq6& a, const fq6& b) { return {fq2_add(a.c0, b.c0), fq2_add(a.c1, b.c1), fq2_add(a.c2, b.c2)}; }
FPG_DEV fq6 fq6_sub(const fq6& a, const fq6& b) { return {fq2_sub(a.c0, b.c0), fq2_sub(a.c1, b.c1), fq2_sub(a.c2, b.c2)}; }
FPG_DEV fq6 fq6_neg(const fq6& a) { return {fq2_neg(a.c0), fq2_neg(a.c1), fq2_neg(a.c2)}; }
FPG_DEV fq6 fq6_mul_v(const fq6& a) { return {fq2_mul_xi(a.c2), a.c0, a.c1}; }
FPG_DEV void fq6_zero(fq6& a) { fq2_zero(a.c0); fq2_zero(a.c1); fq2_zero(a.c2); }
FPG_DEV void fq6_one(fq6& a) { fq2_one(a.c0); fq2_zero(a.c1); fq2_zero(a.c2); }
FPG_NOINL fq6 fq6_mul(const fq6& a, const fq6& b) {
    fq2 t0 = fq2_mul(a.c0, b.c0), t1 = fq2_mul(a.c1, b.c1), t2 = fq2_mul(a.c2, b.c2);
    fq2 c0 = fq2_sub(fq2_sub(fq2_mul(fq2_add(a.c1, a.c2), fq2_add(b.c1, b.c2)), t1), t2);
    c0 = fq2_add(t0, fq2_mul_xi(c0));
    fq2 c1 = fq2_sub(fq2_sub(fq2_mul(fq2_add(a.c0, a.c1), fq2_add(b.c0, b.c1)), t0), t1);
    c1 = fq2_add(c1, fq2_mul_xi(t2));
    fq2 c2 = fq2_sub(fq2_sub(fq2_mul(fq2_add(a.c0, a.c2), fq2_add(b.c0, b.c2)), t0), t2);
    c2 = fq2_add(c2, t1);
    return {c0, c1, c2};
}
// a * (x + y v): c0 = a0 x + xi a2 y, c1 = a0 y + a1 x, c2 = a1 y + a2 x
FPG_NOINL fq6 fq6_mul_01(const fq6& a, const fq2& x, const fq2& y) {
    fq2 c0 = fq2_add(fq2_mul(a.c0, x), fq2_mul_xi(fq2_mul(a.c2, y)));
    fq2 c1 = fq2_add(fq2_mul(a.c0, y), fq2_mul(a.c1, x));
    fq2 c2 = fq2_add(fq2_mul(a.c1, y), fq2_mul(a.c2, x));
    return {c0, c1, c2};
}
// a * (y v) = (xi a2 y, a0 y, a1 y)
FPG_DEV fq6 fq6_mul_1(const fq6& a, const fq2& y) {
    return {fq2_mul_xi(fq2_mul(a.c2, y)), fq2_mul(a.c0, y), fq2_mul(a.c1, y)};
}
FPG_NOINL fq6 fq6_inv(const fq6& a) {
    fq2 c0 = fq2_sub(fq2_sqr(a.c0), fq2_mul_xi(fq2_mul(a.c1, a.c2)));
    fq2 c1 = fq2_sub(fq2_mul_xi(fq2_sqr(a.c2)), fq2_mul(a.c0, a.c1));
    fq2 c2 = fq2_sub(fq2_sqr(a.c1), fq2_mul(a.c0, a.c2));
    fq2 t = fq2_add(fq2_mul(a.c0, c0), fq2_mul_xi(fq2_add(fq2_mul(a.c2, c1), fq2_mul(a.c1, c2))));
    fq2 ti = fq2_inv(t);
    return {fq2_mul(c0, ti), fq2_mul(c1, ti), fq2_mul(c2, ti)};
}

// ------------------------------------------------------------------------------ Fq12
FPG_DEV void fq12_one(fq12& a) { fq6_one(a.c0); fq6_zero(a.c1); }
FPG_DEV fq12 fq12_conj(const fq12& a) { return {a.c0, fq6_neg(a.c1)}; }
FPG_NOINL fq12 fq12_mul(const fq12& a, const fq12& b) {
    fq6 t0 = fq6_mul(a.c0, b.c0), t1 = fq6_mul(a.c1, b.c1);
    fq6 c1 = fq6_sub(fq6_sub(fq6_mul(fq6_add(a.c0, a.c1), fq6_add(b.c0, b.c1)), t0), t1);
    return {fq6_add(t0, fq6_mul_v(t1)), c1};
}
// complex squaring: (a0 + a1 w)^2 = (a0 + a1)(a0 + v a1) - t - v t + 2 t w, t = a0 a1
FPG_NOINL fq12 fq12_sqr(const fq12& a) {
    fq6 t = fq6_mul(a.c0, a.c1);
    fq6 c0 = fq6_mul(fq6_add(a.c0, a.c1), fq6_add(a.c0, fq6_mul_v(a.c1)));
    c0 = fq6_sub(fq6_sub(c0, t), fq6_mul_v(t));
    return {c0, fq6_add(t, t)};
}
FPG_NOINL fq12 fq12_inv(const fq12& a) {
    fq6 t = fq6_sub(fq6_mul(a.c0, a.c0), fq6_mul_v(fq6_mul(a.c1, a.c1)));
    fq6 ti = fq6_inv(t);
    return {fq6_mul(a.c0, ti), fq6_neg(fq6_mul(a.c1, ti))};
}
// f * (l0 + l2 w^2 + l3 w^3): in the tower the line is (l0 + l2 v) + (l3 v) w
FPG_NOINL fq12 fq12_mul_line(const fq12& a, const fq2& l0, const fq2& l2, const fq2& l3) {
    fq6 t0 = fq6_mul_01(a.c0, l0, l2);
    fq6 t1 = fq6_mul_1(a.c1, l3);
    fq6 c1 = fq6_sub(fq6_sub(fq6_mul_01(fq6_add(a.c0, a.c1), l0, fq2_add(l2, l3)), t0), t1);
    return {fq6_add(t0, fq6_mul_v(t1)), c1};
}

// flat coefficient k of w^k: k = 0,2,4 -> c0.c0,c0.c1,c0.c2 ; k = 1,3,5 -> c1.c0,c1.c1,c1.c2
FPG_DEV fq2& fq12_flat(fq12& a, int k) {
    fq6& h = (k & 1) ? a.c1 : a.c0;
    int i = k >> 1;
    return i == 0 ? h.c0 : (i == 1 ? h.c1 : h.c2);
}

FPG_DEV fq2 frob1_coef(int k) {
    fq2 g;
    switch (k) {
        case 1: fq_from_const(g.c0, FROB1_1_C0); fq_from_const(g.c1, FROB1_1_C1); break;
        case 2: fq_from_const(g.c0, FROB1_2_C0); fq_from_const(g.c1, FROB1_2_C1); break;
        case 3: fq_from_const(g.c0, FROB1_3_C0); fq_from_const(g.c1, FROB1_3_C1); break;
        case 4: fq_from_const(g.c0, FROB1_4_C0); fq_from_const(g.c1, FROB1_4_C1); break;
        default: fq_from_const(g.c0, FROB1_5_C0); fq_from_const(g.c1, FROB1_5_C1); break;
    }
    return g;
}
FPG_DEV fq frob2_coef(int k) {
    fq g;
    switch (k) {
        case 1: fq_from_const(g, FROB2_1); break;
        case 2: fq_from_const(g, FROB2_2); break;
        case 3: fq_from_const(g, FROB2_3); break;
        case 4: fq_from_const(g, FROB2_4); break;
        default: fq_from_const(g, FROB2_5); break;
    }
    return g;
}
// f^p: w^p = xi^((p-1)/6) w, coefficients conjugated
FPG_NOINL fq12 fq12_frob(const fq12& a) {
    fq12 r = a;
    fq12_flat(r, 0) = fq2_conj(fq12_flat(r, 0));
#pragma unroll 1
    for (int k = 1; k < 6; k++) fq12_flat(r, k) = fq2_mul(fq2_conj(fq12_flat(r, k)), frob1_coef(k));
    return r;
}
// f^(p^2): coefficients fixed, w^(p^2) = xi^((p^2-1)/6) w with the factor in Fq
FPG_NOINL fq12 fq12_frob2(const fq12& a) {
    fq12 r = a;
#pragma unroll 1
    for (int k = 1; k < 6; k++) fq12_flat(r, k) = fq2_mul_fq(fq12_flat(r, k), frob2_coef(k));
    return r;
}

// (a + b s)^2 = (a^2 + xi b^2) + 2ab s, with 2ab = (a + b)^2 - a^2 - b^2
FPG_DEV void fq4_sqr(fq2& ra, fq2& rb, const fq2& a, const fq2& b) {
    fq2 a2 = fq2_sqr(a), b2 = fq2_sqr(b);
    ra = fq2_add(a2, fq2_mul_xi(b2));
    rb = fq2_sub(fq2_sub(fq2_sqr(fq2_add(a, b)), a2), b2);
}
// Granger-Scott squaring for f with f^(p^6+1)(p^2-1)... in the cyclotomic subgroup:
// with A0 = (c_0, c_3), A1 = (c_1, c_4), A2 = (c_2, c_5) (flat indices) and t_i = A_i^2,
// A0' = 3 t0 - 2 conj(A0), A1' = 3 s t2 + 2 conj(A1), A2' = 3 t1 - 2 conj(A2).
FPG_NOINL fq12 fq12_cyclotomic_sqr(const fq12& f) {
    fq12 z = f;
    fq2 z0 = fq12_flat(z, 0), z3 = fq12_flat(z, 3), z1 = fq12_flat(z, 1), z4 = fq12_flat(z, 4),
        z2 = fq12_flat(z, 2), z5 = fq12_flat(z, 5);
    fq2 t0a, t0b, t1a, t1b, t2a, t2b;
    fq4_sqr(t0a, t0b, z0, z3);
    fq4_sqr(t1a, t1b, z1, z4);
    fq4_sqr(t2a, t2b, z2, z5);
    fq12 r;
    // A0
    fq2 tmp = fq2_sub(t0a, z0);
    fq12_flat(r, 0) = fq2_add(fq2_dbl(tmp), t0a);
    tmp = fq2_add(t0b, z3);
    fq12_flat(r, 3) = fq2_add(fq2_dbl(tmp), t0b);
    // A1 = 3 s t2 + 2 conj(A1), s (a + b s) = xi b + a s
    fq2 s0 = fq2_mul_xi(t2b), s1 = t2a;
    tmp = fq2_add(s0, z1);
    fq12_flat(r, 1) = fq2_add(fq2_dbl(tmp), s0);
    tmp = fq2_sub(s1, z4);
    fq12_flat(r, 4) = fq2_add(fq2_dbl(tmp), s1);
    // A2
    tmp = fq2_sub(t1a, z2);
    fq12_flat(r, 2) = fq2_add(fq2_dbl(tmp), t1a);
    tmp = fq2_add(t1b, z5);
    fq12_flat(r, 5) = fq2_add(fq2_dbl(tmp), t1b);
    return r;
}

FPG_DEV bool fq12_eq(const fq12& a, const fq12& b) {
    return fq2_eq(a.c0.c0, b.c0.c0) && fq2_eq(a.c0.c1, b.c0.c1) && fq2_eq(a.c0.c2, b.c0.c2) &&
           fq2_eq(a.c1.c0, b.c1.c0) && fq2_eq(a.c1.c1, b.c1.c1) && fq2_eq(a.c1.c2, b.c1.c2);
}

// 576-byte canonical big-endian serialisation in tower order
FPG_DEV void fq12_to_be(uint8_t* out, const fq12& a) {
    const fq2* c[6] = {&a.c0.c0, &a.c0.c1, &a.c0.c2, &a.c1.c0, &a.c1.c1, &a.c1.c2};
    for (int t = 0; t < 6; t++) {
        fq_to_be(out + 96 * t, c[t]->c0);
        fq_to_be(out + 96 * t + 48, c[t]->c1);
    }
}
