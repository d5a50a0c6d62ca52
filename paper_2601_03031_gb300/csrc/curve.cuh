// G1 = E(Fq): y^2 = x^3 + 4 and G2 = E'(Fq2): y^2 = x^3 + 4(1 + u) (the M-type sextic twist).
// Points in device memory are affine Montgomery coordinates with (0, 0) as the identity (never
// on either curve since b != 0).  Arithmetic is in Jacobian coordinates, one generic template
// over the coordinate field: doubling dbl-2009-l, mixed addition madd-2007-bl and general
// addition add-2007-bl of the Explicit-Formulas Database (short Weierstrass, a = 0).
#pragma once
#include "tower.cuh"

struct g1a { fq x, y; };
struct g2a { fq2 x, y; };
template <typename F> struct jac { F X, Y, Z; };
using g1j = jac<fq>;
using g2j = jac<fq2>;

// field overload set so one template serves both coordinate fields
FPG_DEV fq f_add(const fq& a, const fq& b) { return fq_add(a, b); }
FPG_DEV fq f_sub(const fq& a, const fq& b) { return fq_sub(a, b); }
FPG_DEV fq f_dbl(const fq& a) { return fq_dbl(a); }
FPG_DEV fq f_mul(const fq& a, const fq& b) { return fq_mul(a, b); }
FPG_DEV fq f_sqr(const fq& a) { return fq_sqr(a); }
FPG_DEV fq f_neg(const fq& a) { return fq_neg(a); }
FPG_DEV fq f_inv(const fq& a) { return fq_inv(a); }
FPG_DEV bool f_is_zero(const fq& a) { return fq_is_zero(a); }
FPG_DEV bool f_eq(const fq& a, const fq& b) { return fq_eq(a, b); }
FPG_DEV void f_set_zero(fq& a) { fq_zero(a); }
FPG_DEV void f_set_one(fq& a) { fq_one(a); }
FPG_DEV fq2 f_add(const fq2& a, const fq2& b) { return fq2_add(a, b); }
FPG_DEV fq2 f_sub(const fq2& a, const fq2& b) { return fq2_sub(a, b); }
FPG_DEV fq2 f_dbl(const fq2& a) { return fq2_dbl(a); }
FPG_DEV fq2 f_mul(const fq2& a, const fq2& b) { return fq2_mul(a, b); }
FPG_DEV fq2 f_sqr(const fq2& a) { return fq2_sqr(a); }
FPG_DEV fq2 f_neg(const fq2& a) { return fq2_neg(a); }
FPG_DEV fq2 f_inv(const fq2& a) { return fq2_inv(a); }
FPG_DEV bool f_is_zero(const fq2& a) { return fq2_is_zero(a); }
FPG_DEV bool f_eq(const fq2& a, const fq2& b) { return fq2_eq(a, b); }
FPG_DEV void f_set_zero(fq2& a) { fq2_zero(a); }
FPG_DEV void f_set_one(fq2& a) { fq2_one(a); }

template <typename F>
FPG_DEV void jac_set_inf(jac<F>& p) { f_set_one(p.X); f_set_one(p.Y); f_set_zero(p.Z); }
template <typename F>
FPG_DEV bool jac_is_inf(const jac<F>& p) { return f_is_zero(p.Z); }

template <typename F>
FPG_NOINL jac<F> jac_dbl(const jac<F>& p) {
    jac<F> r;
    if (jac_is_inf(p)) { jac_set_inf(r); return r; }
    F A = f_sqr(p.X), B = f_sqr(p.Y), C = f_sqr(B);
    F D = f_dbl(f_sub(f_sub(f_sqr(f_add(p.X, B)), A), C));
    F E = f_add(f_dbl(A), A);
    F Fv = f_sqr(E);
    r.X = f_sub(Fv, f_dbl(D));
    F C8 = f_dbl(f_dbl(f_dbl(C)));
    r.Y = f_sub(f_mul(E, f_sub(D, r.X)), C8);
    r.Z = f_dbl(f_mul(p.Y, p.Z));
    return r;
}

// p + (x2, y2) with the second point affine (and not the identity)
template <typename F>
FPG_NOINL jac<F> jac_madd(const jac<F>& p, const F& x2, const F& y2) {
    jac<F> r;
    if (jac_is_inf(p)) { r.X = x2; r.Y = y2; f_set_one(r.Z); return r; }
    F Z1Z1 = f_sqr(p.Z);
    F U2 = f_mul(x2, Z1Z1);
    F S2 = f_mul(f_mul(y2, p.Z), Z1Z1);
    F H = f_sub(U2, p.X);
    F Rr = f_sub(S2, p.Y);
    if (f_is_zero(H)) {
        if (f_is_zero(Rr)) return jac_dbl(p);
        jac_set_inf(r);
        return r;
    }
    F HH = f_sqr(H);
    F I = f_dbl(f_dbl(HH));
    F J = f_mul(H, I);
    F rr = f_dbl(Rr);
    F V = f_mul(p.X, I);
    r.X = f_sub(f_sub(f_sqr(rr), J), f_dbl(V));
    r.Y = f_sub(f_mul(rr, f_sub(V, r.X)), f_dbl(f_mul(p.Y, J)));
    r.Z = f_sub(f_sub(f_sqr(f_add(p.Z, H)), Z1Z1), HH);
    return r;
}

template <typename F>
FPG_NOINL jac<F> jac_add(const jac<F>& p, const jac<F>& q) {
    if (jac_is_inf(p)) return q;
    if (jac_is_inf(q)) return p;
    F Z1Z1 = f_sqr(p.Z), Z2Z2 = f_sqr(q.Z);
    F U1 = f_mul(p.X, Z2Z2), U2 = f_mul(q.X, Z1Z1);
    F S1 = f_mul(f_mul(p.Y, q.Z), Z2Z2), S2 = f_mul(f_mul(q.Y, p.Z), Z1Z1);
    F H = f_sub(U2, U1);
    F Rr = f_sub(S2, S1);
    jac<F> r;
    if (f_is_zero(H)) {
        if (f_is_zero(Rr)) return jac_dbl(p);
        jac_set_inf(r);
        return r;
    }
    F I = f_sqr(f_dbl(H));
    F J = f_mul(H, I);
    F rr = f_dbl(Rr);
    F V = f_mul(U1, I);
    r.X = f_sub(f_sub(f_sqr(rr), J), f_dbl(V));
    r.Y = f_sub(f_mul(rr, f_sub(V, r.X)), f_dbl(f_mul(S1, J)));
    r.Z = f_mul(f_sub(f_sub(f_sqr(f_add(p.Z, q.Z)), Z1Z1), Z2Z2), H);
    return r;
}

// k * (x, y) for an affine point and a canonical (non-Montgomery) little-endian 256-bit scalar,
// most-significant bit first.
template <typename F>
FPG_NOINL jac<F> jac_mul_affine(const F& x, const F& y, bool inf, const uint32_t* k) {
    jac<F> acc;
    jac_set_inf(acc);
    if (inf) return acc;
    int top = 255;
    while (top >= 0 && !((k[top >> 5] >> (top & 31)) & 1)) top--;
    for (int i = top; i >= 0; i--) {
        acc = jac_dbl(acc);
        if ((k[i >> 5] >> (i & 31)) & 1) acc = jac_madd(acc, x, y);
    }
    return acc;
}

template <typename F>
FPG_DEV void jac_to_affine(F& x, F& y, const jac<F>& p) {
    if (jac_is_inf(p)) { f_set_zero(x); f_set_zero(y); return; }
    F zi = f_inv(p.Z);
    F zi2 = f_sqr(zi);
    x = f_mul(p.X, zi2);
    y = f_mul(p.Y, f_mul(zi2, zi));
}

FPG_DEV bool g1a_is_inf(const g1a& p) { return fq_is_zero(p.x) && fq_is_zero(p.y); }
FPG_DEV bool g2a_is_inf(const g2a& p) { return fq2_is_zero(p.x) && fq2_is_zero(p.y); }
FPG_DEV g1a g1_affine(const g1j& p) { g1a r; jac_to_affine(r.x, r.y, p); return r; }
FPG_DEV g2a g2_affine(const g2j& p) { g2a r; jac_to_affine(r.x, r.y, p); return r; }
FPG_DEV g1j g1_from_affine(const g1a& a) {
    g1j r;
    if (g1a_is_inf(a)) { jac_set_inf(r); return r; }
    r.X = a.x; r.Y = a.y; fq_one(r.Z);
    return r;
}
FPG_DEV g2j g2_from_affine(const g2a& a) {
    g2j r;
    if (g2a_is_inf(a)) { jac_set_inf(r); return r; }
    r.X = a.x; r.Y = a.y; fq2_one(r.Z);
    return r;
}
FPG_DEV g1j g1_mul(const g1a& p, const uint32_t* k) { return jac_mul_affine(p.x, p.y, g1a_is_inf(p), k); }
FPG_DEV g2j g2_mul(const g2a& p, const uint32_t* k) { return jac_mul_affine(p.x, p.y, g2a_is_inf(p), k); }
FPG_DEV g1j g1_madd(const g1j& p, const g1a& q) { return g1a_is_inf(q) ? p : jac_madd(p, q.x, q.y); }
FPG_DEV g2j g2_madd(const g2j& p, const g2a& q) { return g2a_is_inf(q) ? p : jac_madd(p, q.x, q.y); }
FPG_DEV g1a g1a_neg(const g1a& p) { return g1a_is_inf(p) ? p : g1a{p.x, fq_neg(p.y)}; }
FPG_DEV g2a g2a_neg(const g2a& p) { return g2a_is_inf(p) ? p : g2a{p.x, fq2_neg(p.y)}; }

FPG_DEV g1a g1_generator() {
    g1a g; fq_from_const(g.x, G1_GEN_X); fq_from_const(g.y, G1_GEN_Y); return g;
}
FPG_DEV g2a g2_generator() {
    g2a g;
    fq_from_const(g.x.c0, G2_GEN_X0); fq_from_const(g.x.c1, G2_GEN_X1);
    fq_from_const(g.y.c0, G2_GEN_Y0); fq_from_const(g.y.c1, G2_GEN_Y1);
    return g;
}

// canonical big-endian serialisation (identity = all zero bytes)
FPG_DEV void g1a_to_be(uint8_t* out, const g1a& p) { fq_to_be(out, p.x); fq_to_be(out + 48, p.y); }
FPG_DEV void g2a_to_be(uint8_t* out, const g2a& p) {
    fq_to_be(out, p.x.c0); fq_to_be(out + 48, p.x.c1); fq_to_be(out + 96, p.y.c0); fq_to_be(out + 144, p.y.c1);
}
