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
FPG_DEV fq f_inv_quad(const fq& a) { return fq_inv_quad(a); }
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
FPG_DEV fq2 f_inv_quad(const fq2& a) { return fq2_inv_quad(a); }
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

// the same with the inverse on the four lanes of a quad (f_inv_quad: all four call converged with
// the same point); the inverse of 0 is 0, so the identity (Z = 0) gives (0, 0) without a branch
template <typename F>
FPG_DEV void jac_to_affine_quad(F& x, F& y, const jac<F>& p) {
    F zi = f_inv_quad(p.Z);
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

// ---------------------------------------------------------------------------------------
// Endomorphism-split scalar multiplication.
//   G1 (GLV): phi(x, y) = (omega x, y) = [-x^2] on G1, so with k = k0 + k1 |x|^2 (k0 < |x|^2),
//             k P = k0 P + k1 (-phi(P)): 128-bit halves, one joint double-and-add.
//   G2 (GLS): psi = untwist-Frobenius-twist acts as [x] on G2, so with base-|x| digits
//             k = d0 + d1 |x| + d2 |x|^2 + d3 |x|^3 (x < 0), k Q = d0 Q - d1 psi Q + d2 psi^2 Q - d3 psi^3 Q:
//             64-bit digits, a 16-entry table of subset sums (normalised to affine with one
//             inversion), one joint double-and-add.
// ---------------------------------------------------------------------------------------

// q = floor(k / D) and rem = k - q D for a 256-bit k and a constant D < 2^(32 ND), using the
// Barrett constant bar = floor(2^256 / D) (NB limbs) and at most a few correction steps.
template <int ND, int NB>
FPG_DEV void div_by_const(uint32_t* q, uint32_t* rem, const uint32_t* k, const uint32_t* D, const uint32_t* bar) {
    uint32_t prod[8 + NB];
    for (int i = 0; i < 8 + NB; i++) prod[i] = 0;
    for (int i = 0; i < 8; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < NB; j++) {
            uint64_t t = (uint64_t)k[i] * bar[j] + prod[i + j] + carry;
            prod[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        prod[i + NB] = (uint32_t)carry;
    }
    for (int j = 0; j < NB; j++) q[j] = prod[8 + j];          // estimate, at most a few too small
    uint32_t r[8];
    {
        uint32_t qd[8];
        for (int i = 0; i < 8; i++) qd[i] = 0;
        for (int i = 0; i < NB; i++) {
            uint64_t carry = 0;
            for (int j = 0; j < ND && i + j < 8; j++) {
                uint64_t t = (uint64_t)q[i] * D[j] + qd[i + j] + carry;
                qd[i + j] = (uint32_t)t;
                carry = t >> 32;
            }
            if (i + ND < 8) qd[i + ND] = (uint32_t)carry;
        }
        int64_t borrow = 0;
        for (int i = 0; i < 8; i++) {
            int64_t d = (int64_t)k[i] - qd[i] - borrow;
            borrow = d < 0;
            r[i] = (uint32_t)d;
        }
    }
    for (int it = 0; it < 4; it++) {                          // while r >= D: r -= D, q += 1
        bool ge = true;
        for (int i = 7; i >= 0; i--) {
            uint32_t di = i < ND ? D[i] : 0;
            if (r[i] != di) { ge = r[i] > di; break; }
        }
        if (!ge) break;
        int64_t borrow = 0;
        for (int i = 0; i < 8; i++) {
            int64_t d = (int64_t)r[i] - (i < ND ? D[i] : 0) - borrow;
            borrow = d < 0;
            r[i] = (uint32_t)d;
        }
        for (int i = 0; i < NB; i++) if (++q[i] != 0) break;
    }
    for (int i = 0; i < ND; i++) rem[i] = r[i];
}

FPG_DEV int bit_of(const uint32_t* a, int i) { return (a[i >> 5] >> (i & 31)) & 1; }

// k P for affine P in G1 and a canonical scalar k < r.  The three non-zero digit pairs select one of
// three affine points (P, -phi(P), P - phi(P)), so every step is one doubling and at most one mixed
// addition with the same code path in every lane.
FPG_NOINL g1j g1_mul_glv(const g1a& P, const uint32_t* k) {
    g1j acc;
    jac_set_inf(acc);
    if (g1a_is_inf(P)) return acc;
    uint32_t k1[5], k0[4];
    div_by_const<4, 5>(k1, k0, k, GLV_D, GLV_BARRETT);
    fq om;
    fq_from_const(om, GLV_OMEGA);
    g1a T[4];
    T[1] = P;
    T[2] = {fq_mul(P.x, om), fq_neg(P.y)};                                     // -phi(P)
    T[3] = g1_affine(jac_madd(g1_from_affine(P), T[2].x, T[2].y));              // P - phi(P) = [1 + x^2] P
    int top = 159;
    while (top >= 0 && !(top < 128 && bit_of(k0, top)) && !bit_of(k1, top)) top--;
    for (int i = top; i >= 0; i--) {
        acc = jac_dbl(acc);
        const int s = (i < 128 ? bit_of(k0, i) : 0) | (bit_of(k1, i) << 1);
        if (s) acc = jac_madd(acc, T[s].x, T[s].y);
    }
    return acc;
}

FPG_DEV g2a g2_psi(const g2a& p) {
    fq2 cx, cy;
    fq_from_const(cx.c0, PSI_CX0); fq_from_const(cx.c1, PSI_CX1);
    fq_from_const(cy.c0, PSI_CY0); fq_from_const(cy.c1, PSI_CY1);
    return {fq2_mul(fq2_conj(p.x), cx), fq2_mul(fq2_conj(p.y), cy)};
}

// k Q for affine Q in G2 and a canonical scalar k < r
FPG_NOINL g2j g2_mul_gls(const g2a& Q, const uint32_t* k) {
    g2j acc;
    jac_set_inf(acc);
    if (g2a_is_inf(Q)) return acc;
    uint32_t q1[7], q2[7], q3[7], d[4][2];
    div_by_const<2, 7>(q1, d[0], k, GLS_D, GLS_BARRETT);
    uint32_t t8[8];
    for (int i = 0; i < 8; i++) t8[i] = i < 7 ? q1[i] : 0;
    div_by_const<2, 7>(q2, d[1], t8, GLS_D, GLS_BARRETT);
    for (int i = 0; i < 8; i++) t8[i] = i < 7 ? q2[i] : 0;
    div_by_const<2, 7>(q3, d[2], t8, GLS_D, GLS_BARRETT);
    d[3][0] = q3[0]; d[3][1] = q3[1];
    // bases B_i = (-1)^i psi^i(Q)
    g2a B[4];
    B[0] = Q;
    for (int i = 1; i < 4; i++) B[i] = g2_psi(B[i - 1]);
    B[1].y = fq2_neg(B[1].y);
    B[3].y = fq2_neg(B[3].y);
    // subset sums T[s] = sum_{i in s} B_i, then affine with one inversion (Montgomery's trick)
    g2j T[16];
    for (int s = 1; s < 16; s++) {
        int top = 31 - __clz(s);
        int rest = s & ~(1 << top);
        T[s] = rest ? jac_madd(T[rest], B[top].x, B[top].y) : g2_from_affine(B[top]);
    }
    fq2 pre[16];
    pre[1] = T[1].Z;
    for (int s = 2; s < 16; s++) pre[s] = fq2_mul(pre[s - 1], T[s].Z);
    fq2 inv = fq2_inv(pre[15]);
    g2a TA[16];
    for (int s = 15; s >= 1; s--) {
        fq2 zi = s > 1 ? fq2_mul(inv, pre[s - 1]) : inv;
        if (s > 1) inv = fq2_mul(inv, T[s].Z);
        fq2 zi2 = fq2_sqr(zi);
        TA[s].x = fq2_mul(T[s].X, zi2);
        TA[s].y = fq2_mul(T[s].Y, fq2_mul(zi2, zi));
    }
    int top = 63;
    while (top >= 0 && !(bit_of(d[0], top) | bit_of(d[1], top) | bit_of(d[2], top) | bit_of(d[3], top))) top--;
    for (int i = top; i >= 0; i--) {
        acc = jac_dbl(acc);
        int s = bit_of(d[0], i) | (bit_of(d[1], i) << 1) | (bit_of(d[2], i) << 2) | (bit_of(d[3], i) << 3);
        if (s) acc = jac_madd(acc, TA[s].x, TA[s].y);
    }
    return acc;
}

// scalar multiplication by a canonical k < r (GLV on G1, GLS on G2)
FPG_DEV g1j g1_mul(const g1a& p, const uint32_t* k) { return g1_mul_glv(p, k); }
FPG_DEV g2j g2_mul(const g2a& p, const uint32_t* k) { return g2_mul_gls(p, k); }

// canonical big-endian serialisation (identity = all zero bytes)
FPG_DEV void g1a_to_be(uint8_t* out, const g1a& p) { fq_to_be(out, p.x); fq_to_be(out + 48, p.y); }
FPG_DEV void g2a_to_be(uint8_t* out, const g2a& p) {
    fq_to_be(out, p.x.c0); fq_to_be(out + 48, p.x.c1); fq_to_be(out + 96, p.y.c0); fq_to_be(out + 144, p.y.c1);
}
