// Optimal-ate pairing on BLS12-381: e(P, Q) = (conj f_{|x|,Q}(P))^((p^12 - 1)/r), x = -0xd201000000010000.
//
// Miller loop: T runs in homogeneous projective coordinates on the twist; each step returns the
// line through T (tangent or chord through Q) evaluated at P, scaled by a factor in Fq2 (which
// the final exponentiation removes) and by w^3 (whose ((p^12-1)/r)-th power is 1):
//   doubling:  l = (Y^2 - 3 b' Z^2) - 3 X^2 xP w^2 + 2 Y Z yP w^3,
//              2T = (2XY(Y^2 - 9b'Z^2), (Y^2 + 9b'Z^2)^2 - 108 b'^2 Z^4, 8 Y^3 Z)
//   addition:  theta = Y - yQ Z, lambda = X - xQ Z,
//              l = (theta xQ - lambda yQ) - theta xP w^2 + lambda yP w^3
// Final exponentiation, exact: (p^12-1)/r = (p^6 - 1)(p^2 + 1) d with
//   d = (p^4 - p^2 + 1)/r = h1 (x + p)(x^2 + p^2 - 1) + 1,  h1 = (x - 1)^2 / 3,
// an identity of the BLS12 parametrisation (r = x^4 - x^2 + 1, p = h1 r + x), evaluated with
// cyclotomic squarings, Frobenius maps and conjugation as the inverse in the cyclotomic subgroup.
#pragma once
#include "curve.cuh"

// b' = 4(1 + u); b' Z^2 = 4 xi Z^2
FPG_DEV fq2 mul_bprime(const fq2& z) { return fq2_dbl(fq2_dbl(fq2_mul_xi(z))); }

struct line3 { fq2 l0, l2, l3; };

// k * a for a small positive integer k (double-and-add on k's bits)
FPG_DEV fq2 fq2_mul_small(const fq2& a, unsigned k) {
    fq2 acc; fq2_zero(acc);
    for (int i = 31 - __clz(k); i >= 0; i--) {
        acc = fq2_dbl(acc);
        if ((k >> i) & 1) acc = fq2_add(acc, a);
    }
    return acc;
}

FPG_DEV void miller_dbl_step(g2j& T, line3& l, const fq& xP, const fq& yP) {
    fq2 XX = fq2_sqr(T.X), YY = fq2_sqr(T.Y), ZZ = fq2_sqr(T.Z);
    fq2 YZ = fq2_mul(T.Y, T.Z);
    fq2 bz = mul_bprime(ZZ);                                   // b' Z^2
    fq2 bz3 = fq2_add(fq2_dbl(bz), bz);                        // 3 b' Z^2
    l.l0 = fq2_sub(YY, bz3);
    fq m3x = fq_neg(fq_add(fq_dbl(xP), xP));                   // -3 xP
    l.l2 = fq2_mul_fq(XX, m3x);
    l.l3 = fq2_mul_fq(fq2_dbl(YZ), yP);
    fq2 bz9 = fq2_add(fq2_dbl(bz3), bz3);                      // 9 b' Z^2
    fq2 XY = fq2_mul(T.X, T.Y);
    fq2 nX = fq2_mul(fq2_dbl(XY), fq2_sub(YY, bz9));
    fq2 s = fq2_add(YY, bz9);
    fq2 b108 = fq2_mul_small(fq2_sqr(bz), 108);                // 108 b'^2 Z^4
    fq2 nY = fq2_sub(fq2_sqr(s), b108);
    fq2 nZ = fq2_dbl(fq2_dbl(fq2_dbl(fq2_mul(YY, YZ))));       // 8 Y^3 Z
    T.X = nX; T.Y = nY; T.Z = nZ;
}

FPG_DEV void miller_add_step(g2j& T, line3& l, const fq2& xQ, const fq2& yQ, const fq& xP, const fq& yP) {
    fq2 th = fq2_sub(T.Y, fq2_mul(yQ, T.Z));
    fq2 la = fq2_sub(T.X, fq2_mul(xQ, T.Z));
    l.l0 = fq2_sub(fq2_mul(th, xQ), fq2_mul(la, yQ));
    l.l2 = fq2_mul_fq(th, fq_neg(xP));
    l.l3 = fq2_mul_fq(la, yP);
    fq2 C = fq2_sqr(th), D = fq2_sqr(la);
    fq2 E = fq2_mul(D, la);
    fq2 F = fq2_mul(T.Z, C);
    fq2 G = fq2_mul(T.X, D);
    fq2 H = fq2_sub(fq2_add(E, F), fq2_dbl(G));
    fq2 nX = fq2_mul(la, H);
    fq2 nY = fq2_sub(fq2_mul(th, fq2_sub(G, H)), fq2_mul(T.Y, E));
    fq2 nZ = fq2_mul(T.Z, E);
    T.X = nX; T.Y = nY; T.Z = nZ;
}

// conj(f_{|x|,Q}(P)); 1 when P or Q is the identity
FPG_NOINL fq12 miller_loop(const g1a& P, const g2a& Q) {
    fq12 f;
    fq12_one(f);
    if (g1a_is_inf(P) || g2a_is_inf(Q)) return f;
    g2j T = g2_from_affine(Q);
    line3 l;
    bool first = true;
    for (int i = 62; i >= 0; i--) {
        if (!first) f = fq12_sqr(f);
        miller_dbl_step(T, l, P.x, P.y);
        f = fq12_mul_line(f, l.l0, l.l2, l.l3);
        first = false;
        if ((BLS_X_ABS >> i) & 1) {
            miller_add_step(T, l, Q.x, Q.y, P.x, P.y);
            f = fq12_mul_line(f, l.l0, l.l2, l.l3);
        }
    }
    return fq12_conj(f);
}

// prod_g conj(f_{|x|,Q_g}(P_g)) for G pairs in one loop: the squaring of f is shared by the pairs
// (a product of Miller functions squares as one), each step multiplies in every pair's line
template <int G>
FPG_NOINL fq12 miller_loop_multi(const g1a* P, const g2a* Q) {
    fq12 f;
    fq12_one(f);
    g2j T[G];
    bool live[G];
    for (int g = 0; g < G; g++) {
        live[g] = !(g1a_is_inf(P[g]) || g2a_is_inf(Q[g]));
        T[g] = g2_from_affine(Q[g]);
    }
    line3 l;
    bool first = true;
    for (int i = 62; i >= 0; i--) {
        if (!first) f = fq12_sqr(f);
        first = false;
        for (int g = 0; g < G; g++) {
            if (!live[g]) continue;
            miller_dbl_step(T[g], l, P[g].x, P[g].y);
            f = fq12_mul_line(f, l.l0, l.l2, l.l3);
        }
        if ((BLS_X_ABS >> i) & 1) {
            for (int g = 0; g < G; g++) {
                if (!live[g]) continue;
                miller_add_step(T[g], l, Q[g].x, Q[g].y, P[g].x, P[g].y);
                f = fq12_mul_line(f, l.l0, l.l2, l.l3);
            }
        }
    }
    return fq12_conj(f);
}

// a^e for a in the cyclotomic subgroup and a plain exponent given as little-endian 32-bit words
FPG_NOINL fq12 cyclotomic_exp(const fq12& a, const uint32_t* e, int bits) {
    fq12 acc;
    fq12_one(acc);
    bool started = false;
    for (int i = bits - 1; i >= 0; i--) {
        if (started) acc = fq12_cyclotomic_sqr(acc);
        if ((e[i >> 5] >> (i & 31)) & 1) {
            acc = started ? fq12_mul(acc, a) : a;
            started = true;
        }
    }
    return acc;
}
FPG_DEV fq12 cyclotomic_exp_xabs(const fq12& a) {
    uint32_t e[2] = {(uint32_t)BLS_X_ABS, (uint32_t)(BLS_X_ABS >> 32)};
    return cyclotomic_exp(a, e, 64);
}

FPG_NOINL fq12 final_exp(const fq12& f) {
    // easy part: f^((p^6 - 1)(p^2 + 1))
    fq12 t = fq12_mul(fq12_conj(f), fq12_inv(f));
    fq12 g = fq12_mul(fq12_frob2(t), t);
    // hard part: g^d, d = h1 (x + p)(x^2 + p^2 - 1) + 1
    uint32_t h1[4] = {BLS_H1[0], BLS_H1[1], BLS_H1[2], BLS_H1[3]};
    fq12 a = cyclotomic_exp(g, h1, 126);                        // g^h1
    fq12 b = fq12_mul(fq12_conj(cyclotomic_exp_xabs(a)), fq12_frob(a));       // a^(x + p), x < 0
    fq12 bx2 = cyclotomic_exp_xabs(cyclotomic_exp_xabs(b));                  // b^(x^2)
    fq12 c = fq12_mul(fq12_mul(bx2, fq12_frob2(b)), fq12_conj(b));          // b^(x^2 + p^2 - 1)
    return fq12_mul(c, g);
}
