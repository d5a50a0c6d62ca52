// Fq12 arithmetic spread over a group of 8 lanes, for the latency-bound pairing steps.
//
// Fq12 is viewed flat as Fq2[w]/(w^6 - xi) (xi = 1 + u): f = sum_k f_k w^k, and lane k (k < 6) of the
// group owns f_k; lanes 6 and 7 run the same instruction stream on dummy data, so every lane of
// the warp executes the same code (no divergence).  Lanes exchange coefficients through a
// per-group shared-memory buffer of 8 Fq2 values, with __syncwarp() as the barrier (all groups of a
// warp execute the same sequence).  Flat index k of w^k maps to the tower as
//   k = 0,2,4 -> c0.c0, c0.c1, c0.c2 and k = 1,3,5 -> c1.c0, c1.c1, c1.c2   (v = w^2).
// A product c = a b has c_k = sum_i a_i b_{k-i} with b_{k-i} taken mod 6 and a factor xi when
// i > k (w^6 = xi): six Fq2 products per lane instead of eighteen in sequence.
#pragma once
#include "pairing.cuh"

struct G12 {
    int k;          // lane within the group (0..7); coefficient index for k < 6
    fq2* x;         // this group's exchange buffer: 8 Fq2
};

FPG_DEV void gsync() { __syncwarp(); }

// tower position (0..5 in c0.c0, c0.c1, c0.c2, c1.c0, c1.c1, c1.c2 order) of flat index k
FPG_DEV int g_tower_pos(int k) { return (k & 1) ? 3 + (k >> 1) : (k >> 1); }

FPG_DEV fq2 g_load(const fq12& f, int k) {
    const fq2* c = &f.c0.c0;              // fq12 is six consecutive fq2 in tower order
    return c[g_tower_pos(k < 6 ? k : 0)];
}
FPG_DEV void g_store(fq12& f, int k, const fq2& v) {
    fq2* c = &f.c0.c0;
    if (k < 6) c[g_tower_pos(k)] = v;
}

// publish v and return after every lane of the warp has published
FPG_DEV void g_pub(const G12& g, const fq2& v) {
    gsync();
    g.x[g.k] = v;
    gsync();
}

FPG_DEV fq2 fq2_select(bool c, const fq2& a, const fq2& b) {
    fq2 r;
#pragma unroll
    for (int j = 0; j < 12; j++) {
        r.c0.v[j] = c ? a.c0.v[j] : b.c0.v[j];
        r.c1.v[j] = c ? a.c1.v[j] : b.c1.v[j];
    }
    return r;
}

// c = a * b where this lane holds a_k and b_k
FPG_NOINL fq2 g_mul(const G12& g, fq2* ybuf, const fq2& ak, const fq2& bk) {
    gsync();
    g.x[g.k] = ak;
    ybuf[g.k] = bk;
    gsync();
    const int k = g.k < 6 ? g.k : 0;
    fq2 acc, hi;
    fq2_zero(acc);
    fq2_zero(hi);
#pragma unroll 1
    for (int i = 0; i < 6; i++) {
        int j = k - i;
        const bool wrap = j < 0;
        if (wrap) j += 6;
        const fq2 p = fq2_mul(g.x[i], ybuf[j]);
        const fq2 s = fq2_add(wrap ? hi : acc, p);       // same instructions in every lane
        hi = wrap ? s : hi;
        acc = wrap ? acc : s;
    }
    return fq2_add(acc, fq2_mul_xi(hi));
}

// Granger-Scott squaring in the cyclotomic subgroup: pairs (z0, z3), (z1, z4), (z2, z5) are Fq4
// elements a + b s (s = w^3, s^2 = xi); with A_p = a^2 + xi b^2 and B_p = 2ab for pair p:
//   c0 = 3 A0 - 2 z0, c3 = 3 B0 + 2 z3, c1 = 3 xi B2 + 2 z1, c4 = 3 A2 - 2 z4,
//   c2 = 3 A1 - 2 z2, c5 = 3 B1 + 2 z5.
FPG_NOINL fq2 g_cyc_sqr(const G12& g, const fq2& zk) {
    g_pub(g, zk);
    const int k = g.k < 6 ? g.k : 0;
    const bool a_lane = k < 3;
    const int p = a_lane ? k : k - 3;
    // lanes 0..2: A_p = z_p^2 + xi z_{p+3}^2; lanes 3..5: B_p = 2 z_p z_{p+3}
    const fq2 zp = g.x[p], zq = g.x[p + 3];
    const fq2 u = fq2_mul(a_lane ? zp : zp, a_lane ? zp : zq);
    const fq2 v = fq2_mul(zq, zq);
    const fq2 res = a_lane ? fq2_add(u, fq2_mul_xi(v)) : fq2_dbl(u);
    g_pub(g, res);
    // lane k takes V from lane src(k) = {0, 5, 1, 3, 2, 4}[k]
    const int src = (k == 0) ? 0 : (k == 1) ? 5 : (k == 2) ? 1 : (k == 3) ? 3 : (k == 4) ? 2 : 4;
    fq2 V = g.x[src];
    if (k == 1) V = fq2_mul_xi(V);
    const fq2 V3 = fq2_add(fq2_dbl(V), V);
    const fq2 z2 = fq2_dbl(zk);
    return (k & 1) ? fq2_add(V3, z2) : fq2_sub(V3, z2);
}

FPG_DEV fq2 g_conj(const G12& g, const fq2& zk) { return (g.k & 1) ? fq2_neg(zk) : zk; }

FPG_DEV fq2 g_frob(const G12& g, const fq2& zk) {
    const int k = g.k < 6 ? g.k : 0;
    return k == 0 ? fq2_conj(zk) : fq2_mul(fq2_conj(zk), frob1_coef(k));
}
FPG_DEV fq2 g_frob2(const G12& g, const fq2& zk) {
    const int k = g.k < 6 ? g.k : 0;
    return k == 0 ? zk : fq2_mul_fq(zk, frob2_coef(k));
}

// a^e for a in the cyclotomic subgroup, e given as little-endian words (same e in every lane)
FPG_NOINL fq2 g_cyc_exp(const G12& g, fq2* ybuf, const fq2& ak, const uint32_t* e, int bits) {
    fq2 acc = ak;
    int i = bits - 1;
    while (i >= 0 && !((e[i >> 5] >> (i & 31)) & 1)) i--;
    for (i = i - 1; i >= 0; i--) {
        acc = g_cyc_sqr(g, acc);
        if ((e[i >> 5] >> (i & 31)) & 1) acc = g_mul(g, ybuf, acc, ak);
    }
    return acc;
}
FPG_DEV fq2 g_exp_xabs(const G12& g, fq2* ybuf, const fq2& ak) {
    uint32_t e[2] = {(uint32_t)BLS_X_ABS, (uint32_t)(BLS_X_ABS >> 32)};
    return g_cyc_exp(g, ybuf, ak, e, 64);
}

// f^((p^12 - 1)/r) for the Fq12 whose flat coefficient k this lane holds (see final_exp)
FPG_NOINL fq2 g_final_exp(const G12& g, fq2* ybuf, const fq2& fk) {
    // easy part: t = conj(f) f^-1 (the inverse is computed redundantly by every lane), g = t^(p^2) t
    g_pub(g, fk);
    fq12 f;
    for (int j = 0; j < 6; j++) g_store(f, j, g.x[j]);
    const fq12 fi = fq12_inv(f);
    const fq2 t = g_mul(g, ybuf, g_conj(g, fk), g_load(fi, g.k));
    const fq2 gg = g_mul(g, ybuf, g_frob2(g, t), t);
    // hard part: d = h1 (x + p)(x^2 + p^2 - 1) + 1
    const uint32_t h1[4] = {BLS_H1[0], BLS_H1[1], BLS_H1[2], BLS_H1[3]};
    const fq2 a = g_cyc_exp(g, ybuf, gg, h1, 126);
    const fq2 b = g_mul(g, ybuf, g_conj(g, g_exp_xabs(g, ybuf, a)), g_frob(g, a));
    const fq2 bx2 = g_exp_xabs(g, ybuf, g_exp_xabs(g, ybuf, b));
    const fq2 c = g_mul(g, ybuf, g_mul(g, ybuf, bx2, g_frob2(g, b)), g_conj(g, b));
    return g_mul(g, ybuf, c, gg);
}

// ---------------------------------------------------------------------------------------
// Miller loop on a group of 8 lanes (same line formulas as miller_loop in pairing.cuh).
// Each doubling step runs in three uniform phases:
//   1. every lane: its coefficient of f^2 (four Fq2 products, table below) and one of the
//      five products X^2, Y^2, Z^2, YZ, XY of the running point T;
//   2. lanes 0..5: one product each: l2 = -3 xP X^2, l3 = 2 yP YZ, 2XY (Y^2 - 9b'Z^2),
//      (Y^2 + 9b'Z^2)^2, (b'Z^2)^2, Y^2 YZ;
//   3. every lane: its coefficient of f^2 * line (three products); T <- 2T.
// The addition step with Q runs in four such phases.  T and the products live in shared memory.
// ---------------------------------------------------------------------------------------
struct GMill {
    fq2 fx[8];      // published f coefficients
    fq2 sc[16];     // step products
    fq2 T[3];       // X, Y, Z of the running point
};

// (f^2)_k = sum_t scale * f_a f_b, scale: 0 none, 1 x1, 2 x2, 3 x xi, 4 x 2 xi  (w^6 = xi)
__constant__ int8_t G_SQR_TAB[6][4][3] = {
    {{0, 0, 1}, {3, 3, 3}, {1, 5, 4}, {2, 4, 4}},
    {{0, 1, 2}, {2, 5, 4}, {3, 4, 4}, {0, 0, 0}},
    {{0, 2, 2}, {1, 1, 1}, {3, 5, 4}, {4, 4, 3}},
    {{0, 3, 2}, {1, 2, 2}, {4, 5, 4}, {0, 0, 0}},
    {{0, 4, 2}, {1, 3, 2}, {2, 2, 1}, {5, 5, 3}},
    {{0, 5, 2}, {1, 4, 2}, {2, 3, 2}, {0, 0, 0}}};

FPG_DEV fq2 fq2_from_fq(const fq& a) { fq2 r; r.c0 = a; fq_zero(r.c1); return r; }

FPG_DEV void gm_publish(GMill& sm, int lane, const fq2& fk) {
    gsync();
    sm.fx[lane] = fk;
    gsync();
}

// lane's coefficient of f * (l0 + l2 w^2 + l3 w^3), f already published in sm.fx
FPG_DEV fq2 gm_line_mul(const GMill& sm, int k, const fq2& fk, const fq2& l0, const fq2& l2, const fq2& l3) {
    fq2 t = fq2_mul(fk, l0);
    fq2 u = fq2_mul(sm.fx[(k + 4) % 6], l2);
    fq2 v = fq2_mul(sm.fx[(k + 3) % 6], l3);
    u = k < 2 ? fq2_mul_xi(u) : u;
    v = k < 3 ? fq2_mul_xi(v) : v;
    return fq2_add(fq2_add(t, u), v);
}

FPG_NOINL fq2 gm_double(GMill& sm, int lane, const fq2& fk, const fq& m3x, const fq& y2) {
    const int k = lane < 6 ? lane : 0;
    // phase 1: f^2 and the T products
    gm_publish(sm, lane, fk);
    fq2 sq;
    fq2_zero(sq);
#pragma unroll 1
    for (int t = 0; t < 4; t++) {
        const int a = G_SQR_TAB[k][t][0], b = G_SQR_TAB[k][t][1], s = G_SQR_TAB[k][t][2];
        fq2 p = fq2_mul(sm.fx[a], sm.fx[b]);
        p = (s >= 3) ? fq2_mul_xi(p) : p;
        p = (s == 2 || s == 4) ? fq2_dbl(p) : p;
        sq = s ? fq2_add(sq, p) : sq;
    }
    const int tk = lane < 5 ? lane : 0;
    const int ia = (tk == 0 || tk == 4) ? 0 : (tk == 2 ? 2 : 1);      // X X, Y Y, Z Z, Y Z, X Y
    const int ib = (tk == 0) ? 0 : (tk == 1 ? 1 : (tk == 4 ? 1 : 2));
    const fq2 tp = fq2_mul(sm.T[ia], sm.T[ib]);
    gsync();
    if (lane < 5) sm.sc[lane] = tp;
    gsync();
    // phase 2
    const fq2 XX = sm.sc[0], YY = sm.sc[1], ZZ = sm.sc[2], YZ = sm.sc[3], XY = sm.sc[4];
    const fq2 bz = mul_bprime(ZZ);
    const fq2 bz3 = fq2_add(fq2_dbl(bz), bz);
    const fq2 bz9 = fq2_add(fq2_dbl(bz3), bz3);
    fq2 a, b;
    switch (k) {
        case 0: a = XX; b = fq2_from_fq(m3x); break;
        case 1: a = YZ; b = fq2_from_fq(y2); break;
        case 2: a = fq2_dbl(XY); b = fq2_sub(YY, bz9); break;
        case 3: a = fq2_add(YY, bz9); b = a; break;
        case 4: a = bz; b = bz; break;
        default: a = YY; b = YZ; break;
    }
    const fq2 r = fq2_mul(a, b);
    gsync();
    if (lane < 6) sm.sc[8 + lane] = r;
    gm_publish(sm, lane, sq);
    // phase 3: f^2 * line, T <- 2T
    const fq2 c = gm_line_mul(sm, k, sq, fq2_sub(YY, bz3), sm.sc[8], sm.sc[9]);
    const fq2 nX = sm.sc[10];
    const fq2 nY = fq2_sub(sm.sc[11], fq2_mul_small(sm.sc[12], 108));
    const fq2 nZ = fq2_dbl(fq2_dbl(fq2_dbl(sm.sc[13])));
    gsync();
    if (lane == 0) { sm.T[0] = nX; sm.T[1] = nY; sm.T[2] = nZ; }
    gsync();
    return c;
}

FPG_NOINL fq2 gm_add(GMill& sm, int lane, const fq2& fk, const fq2& xQ, const fq2& yQ, const fq& xP, const fq& yP) {
    const int k = lane < 6 ? lane : 0;
    const fq2 X = sm.T[0], Y = sm.T[1], Z = sm.T[2];
    // phase A: yQ Z, xQ Z
    const fq2 pa = fq2_mul(k == 1 ? xQ : yQ, Z);
    gsync();
    if (lane < 2) sm.sc[lane] = pa;
    gsync();
    const fq2 th = fq2_sub(Y, sm.sc[0]), la = fq2_sub(X, sm.sc[1]);
    // phase B: th xQ, la yQ, -th xP, la yP, th^2, la^2
    fq2 a, b;
    switch (k) {
        case 0: a = th; b = xQ; break;
        case 1: a = la; b = yQ; break;
        case 2: a = th; b = fq2_from_fq(fq_neg(xP)); break;
        case 3: a = la; b = fq2_from_fq(yP); break;
        case 4: a = th; b = th; break;
        default: a = la; b = la; break;
    }
    const fq2 pb = fq2_mul(a, b);
    gsync();
    if (lane < 6) sm.sc[8 + lane] = pb;
    gm_publish(sm, lane, fk);
    const fq2 l0 = fq2_sub(sm.sc[8], sm.sc[9]), l2 = sm.sc[10], l3 = sm.sc[11], C = sm.sc[12], D = sm.sc[13];
    // phase C: line product, and E = D la, F = Z C, G = X D
    const fq2 c = gm_line_mul(sm, k, fk, l0, l2, l3);
    const int ek = lane < 3 ? lane : 0;
    const fq2 pc = fq2_mul(ek == 0 ? D : (ek == 1 ? Z : X), ek == 0 ? la : (ek == 1 ? C : D));
    gsync();
    if (lane < 3) sm.sc[lane] = pc;
    gsync();
    const fq2 E = sm.sc[0], F = sm.sc[1], G = sm.sc[2];
    const fq2 H = fq2_sub(fq2_add(E, F), fq2_dbl(G));
    // phase D: la H, th (G - H), Y E, Z E
    const int dk = lane < 4 ? lane : 0;
    const fq2 pd = fq2_mul(dk == 0 ? la : (dk == 1 ? th : (dk == 2 ? Y : Z)),
                           dk == 0 ? H : (dk == 1 ? fq2_sub(G, H) : E));
    gsync();
    if (lane < 4) sm.sc[8 + lane] = pd;
    gsync();
    const fq2 nX = sm.sc[8], nY = fq2_sub(sm.sc[9], sm.sc[10]), nZ = sm.sc[11];
    gsync();
    if (lane == 0) { sm.T[0] = nX; sm.T[1] = nY; sm.T[2] = nZ; }
    gsync();
    return c;
}

// lane's flat coefficient of conj(f_{|x|,Q}(P)); the identity when P or Q is (then the loop runs on
// the generators so that every group of the warp executes the same code, and its value is dropped)
FPG_NOINL fq2 g_miller(GMill& sm, int lane, g1a P, g2a Q) {
    const bool inf = g1a_is_inf(P) || g2a_is_inf(Q);
    if (inf) { P = g1_generator(); Q = g2_generator(); }
    const fq m3x = fq_neg(fq_add(fq_dbl(P.x), P.x)), y2 = fq_dbl(P.y);
    gsync();
    if (lane == 0) { sm.T[0] = Q.x; sm.T[1] = Q.y; fq2_one(sm.T[2]); }
    gsync();
    fq2 fk;
    if (lane == 0) fq2_one(fk); else fq2_zero(fk);
    for (int i = 62; i >= 0; i--) {
        fk = gm_double(sm, lane, fk, m3x, y2);
        if ((BLS_X_ABS >> i) & 1) fk = gm_add(sm, lane, fk, Q.x, Q.y, P.x, P.y);
    }
    fk = (lane & 1) ? fq2_neg(fk) : fk;                 // conjugation (x < 0)
    if (inf) { if (lane == 0) fq2_one(fk); else fq2_zero(fk); }
    return fk;
}
