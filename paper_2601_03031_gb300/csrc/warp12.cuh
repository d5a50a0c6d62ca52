// Fq12 arithmetic on one warp: the Fq products of an operation are spread one per lane and round.
//
// A Montgomery product is ~700 multiply-add instructions that one warp issues at the integer
// pipe's rate whatever their dependency structure, so a single lane cannot make one faster; what
// shortens a chain of Fq12 operations is doing all of an operation's products at once.  Values
// live in shared memory, flat as Fq2[w]/(w^6 - xi) (xi = 1 + u): Fq index 2k + e holds component
// e (0 = real, 1 = u) of the coefficient of w^k, k = 0..5 (w^2 = v, so flat k = 0,2,4 are the tower's
// c0.c0, c0.c1, c0.c2 and k = 1,3,5 are c1.c0, c1.c1, c1.c2).  Every operation is
//   1. products: lane L computes products L, L + 32, ... of the operation's list,
//   2. __syncwarp, then 12 (or 24) lanes form the output Fq components as sums of products,
//   3. __syncwarp.
// All lanes of an engine run every operation (no lane-dependent synchronisation).  An engine is one
// warp (NW = 1) or one 128-thread block (NW = 4: a product's 108 Fq products take one round).
//   product c = a b:        36 Fq2 products a_i b_j, each 3 Fq products (Karatsuba): 108
//   cyclotomic squaring:    Granger-Scott, 3 Fq4 squarings of 7 Fq products each: 21
//   Frobenius p / p^2:      20 / 10 Fq products by constants
#pragma once
#include "pairing.cuh"
#include "fq_split.cuh"

struct W12 {
    fq p[108];          // products of the current operation
    fq s[5][12];        // value slots (flat order)
    fq h[24];           // partial sums
};

// NW = 1: one engine per warp (__syncwarp); NW = 4: one engine per 128-thread block (__syncthreads)
template <int NW>
FPG_DEV void wsync() {
    if (NW == 1) __syncwarp();
    else __syncthreads();
}
template <int NW>
FPG_DEV int w_lane() { return (int)(threadIdx.x & (32 * NW - 1)); }

// tower position of flat coefficient k (0..5): even k -> c0.c(k/2), odd k -> c1.c(k/2)
FPG_DEV int w_tower_pos(int k) { return (k & 1) ? 3 + (k >> 1) : (k >> 1); }



// dst (flat) <- f (tower order: six consecutive Fq2, each (c0, c1))
template <int NW>
FPG_DEV void w_from_tower(fq* dst, const fq12& f) {
    const int L = w_lane<NW>();
    if (L < 12) dst[L] = reinterpret_cast<const fq*>(&f)[2 * w_tower_pos(L >> 1) + (L & 1)];
    wsync<NW>();
}
template <int NW>
FPG_DEV void w_copy(fq* dst, const fq* src) {
    const int L = w_lane<NW>();
    wsync<NW>();
    if (L < 12) dst[L] = src[L];
    wsync<NW>();
}

// out = a b (out may alias a or b)
template <int NW>
FPG_NOINL void w_mul(W12& W, fq* out, const fq* a, const fq* b) {
    const int L = w_lane<NW>();
    fq zero;
    fq_zero(zero);
    for (int t = L; t < 108; t += 32 * NW) {
        const int q = t / 3, kind = t - 3 * q, i = q / 6, j = q - 6 * i;
        // kind 0: a_i.0 b_j.0, kind 1: a_i.1 b_j.1, kind 2: (a_i.0 + a_i.1)(b_j.0 + b_j.1)
        const fq x = fq_add(a[2 * i + (kind == 1)], fq_select(kind == 2, a[2 * i + 1], zero));
        const fq y = fq_add(b[2 * j + (kind == 1)], fq_select(kind == 2, b[2 * j + 1], zero));
        W.p[t] = fq_mul(x, y);
    }
    wsync<NW>();
    // lane L < 24: output component o = L % 12 (coefficient k, part e), terms i in [3 hf, 3 hf + 3)
    if (L < 24) {
        const int o = L % 12, hf = L / 12, k = o >> 1, e = o & 1;
        fq acc = zero;
        for (int i = 3 * hf; i < 3 * hf + 3; i++) {
            int j = k - i;
            const bool wrap = j < 0;                 // w^(i + j) with i + j >= 6: times xi
            if (wrap) j += 6;
            const fq* m = &W.p[3 * (6 * i + j)];
            const fq m01 = fq_add(m[0], m[1]);
            const fq re = fq_sub(m[0], m[1]);
            const fq im = fq_sub(m[2], m01);
            // (re + im u)(1 + u) = (re - im) + (re + im) u
            const fq x = fq_select(wrap, fq_select(e, fq_add(re, im), fq_sub(re, im)), fq_select(e, im, re));
            acc = fq_add(acc, x);
        }
        W.h[L] = acc;
    }
    wsync<NW>();
    if (L < 12) out[L] = fq_add(W.h[L], W.h[L + 12]);
    wsync<NW>();
}

// out = a^2 for a in the cyclotomic subgroup (Granger-Scott).  Pairs (z_p, z_{p+3}), p = 0, 1, 2,
// are Fq4 elements a + b s (s = w^3, s^2 = xi): A_p = a^2 + xi b^2, B_p = 2 a b, and
//   c0 = 3 A0 - 2 z0, c3 = 3 B0 + 2 z3, c1 = 3 xi B2 + 2 z1, c4 = 3 A2 - 2 z4, c2 = 3 A1 - 2 z2,
//   c5 = 3 B1 + 2 z5.
// Products per pair (a = a0 + a1 u, b = b0 + b1 u): s1 = (a0 + a1)(a0 - a1), s2 = a0 a1,
// t1 = (b0 + b1)(b0 - b1), t2 = b0 b1, k0 = a0 b0, k1 = a1 b1, k2 = (a0 + a1)(b0 + b1); then
// a^2 = s1 + 2 s2 u, b^2 = t1 + 2 t2 u, a b = (k0 - k1) + (k2 - k0 - k1) u.
template <int NW>
FPG_DEV void w_cyc_sqr(W12& W, fq* out, const fq* z) {
    const int L = w_lane<NW>();
    // the block engine splits each product over its four warps (fq_split.cuh): lane t of every warp
    // forms the operands of product t (lanes t >= 21 those of product 0, discarded)
    if (NW == 4 || L < 21) {
        const int tp = NW == 4 ? ((L & 31) < 21 ? (L & 31) : 0) : L;
        const int p = tp / 7, r = tp - 7 * p;
        const fq a0 = z[2 * p], a1 = z[2 * p + 1], b0 = z[2 * p + 6], b1 = z[2 * p + 7];
        const bool ua = r < 2 || r == 4 || r == 5 || r == 6;            // x built from a
        const fq xs = fq_select(ua, a0, b0), xt = fq_select(ua, a1, b1);
        // x: r in {0, 2, 6}: xs + xt; r in {1, 3, 4}: xs; r == 5: a1
        const fq xsum = fq_add(xs, xt);
        const fq x = fq_select(r == 0 || r == 2 || r == 6, xsum, fq_select(r == 5, a1, xs));
        // y: r == 0: a0 - a1; r == 1: a1; r == 2: b0 - b1; r == 3: b1; r == 4: b0; r == 5: b1;
        //    r == 6: b0 + b1
        const fq ys = fq_select(r < 2, a0, b0), yt = fq_select(r < 2, a1, b1);
        const fq ydiff = fq_sub(ys, yt), ysum = fq_add(ys, yt);
        const fq y = fq_select(r == 0 || r == 2, ydiff,
                               fq_select(r == 6, ysum, fq_select(r == 4, b0, fq_select(r == 1, a1, b1))));
        if (NW == 4) {
            const fq m = fq_mul_split(x, y);
            if (L < 21) W.p[L] = m;
        } else {
            W.p[L] = fq_mul(x, y);
        }
    }
    wsync<NW>();
    if (NW == 4) {
        // each output from its pair's products in one step, one formula per warp (no divergence):
        //   warp 0: c0, c2, c4 real parts  3 (s1 + t1 - 2 t2) - 2 z
        //   warp 1: c0, c2, c4 imag parts  3 (t1 + 2 (s2 + t2)) - 2 z
        //   warp 2: c3.re, c5.re  3 (2 (k0 - k1)) + 2 z;  c1.re = 3 (2 (2 k0 - k2)) + 2 z
        //   warp 3: c3.im, c5.im  3 (2 (k2 - k0 - k1)) + 2 z;  c1.im = 3 (2 (k2 - 2 k1)) + 2 z
        const int w = L >> 5, pl = L & 31;
        if (pl < 3) {
            const fq* m = &W.p[7 * pl];
            int o;
            fq V;
            if (w == 0) {
                o = 4 * pl;
                V = fq_sub(fq_add(m[0], m[2]), fq_dbl(m[3]));
            } else if (w == 1) {
                o = 4 * pl + 1;
                V = fq_add(m[2], fq_dbl(fq_add(m[1], m[3])));
            } else if (w == 2) {
                o = pl == 2 ? 2 : 6 + 4 * pl;
                const fq k0 = m[4];
                const fq u = fq_select(pl == 2, fq_dbl(k0), k0);
                V = fq_dbl(fq_sub(u, fq_select(pl == 2, m[6], m[5])));
            } else {
                o = pl == 2 ? 3 : 7 + 4 * pl;
                const fq y = fq_select(pl == 2, fq_dbl(m[5]), fq_add(m[4], m[5]));
                V = fq_dbl(fq_sub(m[6], y));
            }
            const fq V3 = fq_add(fq_dbl(V), V);
            const fq z2 = fq_dbl(z[o]);
            out[o] = w < 2 ? fq_sub(V3, z2) : fq_add(V3, z2);
        }
        wsync<NW>();
        return;
    } else if (L < 12) {
        const int k = L >> 1, e = L & 1;
        // coefficient k -> (pair, kind): kind 0: 3A - 2z, 1: 3B + 2z, 2: 3 xi B + 2z
        const int pair = (k == 0 || k == 3) ? 0 : (k == 2 || k == 5) ? 1 : 2;
        const int kind = (k == 0 || k == 2 || k == 4) ? 0 : (k == 1 ? 2 : 1);
        const fq* m = &W.p[7 * pair];
        const fq s1 = m[0], s2 = m[1], t1 = m[2], t2 = m[3], k0 = m[4], k1 = m[5], k2 = m[6];
        const fq t2d = fq_dbl(t2);
        const fq Are = fq_sub(fq_add(s1, t1), t2d);
        const fq Aim = fq_add(fq_add(fq_dbl(s2), t1), t2d);
        const fq Bre = fq_dbl(fq_sub(k0, k1));
        const fq Bim = fq_dbl(fq_sub(k2, fq_add(k0, k1)));
        const fq V = fq_select(kind == 0, fq_select(e, Aim, Are),
                               fq_select(kind == 1, fq_select(e, Bim, Bre),
                                         fq_select(e, fq_add(Bre, Bim), fq_sub(Bre, Bim))));
        const fq V3 = fq_add(fq_dbl(V), V);
        const fq z2 = fq_dbl(z[L]);
        W.h[L] = fq_select(kind == 0, fq_sub(V3, z2), fq_add(V3, z2));
    }
    wsync<NW>();
    if (L < 12) out[L] = W.h[L];
    wsync<NW>();
}

// out = conj(a) = a^(p^6): coefficients of odd k negated
template <int NW>
FPG_DEV void w_conj(fq* out, const fq* a) {
    const int L = w_lane<NW>();
    wsync<NW>();
    if (L < 12) {
        const fq v = a[L];
        out[L] = fq_select((L >> 1) & 1, fq_neg(v), v);
    }
    wsync<NW>();
}

// out = a^p: coefficient k -> conj(a_k) gamma1_k (gamma1_0 = 1);
// (x0 - x1 u)(g0 + g1 u) = (x0 g0 + x1 g1) + (x0 g1 - x1 g0) u
template <int NW>
FPG_NOINL void w_frob(W12& W, fq* out, const fq* a) {
    const int L = w_lane<NW>();
    if (L < 20) {
        const int k = 1 + (L >> 2), r = L & 3;
        const fq2 g = frob1_coef(k);
        const fq x = fq_select(r == 0 || r == 2, a[2 * k], a[2 * k + 1]);
        const fq y = fq_select(r == 0 || r == 3, g.c0, g.c1);
        W.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    if (L < 12) {
        const int k = L >> 1, e = L & 1;
        const fq* m = &W.p[4 * (k ? k - 1 : 0)];
        W.h[L] = fq_select(k == 0, fq_select(e, fq_neg(a[1]), a[0]),
                           fq_select(e, fq_sub(m[2], m[3]), fq_add(m[0], m[1])));
    }
    wsync<NW>();
    if (L < 12) out[L] = W.h[L];
    wsync<NW>();
}

// out = a^(p^2): coefficient k times gamma2_k in Fq (gamma2_0 = 1)
template <int NW>
FPG_NOINL void w_frob2(W12& W, fq* out, const fq* a) {
    const int L = w_lane<NW>();
    if (L < 10) {
        const int k = 1 + (L >> 1);
        W.p[L] = fq_mul(a[2 * k + (L & 1)], frob2_coef(k));
    }
    wsync<NW>();
    if (L < 12) W.h[L] = fq_select(L < 2, a[L < 2 ? L : 0], W.p[L < 2 ? 0 : L - 2]);
    wsync<NW>();
    if (L < 12) out[L] = W.h[L];
    wsync<NW>();
}

// a <- a^-1 for a in Fq2 (flat coefficient 0; the others are zero), on the quad of lanes 0 .. 3
template <int NW>
FPG_NOINL void w_inv_fq2(fq* a) {
    const int L = w_lane<NW>();
    wsync<NW>();
    if (L < 4) {
        const fq2 v{a[0], a[1]};
        const fq2 vi = fq2_inv_quad(v);
        if (L == 0) {
            a[0] = vi.c0;
            a[1] = vi.c1;
        }
    }
    wsync<NW>();
}

// acc = base^e for base in the cyclotomic subgroup (e little-endian words, e > 0); acc != base
template <int NW>
FPG_NOINL void w_cyc_exp(W12& W, fq* acc, const fq* base, const uint32_t* e, int bits) {
    int i = bits - 1;
    while (i >= 0 && !((e[i >> 5] >> (i & 31)) & 1)) i--;
    w_copy<NW>(acc, base);
    for (i = i - 1; i >= 0; i--) {
        w_cyc_sqr<NW>(W, acc, acc);
        if ((e[i >> 5] >> (i & 31)) & 1) w_mul<NW>(W, acc, acc, base);
    }
}

// acc = base^e for base in the cyclotomic subgroup and e > 0 given by its width-4 NAF (d[0] least
// significant, n digits, the top one positive): base, base^3, base^5, base^7 (t3, t5, t7 hold the
// powers; acc, base, t3, t5, t7 distinct slots), then a squaring per digit and a product per nonzero
// digit; a negative digit multiplies by the inverse, which in the cyclotomic subgroup is the
// conjugate: acc T^-1 = conj(conj(acc) T)
template <int NW>
FPG_NOINL void w_cyc_exp_wnaf4(W12& W, fq* acc, const fq* base, fq* t3, fq* t5, fq* t7, const signed char* d,
                               int n) {
    w_cyc_sqr<NW>(W, acc, base);            // base^2
    w_mul<NW>(W, t3, acc, base);
    w_mul<NW>(W, t5, t3, acc);
    w_mul<NW>(W, t7, t5, acc);
    const int top = d[n - 1];
    w_copy<NW>(acc, top == 1 ? base : top == 3 ? t3 : top == 5 ? t5 : t7);
    for (int i = n - 2; i >= 0; i--) {
        w_cyc_sqr<NW>(W, acc, acc);
        const int di = d[i];
        if (di) {
            const int a = di < 0 ? -di : di;
            const fq* T = a == 1 ? base : a == 3 ? t3 : a == 5 ? t5 : t7;
            if (di < 0) w_conj<NW>(acc, acc);
            w_mul<NW>(W, acc, acc, T);
            if (di < 0) w_conj<NW>(acc, acc);
        }
    }
}

// slot 2 <- f^((p^12 - 1)/r) for f in slot 0 (slots 0..4 are used).  Easy part t = conj(f) f^-1,
// g = t^(p^2) t; hard part g^d with d = h1 (x + p)(x^2 + p^2 - 1) + 1, h1 = (x - 1)^2 / 3, x < 0.
// The inverse goes through norms: n = f conj(f) lies in Fq6, u = n^(p^2) n^(p^4), and n u is the
// norm of n to Fq2, so f^-1 = conj(f) / n = conj(f) u / (n u) and t = conj(f)^2 u (n u)^-1: six
// lane-parallel Fq12 products, two Frobenius maps and one Fq2 inversion on a quad of lanes.  g^h1 runs on
// the width-4 NAF of h1 (24 nonzero digits instead of 48 set bits).
template <int NW>
FPG_NOINL void w_final_exp(W12& W) {
    fq* s0 = W.s[0];
    fq* s1 = W.s[1];
    fq* s2 = W.s[2];
    fq* s3 = W.s[3];
    fq* s4 = W.s[4];
    const uint32_t xabs[2] = {(uint32_t)BLS_X_ABS, (uint32_t)(BLS_X_ABS >> 32)};
    w_conj<NW>(s1, s0);                     // c = conj(f)
    w_mul<NW>(W, s2, s0, s1);               // n = f c, in Fq6
    w_frob2<NW>(W, s3, s2);
    w_frob2<NW>(W, s4, s3);
    w_mul<NW>(W, s3, s3, s4);               // u = n^(p^2 + p^4)
    w_mul<NW>(W, s4, s2, s3);               // n u, in Fq2
    w_inv_fq2<NW>(s4);
    w_mul<NW>(W, s2, s1, s1);
    w_mul<NW>(W, s2, s2, s3);
    w_mul<NW>(W, s2, s2, s4);               // t = c^2 u (n u)^-1 = conj(f) f^-1
    w_frob2<NW>(W, s3, s2);
    w_mul<NW>(W, s3, s3, s2);               // g = t^(p^2) t
    w_cyc_exp_wnaf4<NW>(W, s4, s3, s0, s1, s2, BLS_H1_WNAF, BLS_H1_WNAF_LEN);   // a = g^h1
    w_cyc_exp<NW>(W, s0, s4, xabs, 64);     // a^|x|
    w_conj<NW>(s0, s0);                     // a^x
    w_frob<NW>(W, s1, s4);                  // a^p
    w_mul<NW>(W, s0, s0, s1);               // b = a^(x + p)
    w_cyc_exp<NW>(W, s1, s0, xabs, 64);
    w_cyc_exp<NW>(W, s2, s1, xabs, 64);     // b^(x^2)
    w_frob2<NW>(W, s1, s0);
    w_mul<NW>(W, s2, s2, s1);               // b^(x^2 + p^2)
    w_conj<NW>(s1, s0);
    w_mul<NW>(W, s2, s2, s1);               // c = b^(x^2 + p^2 - 1)
    w_mul<NW>(W, s2, s2, s3);               // c g
}

// ---------------------------------------------------------------------------------------
// Miller loop on one warp: same projective formulas as miller_loop in pairing.cuh.
// Doubling step, T = (X, Y, Z), P with m3x = -3 xP, y2 = 2 yP, b' = 4 xi:
//   line l0 + l2 w^2 + l3 w^3 = (Y^2 - 3 b' Z^2) + (m3x X^2) w^2 + (y2 Y Z) w^3,
//   2T = (2 X Y (Y^2 - 9 b' Z^2), (Y^2 + 9 b' Z^2)^2 - 108 (b' Z^2)^2, 8 Y^2 Y Z),
//   rounds: A = f^2 products (57) + X^2, Y^2, Z^2, YZ, XY (12); B = the line and 2T products
//   (14); C = f^2 * line (54).
// Addition step with Q: theta = Y - yQ Z, lambda = X - xQ Z,
//   line = (theta xQ - lambda yQ) + (-theta xP) w^2 + (lambda yP) w^3,
//   C = theta^2, D = lambda^2, E = D lambda, F = Z C, G = X D, H = E + F - 2G,
//   T + Q = (lambda H, theta (G - H) - Y E, Z E),
//   rounds: A = yQ Z, xQ Z (6); B = line, theta^2, lambda^2 (14); C = f * line (54) + E, F, G
//   (9); D = lambda H, theta (G - H), Y E, Z E (12).
// Fq2 products x y by Karatsuba: m0 = x0 y0, m1 = x1 y1, m2 = (x0 + x1)(y0 + y1),
// re = m0 - m1, im = m2 - m0 - m1; squares x^2: m0 = (x0 + x1)(x0 - x1), m1 = x0 x1, re = m0,
// im = 2 m1.
// ---------------------------------------------------------------------------------------
// The block engine's narrow Miller rounds (up to 15 products) run one product per lane.  Split over
// the four warps (fq_split.cuh) they were slower in the whole ProveAll step (N = 2^16, b = 256: 0.82
// against 0.89 ms per round's Miller loops): the rounds between them are one product per lane on
// three warps anyway, and the split's extra instructions compete with the kernels running beside the
// chain.

struct WMill {
    fq p[72];       // products of a round
    fq f[12];       // running value (flat)
    fq g[12];       // f^2
    fq T[6];        // X, Y, Z
    fq Q[4];        // xQ, yQ
    fq v[28];       // round results: T products, line helpers; 16..27 round B's operands (block engine)
    fq l[6];        // line l0, l2, l3
    fq h[24];
    fq tm[72];      // per-term partial sums of the combines (block-wide engine)
};

// Operands x, y of one Fq product, formed with the same instructions on every lane (the lanes of a
// round do different products; a per-lane branch between formulas would run the formulas one after
// another):
//   mode 0: Karatsuba product of Fq2 values a, b: kind 0: a0 b0, 1: a1 b1, 2: (a0 + a1)(b0 + b1);
//   mode 1: square of a: kind 0: (a0 + a1)(a0 - a1), 1: a0 a1 (b is not read past b[1]: pass a);
//   mode 2: component kind of a times the Fq value s (b as for mode 1).
FPG_DEV void prod_ops(fq& x, fq& y, const fq* a, const fq* b, int kind, int mode, const fq& s) {
    fq zero;
    fq_zero(zero);
    const bool sq = mode == 1, plain = mode == 2;
    const bool with1 = (mode == 0 && kind == 2) || (sq && kind == 0);      // the other component added in
    x = fq_add(a[(mode != 1 && kind == 1) ? 1 : 0], fq_select(with1, a[1], zero));
    const fq* yb = mode == 0 ? b : a;
    const int iy = mode == 0 ? (kind == 1) : (sq ? kind : 0);
    const fq t = fq_select(with1, yb[1], zero);
    y = fq_select(plain, s, fq_select(sq && kind == 0, fq_sub(yb[iy], t), fq_add(yb[iy], t)));
}
FPG_DEV void kara_ops(fq& x, fq& y, const fq* a, const fq* b, int kind) {
    fq zero;
    fq_zero(zero);
    x = fq_add(a[kind == 1], fq_select(kind == 2, a[1], zero));
    y = fq_add(b[kind == 1], fq_select(kind == 2, b[1], zero));
}
FPG_DEV void sq_ops(fq& x, fq& y, const fq* a, int kind) {
    x = fq_select(kind, a[0], fq_add(a[0], a[1]));
    y = fq_select(kind, a[1], fq_sub(a[0], a[1]));
}
// component e of a Karatsuba product / of a square, from its products m
FPG_DEV fq kara_part(const fq* m, int e) {
    return fq_select(e, fq_sub(m[2], fq_add(m[0], m[1])), fq_sub(m[0], m[1]));
}
FPG_DEV fq sq_part(const fq* m, int e) { return fq_select(e, fq_dbl(m[1]), m[0]); }
// component e of (re + im u) times xi = 1 + u when tw
FPG_DEV fq twist_part(const fq& re, const fq& im, int e, bool tw) {
    return fq_select(tw, fq_select(e, fq_add(re, im), fq_sub(re, im)), fq_select(e, im, re));
}
FPG_DEV fq fq_mul_small(const fq& a, unsigned k) {          // k a for a small constant k
    fq acc;
    fq_zero(acc);
    for (int i = 31 - __clz(k); i >= 0; i--) {
        acc = fq_dbl(acc);
        if ((k >> i) & 1) acc = fq_add(acc, a);
    }
    return acc;
}

// f (S.f) times the sparse line (S.l) -> products S.p[0..53]; combine writes S.f
FPG_DEV void wm_line_products(WMill& S, const fq* src, int t) {
    const int q = t / 3, kind = t - 3 * q, term = q / 6, k = q - 6 * term;
    const int i = term == 0 ? k : (term == 1 ? (k + 4) % 6 : (k + 3) % 6);
    fq x, y;
    kara_ops(x, y, src + 2 * i, S.l + 2 * term, kind);
    S.p[t] = fq_mul(x, y);
}
FPG_DEV fq wm_line_combine(const WMill& S, int o) {
    const int k = o >> 1, e = o & 1;
    fq acc = twist_part(kara_part(&S.p[3 * k], 0), kara_part(&S.p[3 * k], 1), e, false);
    acc = fq_add(acc, twist_part(kara_part(&S.p[3 * (6 + k)], 0), kara_part(&S.p[3 * (6 + k)], 1), e, k < 2));
    acc = fq_add(acc, twist_part(kara_part(&S.p[3 * (12 + k)], 0), kara_part(&S.p[3 * (12 + k)], 1), e, k < 3));
    return acc;
}

// block-wide combine of f * line: lane L < 36 forms term L / 12 of output component L % 12
FPG_DEV void wm_line_terms(WMill& S, int L) {
    if (L < 36) {
        const int o = L % 12, term = L / 12, k = o >> 1, e = o & 1;
        const fq* m = &S.p[3 * (6 * term + k)];
        S.tm[L] = twist_part(kara_part(m, 0), kara_part(m, 1), e, (term == 1 && k < 2) || (term == 2 && k < 3));
    }
}
FPG_DEV fq wm_line_sum(const WMill& S, int o) { return fq_add(fq_add(S.tm[o], S.tm[12 + o]), S.tm[24 + o]); }

template <int NW>
FPG_NOINL void wm_dbl(WMill& S, const fq& m3x, const fq& y2) {
    const int L = w_lane<NW>();
    // round A
    for (int t = L; t < 69; t += 32 * NW) {
        const fq* a;
        const fq* b;
        int kind, mode;
        if (t < 12) {                                                            // f_k^2
            a = b = S.f + 2 * (t >> 1);
            kind = t & 1;
            mode = 1;
        } else if (t < 57) {                                                     // f_i f_j, i < j
            const int c = (t - 12) / 3;
            int i = 0, rem = c;
            while (rem >= 5 - i) { rem -= 5 - i; i++; }
            a = S.f + 2 * i;
            b = S.f + 2 * (i + 1 + rem);
            kind = t - 12 - 3 * c;
            mode = 0;
        } else {
            const int u = t - 57;
            if (u < 6) { a = b = S.T + 2 * (u >> 1); kind = u & 1; mode = 1; }  // X^2, Y^2, Z^2
            else if (u < 9) { a = S.T + 2; b = S.T + 4; kind = u - 6; mode = 0; }  // Y Z
            else { a = S.T; b = S.T + 2; kind = u - 9; mode = 0; }                 // X Y
        }
        fq x, y;
        prod_ops(x, y, a, b, kind, mode, m3x);
        S.p[t] = fq_mul(x, y);
    }
    wsync<NW>();
    if (NW == 4 && L < 72) {                       // f^2 terms: lane L -> component L % 12, term i = L / 12
        const int o = L % 12, i = L / 12, k = o >> 1, e = o & 1;
        int j = k - i;
        if (j < 0) j += 6;
        // i == j: the square's parts; i < j: twice the Karatsuba parts; i > j: nothing (the pair is
        // counted once, at i < j)
        const int c = i < j ? i * (11 - i) / 2 + (j - i - 1) : 0;
        const fq* ms = &S.p[2 * i];
        const fq* mk = &S.p[12 + 3 * c];
        const fq re = fq_select(i == j, sq_part(ms, 0), fq_dbl(kara_part(mk, 0)));
        const fq im = fq_select(i == j, sq_part(ms, 1), fq_dbl(kara_part(mk, 1)));
        fq zero;
        fq_zero(zero);
        S.tm[L] = fq_select(i <= j, twist_part(re, im, e, i + j >= 6), zero);
    }
    if (NW == 4 && L >= 96 && L < 106) {           // XX, YY, ZZ, YZ, XY (re, im)
        const int v = L - 96, which = v >> 1, e = v & 1;
        S.v[v] = fq_select(which < 3, sq_part(&S.p[57 + 2 * (which < 3 ? which : 0)], e),
                           kara_part(&S.p[57 + 6 + 3 * (which < 3 ? 0 : which - 3)], e));
    }
    if (NW == 4) {
        wsync<NW>();
        if (L < 12) {
            fq acc = S.tm[L];
            for (int i = 1; i < 6; i++) acc = fq_add(acc, S.tm[12 * i + L]);
            S.g[L] = acc;
        } else if (L >= 96 && L < 108) {
            // beside the sums, warp 3 forms round B's operands from ZZ and YY (re, im each):
            // 16: bz = b' ZZ = 4 (1 + u) ZZ, 18: YY - 9 bz, 20: YY + 9 bz, 22: l0 = YY - 3 bz,
            // 24: 6 bz, 26: 18 bz (so that (6 bz)(18 bz) = 108 bz^2 is a product of round B)
            const int u = L - 96, e = u & 1, kind = u >> 1;
            const fq zr = S.p[61], zi = fq_dbl(S.p[62]);
            const fq bze = fq_dbl(fq_dbl(fq_select(e, fq_add(zr, zi), fq_sub(zr, zi))));
            const fq yy = fq_select(e, fq_dbl(S.p[60]), S.p[59]);
            const fq b3 = fq_add(fq_dbl(bze), bze);
            const fq b9 = fq_add(fq_dbl(b3), b3);
            const fq b6 = fq_dbl(b3);
            // kind 0: bz, 1: YY - 9 bz, 2: YY + 9 bz, 3: YY - 3 bz, 4: 6 bz, 5: 18 bz
            const fq sub_t = fq_select(kind == 1, b9, b3), add_t = fq_select(kind == 2, b9, b6);
            const fq r_sub = fq_sub(yy, sub_t);
            const fq r_add = fq_add(fq_select(kind == 2, yy, fq_dbl(b6)), add_t);   // kind 5: 12 bz + 6 bz
            S.v[16 + u] = fq_select(kind == 0, bze,
                                    fq_select(kind == 1 || kind == 3, r_sub, fq_select(kind == 4, b6, r_add)));
        }
    } else if (L < 12) {                           // f^2, coefficient k, component e
        const int k = L >> 1, e = L & 1;
        fq acc;
        fq_zero(acc);
        for (int i = 0; i < 6; i++) {
            int j = k - i;
            if (j < 0) j += 6;
            if (i > j) continue;
            const bool wrap = i + j >= 6;
            fq re, im;
            if (i == j) {
                re = sq_part(&S.p[2 * i], 0);
                im = sq_part(&S.p[2 * i], 1);
            } else {
                const int c = i * (11 - i) / 2 + (j - i - 1);
                re = fq_dbl(kara_part(&S.p[12 + 3 * c], 0));
                im = fq_dbl(kara_part(&S.p[12 + 3 * c], 1));
            }
            acc = fq_add(acc, twist_part(re, im, e, wrap));
        }
        S.g[L] = acc;
    } else if (NW == 1 && L < 22) {                // XX, YY, ZZ, YZ, XY (re, im)
        const int v = L - 12, which = v >> 1, e = v & 1;
        S.v[v] = which < 3 ? sq_part(&S.p[57 + 2 * which], e) : kara_part(&S.p[57 + 6 + 3 * (which - 3)], e);
    }
    wsync<NW>();
    // round B
    if (NW == 4) {
        if (L < 15) {                               // 15 products, one per lane
            const int t = L;
            const fq* XX = S.v;
            const fq* YY = S.v + 2;
            const fq* YZ = S.v + 6;
            const fq* XY = S.v + 8;
            const fq* a;
            const fq* b;
            int kind, mode;
            if (t < 2) { a = b = XX; kind = t; mode = 2; }                           // m3x XX
            else if (t < 4) { a = b = YZ; kind = t - 2; mode = 2; }                  // y2 YZ
            else if (t < 7) { a = XY; b = S.v + 18; kind = t - 4; mode = 0; }        // XY (YY - 9 bz)
            else if (t < 9) { a = b = S.v + 20; kind = t - 7; mode = 1; }            // (YY + 9 bz)^2
            else if (t < 12) { a = S.v + 24; b = S.v + 26; kind = t - 9; mode = 0; } // 108 bz^2
            else { a = YY; b = YZ; kind = t - 12; mode = 0; }                        // YY YZ
            fq x, y;
            prod_ops(x, y, a, b, kind, mode, fq_select(t < 2, m3x, y2));
            S.p[L] = fq_mul(x, y);
        }
        wsync<NW>();
        // the line (warp 0) and 2T (X' on warp 1, Y' on warp 2, Z' on warp 3)
        const int w = L >> 5, pl = L & 31;
        if (w == 0 && pl < 6) {
            const int e = pl & 1, which = pl >> 1;                      // l0 = YY - 3 bz, l2, l3
            S.l[pl] = fq_select(which == 0, S.v[22 + e], S.p[2 * (which ? which - 1 : 0) + e]);
        } else if (w > 0 && pl < 2) {
            const int e = pl;
            if (w == 1) S.T[e] = fq_dbl(kara_part(&S.p[4], e));
            else if (w == 2) S.T[2 + e] = fq_sub(sq_part(&S.p[7], e), kara_part(&S.p[9], e));
            else S.T[4 + e] = fq_dbl(fq_dbl(fq_dbl(kara_part(&S.p[12], e))));
        }
    } else {
        if (L < 14) {
            const fq* XX = S.v;
            const fq* YY = S.v + 2;
            const fq* ZZ = S.v + 4;
            const fq* YZ = S.v + 6;
            const fq* XY = S.v + 8;
            // bz = b' Z^2 = 4 (1 + u) ZZ
            fq bz[2], bz9[2], yp[2], ym[2];
            bz[0] = fq_dbl(fq_dbl(fq_sub(ZZ[0], ZZ[1])));
            bz[1] = fq_dbl(fq_dbl(fq_add(ZZ[0], ZZ[1])));
            for (int e = 0; e < 2; e++) {
                const fq b3 = fq_add(fq_dbl(bz[e]), bz[e]);
                bz9[e] = fq_add(fq_dbl(b3), b3);
                yp[e] = fq_add(YY[e], bz9[e]);
                ym[e] = fq_sub(YY[e], bz9[e]);
            }
            fq x, y;
            if (L < 2) { x = XX[L]; y = m3x; }
            else if (L < 4) { x = YZ[L - 2]; y = y2; }
            else if (L < 7) kara_ops(x, y, XY, ym, L - 4);
            else if (L < 9) sq_ops(x, y, yp, L - 7);
            else if (L < 11) sq_ops(x, y, bz, L - 9);
            else kara_ops(x, y, YY, YZ, L - 11);
            S.p[L] = fq_mul(x, y);
        }
        wsync<NW>();
        if (L < 12) {
            const int w = L >> 1, e = L & 1;
            fq r;
            if (w == 0) {                               // l0 = YY - 3 bz
                const fq zz0 = S.v[4], zz1 = S.v[5];
                const fq bze = fq_dbl(fq_dbl(e ? fq_add(zz0, zz1) : fq_sub(zz0, zz1)));
                r = fq_sub(S.v[2 + e], fq_add(fq_dbl(bze), bze));
                S.l[e] = r;
            } else if (w == 1) {                        // l2 = m3x XX
                S.l[2 + e] = S.p[e];
            } else if (w == 2) {                        // l3 = y2 YZ
                S.l[4 + e] = S.p[2 + e];
            } else if (w == 3) {                        // X' = 2 XY (YY - 9 bz)
                S.T[e] = fq_dbl(kara_part(&S.p[4], e));
            } else if (w == 4) {                        // Y' = (YY + 9 bz)^2 - 108 bz^2
                S.T[2 + e] = fq_sub(sq_part(&S.p[7], e), fq_mul_small(sq_part(&S.p[9], e), 108));
            } else {                                    // Z' = 8 YY YZ
                S.T[4 + e] = fq_dbl(fq_dbl(fq_dbl(kara_part(&S.p[11], e))));
            }
        }
    }
    wsync<NW>();
    // round C: f^2 * line
    for (int t = L; t < 54; t += 32 * NW) wm_line_products(S, S.g, t);
    wsync<NW>();
    if (NW == 4) {
        wm_line_terms(S, L);
        wsync<NW>();
        if (L < 12) S.f[L] = wm_line_sum(S, L);
    } else {
        if (L < 12) S.h[L] = wm_line_combine(S, L);
        wsync<NW>();
        if (L < 12) S.f[L] = S.h[L];
    }
    wsync<NW>();
}

template <int NW>
FPG_NOINL void wm_add(WMill& S, const fq& mxP, const fq& yP) {
    const int L = w_lane<NW>();
    const fq* X = S.T;
    const fq* Y = S.T + 2;
    const fq* Z = S.T + 4;
    const fq* xQ = S.Q;
    const fq* yQ = S.Q + 2;
    // round A: yQ Z, xQ Z
    if (L < 6) {
        fq x, y;
        kara_ops(x, y, L < 3 ? yQ : xQ, Z, L % 3);
        S.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    if (L < 4) {                                    // theta = Y - yQ Z, lambda = X - xQ Z
        const int e = L & 1;
        S.v[L] = fq_sub(L < 2 ? Y[e] : X[e], kara_part(&S.p[L < 2 ? 0 : 3], e));
    }
    wsync<NW>();
    const fq* th = S.v;
    const fq* la = S.v + 2;
    // round B: theta xQ, lambda yQ, -theta xP, lambda yP, theta^2, lambda^2
    if (L < 14) {
        const int t = L;
        const fq* a;
        const fq* b;
        int kind, mode;
        if (t < 3) { a = th; b = xQ; kind = t; mode = 0; }
        else if (t < 6) { a = la; b = yQ; kind = t - 3; mode = 0; }
        else if (t < 8) { a = b = th; kind = t - 6; mode = 2; }
        else if (t < 10) { a = b = la; kind = t - 8; mode = 2; }
        else if (t < 12) { a = b = th; kind = t - 10; mode = 1; }
        else { a = b = la; kind = t - 12; mode = 1; }
        fq x, y;
        prod_ops(x, y, a, b, kind, mode, fq_select(t < 8, mxP, yP));
        S.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    if (L < 10) {
        const int w = L >> 1, e = L & 1;
        // w 0: l0 = theta xQ - lambda yQ, 1: l2, 2: l3, 3: C = theta^2, 4: D = lambda^2
        const fq l0 = fq_sub(kara_part(&S.p[0], e), kara_part(&S.p[3], e));
        const fq sq = sq_part(&S.p[w == 3 ? 10 : 12], e);
        const fq r = fq_select(w == 0, l0, fq_select(w < 3, S.p[6 + 2 * (w == 2) + e], sq));
        fq* dst = w < 3 ? &S.l[2 * w + e] : &S.v[4 + 2 * (w - 3) + e];
        *dst = r;
    }
    wsync<NW>();
    // round C: f * line (54) and E = D lambda, F = Z C, G = X D (9)
    for (int t = L; t < 63; t += 32 * NW) {
        const fq* a;
        const fq* b;
        int kind;
        if (t < 54) {                                   // f * line: f_i l_term
            const int q = t / 3, term = q / 6, k = q - 6 * term;
            const int i = term == 0 ? k : (term == 1 ? (k + 4) % 6 : (k + 3) % 6);
            a = S.f + 2 * i;
            b = S.l + 2 * term;
            kind = t - 3 * q;
        } else {                                        // E = D lambda, F = Z C, G = X D
            const int u = t - 54, which = u / 3;
            a = which == 0 ? S.v + 6 : (which == 1 ? Z : X);
            b = which == 0 ? la : (which == 1 ? S.v + 4 : S.v + 6);
            kind = u % 3;
        }
        fq x, y;
        kara_ops(x, y, a, b, kind);
        S.p[t] = fq_mul(x, y);
    }
    wsync<NW>();
    if (NW == 4) {
        wm_line_terms(S, L);
        if (L >= 64 && L < 70) {                     // E, F, G
            const int v = L - 64;
            S.v[8 + v] = kara_part(&S.p[54 + 3 * (v >> 1)], v & 1);
        }
        wsync<NW>();
        if (L < 12) S.f[L] = wm_line_sum(S, L);
    } else {
        if (L < 12) S.h[L] = wm_line_combine(S, L);
        else if (L < 18) {                          // E, F, G
            const int v = L - 12;
            S.v[8 + v] = kara_part(&S.p[54 + 3 * (v >> 1)], v & 1);
        }
        wsync<NW>();
        if (L < 12) S.f[L] = S.h[L];
    }
    // round D: lambda H, theta (G - H), Y E, Z E, with H = E + F - 2 G
    const fq* E = S.v + 8;
    const fq* Fv = S.v + 10;
    const fq* G = S.v + 12;
    if (L >= 16 && L < 28) {
        const int u = L - 16, which = u / 3;
        fq H[2], GH[2];
        for (int e = 0; e < 2; e++) {
            H[e] = fq_sub(fq_add(E[e], Fv[e]), fq_dbl(G[e]));
            GH[e] = fq_sub(G[e], H[e]);
        }
        fq x, y;
        kara_ops(x, y, which == 0 ? la : (which == 1 ? th : (which == 2 ? Y : Z)),
                 which == 0 ? H : (which == 1 ? GH : E), u % 3);
        S.p[u] = fq_mul(x, y);
    }
    wsync<NW>();
    if (L < 6) {
        const int w = L >> 1, e = L & 1;
        // w 0: X' = lambda H, 1: Y' = theta (G - H) - Y E, 2: Z' = Z E
        const fq k0 = kara_part(&S.p[w == 0 ? 0 : (w == 1 ? 3 : 9)], e);
        fq zero;
        fq_zero(zero);
        S.h[L] = fq_sub(k0, fq_select(w == 1, kara_part(&S.p[6], e), zero));
    }
    wsync<NW>();
    if (L < 6) S.T[L] = S.h[L];
    wsync<NW>();
}

// ---------------------------------------------------------------------------------------
// Pipelined doubling steps on the block engine.  The line of a doubling step and the next point
// 2T depend on T alone, not on f, so the point's chain runs one round ahead of f's:
//   round 1: f^2 (57 products) and the line / 2T products of T (15, from the operands formed in
//            the previous round);  round 2: f^2 * line (54) and the products of the new T (12).
// Two product rounds per doubling step instead of three; the same products and sums as wm_dbl.
// Layout of S.p: round 1: f^2 at 0..56, line / 2T at 57..71; round 2: f^2 * line at 0..53, the
// point's products at 54..65 (X^2 54, 55; Y^2 56, 57; Z^2 58, 59; Y Z 60..62; X Y 63..65).
// ---------------------------------------------------------------------------------------
constexpr int WMP_T = 54, WMP_B = 57;

// product u < 12 of the point T (S.T): X^2, Y^2, Z^2 (squares), Y Z, X Y (Karatsuba)
FPG_DEV void wmp_point_ops(const WMill& S, int u, fq& x, fq& y) {
    fq zero;
    fq_zero(zero);
    const fq* a;
    const fq* b;
    int kind, mode;
    if (u < 6) { a = b = S.T + 2 * (u >> 1); kind = u & 1; mode = 1; }
    else if (u < 9) { a = S.T + 2; b = S.T + 4; kind = u - 6; mode = 0; }
    else { a = S.T; b = S.T + 2; kind = u - 9; mode = 0; }
    prod_ops(x, y, a, b, kind, mode, zero);
}
// from the point's products: XX, YY, ZZ, YZ, XY (S.v[0..9]) on lanes 96..105
FPG_DEV void wmp_point_parts(WMill& S, int L) {
    if (L >= 96 && L < 106) {
        const int v = L - 96, which = v >> 1, e = v & 1;
        S.v[v] = fq_select(which < 3, sq_part(&S.p[WMP_T + 2 * (which < 3 ? which : 0)], e),
                           kara_part(&S.p[WMP_T + 6 + 3 * (which < 3 ? 0 : which - 3)], e));
    }
}
// round B's operands from ZZ and YY (S.v[16..27]) on lanes 96..107, as in wm_dbl
FPG_DEV void wmp_line_operands(WMill& S, int L) {
    if (L >= 96 && L < 108) {
        const int u = L - 96, e = u & 1, kind = u >> 1;
        const fq zr = S.p[WMP_T + 4], zi = fq_dbl(S.p[WMP_T + 5]);
        const fq bze = fq_dbl(fq_dbl(fq_select(e, fq_add(zr, zi), fq_sub(zr, zi))));
        const fq yy = fq_select(e, fq_dbl(S.p[WMP_T + 3]), S.p[WMP_T + 2]);
        const fq b3 = fq_add(fq_dbl(bze), bze);
        const fq b9 = fq_add(fq_dbl(b3), b3);
        const fq b6 = fq_dbl(b3);
        const fq sub_t = fq_select(kind == 1, b9, b3), add_t = fq_select(kind == 2, b9, b6);
        const fq r_sub = fq_sub(yy, sub_t);
        const fq r_add = fq_add(fq_select(kind == 2, yy, fq_dbl(b6)), add_t);
        S.v[16 + u] = fq_select(kind == 0, bze,
                                fq_select(kind == 1 || kind == 3, r_sub, fq_select(kind == 4, b6, r_add)));
    }
}
// the point's products of S.T and what the next step's line needs from them (start of the chain,
// and after an addition step)
template <int NW>
FPG_NOINL void wmp_prime(WMill& S) {
    const int L = w_lane<NW>();
    if (L >= WMP_T && L < WMP_T + 12) {
        fq x, y;
        wmp_point_ops(S, L - WMP_T, x, y);
        S.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    wmp_point_parts(S, L);
    wsync<NW>();
    wmp_line_operands(S, L);
    wsync<NW>();
}
// one doubling step: S.f <- S.f^2 * line(T), S.T <- 2T, with XX .. XY and round B's operands of T
// in S.v on entry and of 2T on exit
template <int NW>
FPG_NOINL void wmp_dbl(WMill& S, const fq& m3x, const fq& y2) {
    const int L = w_lane<NW>();
    // round 1: f^2 and the line / 2T products (the lanes choose their operands, then one product
    // call for all: a warp whose lanes reached the product through two branches would run it twice)
    if (L < WMP_B + 15) {
        const fq* a;
        const fq* b;
        int kind, mode;
        fq sc = m3x;
        if (L < 12) {                                                            // f_k^2
            a = b = S.f + 2 * (L >> 1);
            kind = L & 1;
            mode = 1;
        } else if (L < WMP_B) {                                                  // f_i f_j, i < j
            const int c = (L - 12) / 3;
            int i = 0, rem = c;
            while (rem >= 5 - i) { rem -= 5 - i; i++; }
            a = S.f + 2 * i;
            b = S.f + 2 * (i + 1 + rem);
            kind = L - 12 - 3 * c;
            mode = 0;
        } else {
            const int t = L - WMP_B;
            const fq* XX = S.v;
            const fq* YY = S.v + 2;
            const fq* YZ = S.v + 6;
            const fq* XY = S.v + 8;
            if (t < 2) { a = b = XX; kind = t; mode = 2; }                           // m3x XX
            else if (t < 4) { a = b = YZ; kind = t - 2; mode = 2; sc = y2; }         // y2 YZ
            else if (t < 7) { a = XY; b = S.v + 18; kind = t - 4; mode = 0; }        // XY (YY - 9 bz)
            else if (t < 9) { a = b = S.v + 20; kind = t - 7; mode = 1; }            // (YY + 9 bz)^2
            else if (t < 12) { a = S.v + 24; b = S.v + 26; kind = t - 9; mode = 0; } // 108 bz^2
            else { a = YY; b = YZ; kind = t - 12; mode = 0; }                        // YY YZ
        }
        fq x, y;
        prod_ops(x, y, a, b, kind, mode, sc);
        S.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    // f^2 terms (lanes 0..71); then beside their sums (warp 0) the line (warp 3: l0 = YY - 3 bz,
    // l2 = m3x XX, l3 = y2 YZ) and 2T, one formula per warp (X' = 2 XY (YY - 9 bz) on warp 1,
    // Y' = (YY + 9 bz)^2 - 108 bz^2 on warp 2, Z' = 8 YY YZ on warp 3)
    if (L < 72) {
        const int o = L % 12, i = L / 12, k = o >> 1, e = o & 1;
        int j = k - i;
        if (j < 0) j += 6;
        const int c = i < j ? i * (11 - i) / 2 + (j - i - 1) : 0;
        const fq* ms = &S.p[2 * i];
        const fq* mk = &S.p[12 + 3 * c];
        const fq re = fq_select(i == j, sq_part(ms, 0), fq_dbl(kara_part(mk, 0)));
        const fq im = fq_select(i == j, sq_part(ms, 1), fq_dbl(kara_part(mk, 1)));
        fq zero;
        fq_zero(zero);
        S.tm[L] = fq_select(i <= j, twist_part(re, im, e, i + j >= 6), zero);
    }
    wsync<NW>();
    {
        const int w = L >> 5, pl = L & 31;
        if (w == 0 && pl < 12) {
            fq acc = S.tm[L];
            for (int i = 1; i < 6; i++) acc = fq_add(acc, S.tm[12 * i + L]);
            S.g[L] = acc;
        } else if (w == 1 && pl < 2) {
            S.T[pl] = fq_dbl(kara_part(&S.p[WMP_B + 4], pl));
        } else if (w == 2 && pl < 2) {
            S.T[2 + pl] = fq_sub(sq_part(&S.p[WMP_B + 7], pl), kara_part(&S.p[WMP_B + 9], pl));
        } else if (w == 3 && pl < 2) {
            S.T[4 + pl] = fq_dbl(fq_dbl(fq_dbl(kara_part(&S.p[WMP_B + 12], pl))));
        } else if (w == 3 && pl >= 8 && pl < 14) {
            const int q = pl - 8, e = q & 1, which = q >> 1;
            S.l[q] = fq_select(which == 0, S.v[22 + e], S.p[WMP_B + 2 * (which ? which - 1 : 0) + e]);
        }
    }
    wsync<NW>();
    // round 2: f^2 * line and the products of the new point (one product call, as above)
    if (L < WMP_T + 12) {
        const fq* a;
        const fq* b;
        int kind, mode;
        if (L < 54) {                              // f^2 * line: f^2_i l_term (wm_line_products)
            const int q = L / 3, term = q / 6, k = q - 6 * term;
            const int i = term == 0 ? k : (term == 1 ? (k + 4) % 6 : (k + 3) % 6);
            a = S.g + 2 * i;
            b = S.l + 2 * term;
            kind = L - 3 * q;
            mode = 0;
        } else {
            const int u = L - WMP_T;
            if (u < 6) { a = b = S.T + 2 * (u >> 1); kind = u & 1; mode = 1; }
            else if (u < 9) { a = S.T + 2; b = S.T + 4; kind = u - 6; mode = 0; }
            else { a = S.T; b = S.T + 2; kind = u - 9; mode = 0; }
        }
        fq x, y;
        prod_ops(x, y, a, b, kind, mode, m3x);
        S.p[L] = fq_mul(x, y);
    }
    wsync<NW>();
    wm_line_terms(S, L);
    wmp_point_parts(S, L);
    wsync<NW>();
    if (L < 12) S.f[L] = wm_line_sum(S, L);
    wmp_line_operands(S, L);
    wsync<NW>();
}

// S.f <- conj(f_{|x|,Q}(P)) in flat order; 1 when P or Q is the identity
template <int NW>
FPG_NOINL void w_miller(WMill& S, g1a P, g2a Q) {
    const int L = w_lane<NW>();
    const bool inf = g1a_is_inf(P) || g2a_is_inf(Q);
    if (inf) {
        P = g1_generator();
        Q = g2_generator();
    }
    const fq m3x = fq_neg(fq_add(fq_dbl(P.x), P.x)), y2 = fq_dbl(P.y), mxP = fq_neg(P.x);
    if (L < 12) {
        fq one;
        fq_one(one);
        fq z;
        fq_zero(z);
        S.f[L] = fq_select(L == 0, one, z);
    }
    if (L == 0) {
        S.T[0] = Q.x.c0; S.T[1] = Q.x.c1; S.T[2] = Q.y.c0; S.T[3] = Q.y.c1;
        fq_one(S.T[4]);
        fq_zero(S.T[5]);
        S.Q[0] = Q.x.c0; S.Q[1] = Q.x.c1; S.Q[2] = Q.y.c0; S.Q[3] = Q.y.c1;
    }
    wsync<NW>();
    if (NW == 4) {                                  // pipelined doubling steps
        wmp_prime<NW>(S);
        for (int i = 62; i >= 0; i--) {
            wmp_dbl<NW>(S, m3x, y2);
            if ((BLS_X_ABS >> i) & 1) {
                wm_add<NW>(S, mxP, P.y);
                if (i) wmp_prime<NW>(S);
            }
        }
    } else {
        for (int i = 62; i >= 0; i--) {
            wm_dbl<NW>(S, m3x, y2);
            if ((BLS_X_ABS >> i) & 1) wm_add<NW>(S, mxP, P.y);
        }
    }
    if (L < 12) {
        fq one;
        fq_one(one);
        fq z;
        fq_zero(z);
        const fq v = fq_select((L >> 1) & 1, fq_neg(S.f[L]), S.f[L]);   // conjugation (x < 0)
        S.f[L] = fq_select(inf, fq_select(L == 0, one, z), v);
    }
    wsync<NW>();
}

// acc = base^e for any base (e little-endian words, squarings as products); acc != base
template <int NW>
FPG_NOINL void w_exp(W12& W, fq* acc, const fq* base, const uint32_t* e, int bits) {
    const int L = w_lane<NW>();
    int i = bits - 1;
    while (i >= 0 && !((e[i >> 5] >> (i & 31)) & 1)) i--;
    if (i < 0) {                                   // e = 0: acc = 1
        wsync<NW>();
        if (L < 12) {
            fq v;
            if (L == 0) fq_one(v);
            else fq_zero(v);
            acc[L] = v;
        }
        wsync<NW>();
        return;
    }
    w_copy<NW>(acc, base);
    for (i = i - 1; i >= 0; i--) {
        w_mul<NW>(W, acc, acc, acc);
        if ((e[i >> 5] >> (i & 31)) & 1) w_mul<NW>(W, acc, acc, base);
    }
}
