// Scalar multiplication on a group of 8 lanes, for the latency-bound folds of Step 1.
//
// Points are homogeneous projective (X : Y : Z) with the identity (0 : 1 : 0), and every addition
// and doubling uses the complete formulas of Renes, Costello and Batina (EUROCRYPT 2016) for a = 0
// (addition: Algorithm 7, doubling: Algorithm 9, b3 = 3b).  They have no exceptional cases, so the
// identity, P + P and P + (-P) need no branch, and each formula is two phases of at most six
// independent field products: lane t (t < 6) computes product t of the phase, the lanes exchange
// the products through shared memory, and every lane forms the linear combinations itself.
// The scalar is split by the endomorphisms (GLV on G1, GLS on G2, see curve.cuh) and consumed by a
// joint double-and-add over a table of subset sums that always adds (the empty subset is the
// identity), so all groups of a warp run the same instruction stream.
#pragma once
#include "pairing.cuh"

// barrier of the lanes of a warp (the groups of a warp run the same instruction stream)
FPG_DEV void gsync() { __syncwarp(); }

// The formulas' additions are called out of line: inlined, the linear combinations of a doubling
// and an addition outgrow the instruction cache, and instruction fetch then stalls every lane.
static __device__ __noinline__ fq e_add(fq a, fq b) { return fq_add(a, b); }
static __device__ __noinline__ fq e_sub(fq a, fq b) { return fq_sub(a, b); }
static __device__ __noinline__ fq e_dbl(fq a) { return fq_dbl(a); }
static __device__ __noinline__ fq2 e_add(fq2 a, fq2 b) { return fq2_add(a, b); }
static __device__ __noinline__ fq2 e_sub(fq2 a, fq2 b) { return fq2_sub(a, b); }
static __device__ __noinline__ fq2 e_dbl(fq2 a) { return fq2_dbl(a); }

template <typename F> struct GPt { F X, Y, Z; };

FPG_DEV fq f_sel(bool c, const fq& a, const fq& b) { return fq_select(c, a, b); }
FPG_DEV fq2 f_sel(bool c, const fq2& a, const fq2& b) { return fq2_select(c, a, b); }
// coordinate i (0: X, 1: Y, 2: Z) of P, without a per-lane branch
template <typename F>
FPG_DEV F gec_coord(const GPt<F>& P, int i) { return f_sel(i == 0, P.X, f_sel(i == 1, P.Y, P.Z)); }
// the first phase of an addition: lanes 0..2 multiply coordinate q of P and Q, lanes 3..5 the sums
// (X + Y), (Y + Z), (X + Z); every lane forms its operands with the same instructions
template <typename F>
FPG_DEV void gec_add_ops(int q, const GPt<F>& P, const GPt<F>& Q, F& a, F& b) {
    const int i1 = q < 3 ? q : (q == 4 ? 1 : 0), i2 = q == 3 ? 1 : 2;
    const F pa = gec_coord(P, i1), qa = gec_coord(Q, i1);
    const F ps = e_add(pa, gec_coord(P, i2)), qs = e_add(qa, gec_coord(Q, i2));
    a = f_sel(q >= 3, ps, pa);
    b = f_sel(q >= 3, qs, qa);
}
// the second phase of an addition: (t4 y3), (t3 u1), (y3 x3), (u1 z3), (x3 t3), (z3 t4)
template <typename F>
FPG_DEV void gec_add_ops2(int q, const F& t3, const F& t4, const F& x3, const F& y3, const F& z3, const F& u1, F& a,
                          F& b) {
    a = f_sel(q == 0, t4, f_sel(q == 1, t3, f_sel(q == 2, y3, f_sel(q == 3, u1, f_sel(q == 4, x3, z3)))));
    b = f_sel(q == 0, y3, f_sel(q == 1, u1, f_sel(q == 2, x3, f_sel(q == 3, z3, f_sel(q == 4, t3, t4)))));
}
// the formulas' scratch (products of the current phase), and the engine with a table of 16 points
template <typename F> struct GEcs {
    F sc[8];
};
template <typename F> struct GEc : GEcs<F> {
    GPt<F> tab[16];   // subset sums of the split bases
};

static __device__ __noinline__ fq f_b3(fq a) {            // 3 b = 12 on G1
    const fq t = fq_add(fq_dbl(a), a);
    return fq_dbl(fq_dbl(t));
}
static __device__ __noinline__ fq2 f_b3(fq2 a) {          // 3 b' = 12 (1 + u) on the twist
    const fq2 x = fq2_mul_xi(a);
    const fq2 t = fq2_add(fq2_dbl(x), x);
    return fq2_dbl(fq2_dbl(t));
}

template <typename F>
FPG_DEV void gec_phase(GEcs<F>& sm, int lane, const F& a, const F& b) {
    const F p = f_mul(a, b);
    gsync();
    if (lane < 6) sm.sc[lane] = p;
    gsync();
}

template <typename F>
FPG_DEV GPt<F> gec_identity() {
    GPt<F> r;
    f_set_zero(r.X); f_set_one(r.Y); f_set_zero(r.Z);
    return r;
}

// P + Q, complete (RCB16 Algorithm 7, a = 0)
template <typename F>
FPG_NOINL GPt<F> gec_add(GEcs<F>& sm, int lane, const GPt<F>& P, const GPt<F>& Q) {
    F a, b;
    gec_add_ops(lane < 6 ? lane : 5, P, Q, a, b);
    gec_phase(sm, lane, a, b);
    const F t0 = sm.sc[0], t1 = sm.sc[1], t2 = sm.sc[2];
    const F t3 = e_sub(sm.sc[3], e_add(t0, t1));
    const F t4 = e_sub(sm.sc[4], e_add(t1, t2));
    const F y3 = f_b3(e_sub(sm.sc[5], e_add(t0, t2)));
    const F x3 = e_add(e_dbl(t0), t0);
    const F bt2 = f_b3(t2);
    const F z3 = e_add(t1, bt2);
    const F u1 = e_sub(t1, bt2);
    gec_add_ops2(lane < 6 ? lane : 5, t3, t4, x3, y3, z3, u1, a, b);
    gec_phase(sm, lane, a, b);
    GPt<F> r;
    r.X = e_sub(sm.sc[1], sm.sc[0]);
    r.Y = e_add(sm.sc[3], sm.sc[2]);
    r.Z = e_add(sm.sc[5], sm.sc[4]);
    return r;
}

// 2P, complete (RCB16 Algorithm 9, a = 0)
template <typename F>
FPG_NOINL GPt<F> gec_dbl(GEcs<F>& sm, int lane, const GPt<F>& P) {
    // lanes: 0 Y Y, 1 Y Z, 2 Z Z, 3 X Y
    F a = f_sel(lane >= 3, P.X, f_sel(lane == 2, P.Z, P.Y));
    F b = f_sel(lane == 0, P.Y, f_sel(lane >= 3, P.Y, P.Z));
    gec_phase(sm, lane, a, b);
    const F t0 = sm.sc[0], t1 = sm.sc[1], xy = sm.sc[3];
    const F z8 = e_dbl(e_dbl(e_dbl(t0)));
    const F bt2 = f_b3(sm.sc[2]);
    const F y3a = e_add(t0, bt2);
    const F t0p = e_sub(t0, e_add(e_dbl(bt2), bt2));
    // lanes: 0 bt2 z8, 1 t1 z8, 2 t0p y3a, 3 t0p xy
    a = f_sel(lane == 0, bt2, f_sel(lane == 1, t1, t0p));
    b = f_sel(lane < 2, z8, f_sel(lane == 2, y3a, xy));
    gec_phase(sm, lane, a, b);
    GPt<F> r;
    r.X = e_dbl(sm.sc[3]);
    r.Y = e_add(sm.sc[0], sm.sc[2]);
    r.Z = sm.sc[1];
    return r;
}

template <typename F>
FPG_DEV GPt<F> gec_from_affine(const F& x, const F& y) {
    GPt<F> r;
    r.X = x; r.Y = y; f_set_one(r.Z);
    return r;
}

// affine (x, y) = (X/Z, Y/Z); (0, 0) for the identity
template <typename F>
FPG_DEV void gec_to_affine(F& x, F& y, const GPt<F>& P) {
    if (f_is_zero(P.Z)) { f_set_zero(x); f_set_zero(y); return; }
    const F zi = f_inv(P.Z);
    x = f_mul(P.X, zi);
    y = f_mul(P.Y, zi);
}

// the same with the inverse on the four lanes of each quad (f_inv_quad; every lane of a quad calls it
// converged with the same point): the inverse of Z = 0 is 0, so the identity gives (0, 0) without a
// branch
template <typename F>
FPG_DEV void gec_to_affine_quad(F& x, F& y, const GPt<F>& P) {
    const F zi = f_inv_quad(P.Z);
    x = f_mul(P.X, zi);
    y = f_mul(P.Y, zi);
}

template <typename F>
FPG_DEV GPt<F> gec_from_affine_or_inf(const F& x, const F& y) {
    return (f_is_zero(x) && f_is_zero(y)) ? gec_identity<F>() : gec_from_affine(x, y);
}

// ---------------------------------------------------------------------------------------
// G2 on one warp: the same complete formulas, but each of a phase's six Fq2 products is split
// into its three Karatsuba Fq products (m0 = a0 b0, m1 = a1 b1, m2 = (a0 + a1)(b0 + b1)), one per
// lane 0..17, so a phase costs one Fq product instead of three.  Lanes 0..11 then form the six
// Fq2 results (re = m0 - m1, im = m2 - m0 - m1) and every lane continues with the same linear
// combinations.
// ---------------------------------------------------------------------------------------
struct GEcWs {       // the formulas' scratch
    fq2 sc[8];
    fq p[18];
};
struct GEcW : GEcWs {
    GPt<fq2> tab[16];
};

// operands of product q = L / 3 come from sel(q, a, b); lane L computes component L % 3
template <typename Sel>
FPG_DEV void gecw_phase(GEcWs& sm, int L, Sel&& sel) {
    if (L < 18) {
        const int q = L / 3, kind = L - 3 * q;
        fq2 a, b;
        sel(q, a, b);
        fq zero;
        fq_zero(zero);
        const fq x = fq_add(fq_select(kind == 1, a.c1, a.c0), fq_select(kind == 2, a.c1, zero));
        const fq y = fq_add(fq_select(kind == 1, b.c1, b.c0), fq_select(kind == 2, b.c1, zero));
        sm.p[L] = fq_mul(x, y);
    }
    __syncwarp();
    fq r;
    if (L < 12) {
        const fq* m = &sm.p[3 * (L >> 1)];
        r = fq_select(L & 1, fq_sub(m[2], fq_add(m[0], m[1])), fq_sub(m[0], m[1]));
    }
    __syncwarp();
    if (L < 12) {
        fq* c = &sm.sc[L >> 1].c0;
        c[L & 1] = r;
    }
    __syncwarp();
}

// P + Q, complete (RCB16 Algorithm 7, a = 0), on one warp
FPG_NOINL GPt<fq2> gecw_add(GEcWs& sm, int L, const GPt<fq2>& P, const GPt<fq2>& Q) {
    gecw_phase(sm, L, [&](int q, fq2& a, fq2& b) { gec_add_ops(q, P, Q, a, b); });
    const fq2 t0 = sm.sc[0], t1 = sm.sc[1], t2 = sm.sc[2];
    const fq2 t3 = e_sub(sm.sc[3], e_add(t0, t1));
    const fq2 t4 = e_sub(sm.sc[4], e_add(t1, t2));
    const fq2 y3 = f_b3(e_sub(sm.sc[5], e_add(t0, t2)));
    const fq2 x3 = e_add(e_dbl(t0), t0);
    const fq2 bt2 = f_b3(t2);
    const fq2 z3 = e_add(t1, bt2);
    const fq2 u1 = e_sub(t1, bt2);
    gecw_phase(sm, L, [&](int q, fq2& a, fq2& b) { gec_add_ops2(q, t3, t4, x3, y3, z3, u1, a, b); });
    GPt<fq2> r;
    r.X = e_sub(sm.sc[1], sm.sc[0]);
    r.Y = e_add(sm.sc[3], sm.sc[2]);
    r.Z = e_add(sm.sc[5], sm.sc[4]);
    return r;
}

// 2P, complete (RCB16 Algorithm 9, a = 0), on one warp
FPG_NOINL GPt<fq2> gecw_dbl(GEcWs& sm, int L, const GPt<fq2>& P) {
    gecw_phase(sm, L, [&](int q, fq2& a, fq2& b) {
        a = fq2_select(q >= 3, P.X, fq2_select(q == 2, P.Z, P.Y));
        b = fq2_select(q == 0, P.Y, fq2_select(q >= 3, P.Y, P.Z));
    });
    const fq2 t0 = sm.sc[0], t1 = sm.sc[1], xy = sm.sc[3];
    const fq2 z8 = e_dbl(e_dbl(e_dbl(t0)));
    const fq2 bt2 = f_b3(sm.sc[2]);
    const fq2 y3a = e_add(t0, bt2);
    const fq2 t0p = e_sub(t0, e_add(e_dbl(bt2), bt2));
    gecw_phase(sm, L, [&](int q, fq2& a, fq2& b) {
        a = fq2_select(q == 0, bt2, fq2_select(q == 1, t1, t0p));
        b = fq2_select(q < 2, z8, fq2_select(q == 2, y3a, xy));
    });
    GPt<fq2> r;
    r.X = e_dbl(sm.sc[3]);
    r.Y = e_add(sm.sc[0], sm.sc[2]);
    r.Z = sm.sc[1];
    return r;
}

// GLS digits of a canonical k < r: k = sum_i d_i |x|^i with 64-bit d_i (two words each)
FPG_DEV void gls_digits(uint32_t (*d)[2], const uint32_t* k) {
    uint32_t q1[7], q2[7], q3[7];
    div_by_const<2, 7>(q1, d[0], k, GLS_D, GLS_BARRETT);
    uint32_t t8[8];
    for (int i = 0; i < 8; i++) t8[i] = i < 7 ? q1[i] : 0;
    div_by_const<2, 7>(q2, d[1], t8, GLS_D, GLS_BARRETT);
    for (int i = 0; i < 8; i++) t8[i] = i < 7 ? q2[i] : 0;
    div_by_const<2, 7>(q3, d[2], t8, GLS_D, GLS_BARRETT);
    d[3][0] = q3[0];
    d[3][1] = q3[1];
}

// sm.tab[s] = sum_{i in s} (-1)^i psi^i(Q) for s < 16, on one warp
FPG_DEV void gecw_g2_table(GEcW& sm, int L, const g2a& Q) {
    const bool inf = g2a_is_inf(Q);
    g2a b = Q;
    GPt<fq2> B[4];
    for (int i = 0; i < 4; i++) {
        if (i) b = g2_psi(b);
        const fq2 y = (i & 1) ? fq2_neg(b.y) : b.y;
        B[i] = inf ? gec_identity<fq2>() : gec_from_affine(b.x, y);
    }
    __syncwarp();
    if (L == 0) {
        sm.tab[0] = gec_identity<fq2>();
        for (int i = 0; i < 4; i++) sm.tab[1 << i] = B[i];
    }
    __syncwarp();
    for (int s = 3; s < 16; s++) {
        if (!(s & (s - 1))) continue;
        const int top = 31 - __clz(s);
        const GPt<fq2> r = gecw_add(sm, L, sm.tab[s & ~(1 << top)], sm.tab[1 << top]);
        __syncwarp();
        if (L == 0) sm.tab[s] = r;
        __syncwarp();
    }
}

// joint double-and-add over bits i0 + n - 1 .. i0 of the four digits on the table above:
// sum_i 2^(i - i0) sum_j bit_i(d_j) (-1)^j psi^j(Q)
FPG_DEV GPt<fq2> gecw_g2_bits(GEcW& sm, int L, const uint32_t (*d)[2], int i0, int n) {
    GPt<fq2> acc = gec_identity<fq2>();
    for (int i = i0 + n - 1; i >= i0; i--) {
        acc = gecw_dbl(sm, L, acc);
        const int s = bit_of(d[0], i) | (bit_of(d[1], i) << 1) | (bit_of(d[2], i) << 2) | (bit_of(d[3], i) << 3);
        acc = gecw_add(sm, L, acc, sm.tab[s]);
    }
    return acc;
}

// k Q on G2 for a canonical k < r (GLS: base-|x| digits, bases (-1)^i psi^i(Q)), on one warp
FPG_NOINL GPt<fq2> gecw_g2_mul_proj(GEcW& sm, int L, const g2a& Q, const uint32_t* k) {
    uint32_t d[4][2];
    gls_digits(d, k);
    gecw_g2_table(sm, L, Q);
    return gecw_g2_bits(sm, L, d, 0, 64);
}

// Part `part` of NP of k Q on G2, on one warp: bits [part 64/NP, (part + 1) 64/NP) of the four GLS
// digits on the bases of Qp = 2^(64 part / NP) Q (computed beforehand), so that k Q is the sum of
// the NP parts and each part is a chain of 64/NP steps instead of 64.
template <int NP>
FPG_NOINL GPt<fq2> gecw_g2_mul_part(GEcW& sm, int L, const g2a& Qp, const uint32_t* k, int part) {
    uint32_t d[4][2];
    gls_digits(d, k);
    gecw_g2_table(sm, L, Qp);
    return gecw_g2_bits(sm, L, d, part * (64 / NP), 64 / NP);
}

// 2^n P by n complete doublings, on one warp
FPG_NOINL GPt<fq2> gecw_g2_dbl_n(GEcWs& sm, int L, GPt<fq2> acc, int n) {
    for (int i = 0; i < n; i++) acc = gecw_dbl(sm, L, acc);
    return acc;
}

// tab[a + 4 b] = a P + b (-phi(P)) for a, b < 4 on an 8-lane group
FPG_DEV void gec_g1_w2_table(GEc<fq>& sm, int lane, const g1a& P) {
    fq om;
    fq_from_const(om, GLV_OMEGA);
    const bool inf = g1a_is_inf(P);
    const GPt<fq> B0 = inf ? gec_identity<fq>() : gec_from_affine(P.x, P.y);
    const GPt<fq> B1 = inf ? gec_identity<fq>() : gec_from_affine(fq_mul(P.x, om), fq_neg(P.y));
    const GPt<fq> B0x2 = gec_dbl(sm, lane, B0);
    const GPt<fq> B0x3 = gec_add(sm, lane, B0x2, B0);
    const GPt<fq> B1x2 = gec_dbl(sm, lane, B1);
    const GPt<fq> B1x3 = gec_add(sm, lane, B1x2, B1);
    gsync();
    if (lane == 0) {
        sm.tab[0] = gec_identity<fq>();
        sm.tab[1] = B0; sm.tab[2] = B0x2; sm.tab[3] = B0x3;
        sm.tab[4] = B1; sm.tab[8] = B1x2; sm.tab[12] = B1x3;
    }
    gsync();
    for (int b = 1; b < 4; b++) {
        for (int a = 1; a < 4; a++) {
            const GPt<fq> r = gec_add(sm, lane, sm.tab[a], sm.tab[4 * b]);
            gsync();
            if (lane == 0) sm.tab[a + 4 * b] = r;
            gsync();
        }
    }
}

// Horner over the 2-bit joint windows w = w0 + n - 1 .. w0 of the GLV halves (window w: bits 2w,
// 2w + 1 of k0 and k1) on the table above: two doublings and one addition per window
FPG_DEV GPt<fq> gec_g1_w2_windows(GEc<fq>& sm, int lane, const uint32_t* k0, const uint32_t* k1, int w0, int n) {
    GPt<fq> acc = gec_identity<fq>();
    for (int i = w0 + n - 1; i >= w0; i--) {
        acc = gec_dbl(sm, lane, gec_dbl(sm, lane, acc));
        const int a = (k0[i >> 4] >> (2 * (i & 15))) & 3;
        const int bb = (k1[i >> 4] >> (2 * (i & 15))) & 3;
        acc = gec_add(sm, lane, acc, sm.tab[a + 4 * bb]);
    }
    return acc;
}

// k P on G1 for a canonical k < r with 2-bit joint windows of the GLV halves: table
// tab[a + 4 b] = a P + b (-phi(P)) for a, b < 4, then 64 steps of two doublings and one addition
// (384 formula phases instead of 512 for the bit-by-bit ladder)
FPG_NOINL GPt<fq> gec_g1_mul_proj_w2(GEc<fq>& sm, int lane, const g1a& P, const uint32_t* k) {
    uint32_t k1[5], k0[4];
    div_by_const<4, 5>(k1, k0, k, GLV_D, GLV_BARRETT);
    gec_g1_w2_table(sm, lane, P);
    return gec_g1_w2_windows(sm, lane, k0, k1, 0, 64);
}

// Part `part` of NP of k P on G1, on an 8-lane group: 2-bit windows [part 64/NP, (part + 1) 64/NP)
// of the GLV halves on the bases of Pp = 2^(128 part / NP) P (computed beforehand), so that k P is
// the sum of the NP parts and each part is a chain of 64/NP steps instead of 64.
template <int NP>
FPG_NOINL GPt<fq> gec_g1_mul_part(GEc<fq>& sm, int lane, const g1a& Pp, const uint32_t* k, int part) {
    uint32_t k1[5], k0[4];
    div_by_const<4, 5>(k1, k0, k, GLV_D, GLV_BARRETT);
    gec_g1_w2_table(sm, lane, Pp);
    return gec_g1_w2_windows(sm, lane, k0, k1, part * (64 / NP), 64 / NP);
}

// 2^n P by n complete doublings, on an 8-lane group
FPG_NOINL GPt<fq> gec_g1_dbl_n(GEcs<fq>& sm, int lane, GPt<fq> acc, int n) {
    for (int i = 0; i < n; i++) acc = gec_dbl(sm, lane, acc);
    return acc;
}

// ---------------------------------------------------------------------------------------
// Fixed-base combs.  When the base of a scalar multiplication is known before its scalar, the
// doublings can run ahead: with B_w = 4^w P (G1, two bits of each GLV half per window) or
// B_i = 2^i Q (G2, one bit of each GLS digit per position) and a table of the window's or
// position's 16 combinations, k P is the sum of one table entry per window, and the additions of
// that sum are independent of each other.
// ---------------------------------------------------------------------------------------
// -phi(P) = (omega X : -Y : Z) for a projective P on G1 (phi: (x, y) -> (omega x, y))
FPG_DEV GPt<fq> gec_g1_mphi(const GPt<fq>& P) {
    fq om;
    fq_from_const(om, GLV_OMEGA);
    return {fq_mul(P.X, om), fq_neg(P.Y), P.Z};
}
// psi(P) = (cx conj(X) : cy conj(Y) : conj(Z)) for a projective P on the twist
FPG_DEV GPt<fq2> gec_g2_psi(const GPt<fq2>& P) {
    fq2 cx, cy;
    fq_from_const(cx.c0, PSI_CX0); fq_from_const(cx.c1, PSI_CX1);
    fq_from_const(cy.c0, PSI_CY0); fq_from_const(cy.c1, PSI_CY1);
    return {fq2_mul(fq2_conj(P.X), cx), fq2_mul(fq2_conj(P.Y), cy), fq2_conj(P.Z)};
}

// P + Q on one thread: the formulas of gec_add (RCB16 Algorithm 7, a = 0) without the lanes, for
// throughput work where many independent additions keep every lane busy
template <typename F>
FPG_NOINL GPt<F> gpt_add(const GPt<F> P, const GPt<F> Q) {
    const F t0 = f_mul(P.X, Q.X), t1 = f_mul(P.Y, Q.Y), t2 = f_mul(P.Z, Q.Z);
    const F s3 = f_mul(e_add(P.X, P.Y), e_add(Q.X, Q.Y));
    const F s4 = f_mul(e_add(P.Y, P.Z), e_add(Q.Y, Q.Z));
    const F s5 = f_mul(e_add(P.X, P.Z), e_add(Q.X, Q.Z));
    const F t3 = e_sub(s3, e_add(t0, t1));
    const F t4 = e_sub(s4, e_add(t1, t2));
    const F y3 = f_b3(e_sub(s5, e_add(t0, t2)));
    const F x3 = e_add(e_dbl(t0), t0);
    const F bt2 = f_b3(t2);
    const F z3 = e_add(t1, bt2), u1 = e_sub(t1, bt2);
    GPt<F> r;
    r.X = e_sub(f_mul(t3, u1), f_mul(t4, y3));
    r.Y = e_add(f_mul(y3, x3), f_mul(u1, z3));
    r.Z = e_add(f_mul(z3, t4), f_mul(x3, t3));
    return r;
}

// out[a + 4 b] = a B + b (-phi(B)) for a, b < 4, from B and 2B, on one thread (the entries are read
// back from out, which only this thread writes)
FPG_DEV void gpt_g1_comb_table(const GPt<fq>& B, const GPt<fq>& B2, GPt<fq>* out) {
    out[0] = gec_identity<fq>();
    out[1] = B;
    out[2] = B2;
    out[3] = gpt_add(B2, B);
    for (int i = 1; i < 4; i++) out[4 * i] = gec_g1_mphi(out[i]);
    for (int b = 1; b < 4; b++)
        for (int i = 1; i < 4; i++) out[i + 4 * b] = gpt_add(out[i], out[4 * b]);
}
// out[s] = sum_{j in s} (-1)^j psi^j(B) for s < 16, on one thread.  -psi maps T[s] to T[2 s] for s
// without bit 3, so the seven subsets holding base 0 are additions and the others psi maps:
//   1, 2 = -psi(1), 4 = -psi(2), 8 = -psi(4); 3 = 1 + 2, 5 = 1 + 4, 9 = 1 + 8, 7 = 3 + 4, 11 = 3 + 8,
//   13 = 5 + 8, 15 = 7 + 8; 6 = -psi(3), 10 = -psi(5), 12 = -psi(6), 14 = -psi(7)
// (entries indexed by the subset's bit mask)
FPG_DEV GPt<fq2> gpt_mpsi(const GPt<fq2>& P) {             // -psi(P), projective
    GPt<fq2> r = gec_g2_psi(P);
    r.Y = fq2_neg(r.Y);
    return r;
}
FPG_DEV void gpt_g2_comb_table(const GPt<fq2>& B, GPt<fq2>* out) {
    out[0] = gec_identity<fq2>();
    out[1] = B;
    out[2] = gpt_mpsi(out[1]);
    out[4] = gpt_mpsi(out[2]);
    out[8] = gpt_mpsi(out[4]);
    out[3] = gpt_add(out[1], out[2]);
    out[5] = gpt_add(out[1], out[4]);
    out[9] = gpt_add(out[1], out[8]);
    out[7] = gpt_add(out[3], out[4]);
    out[11] = gpt_add(out[3], out[8]);
    out[13] = gpt_add(out[5], out[8]);
    out[15] = gpt_add(out[7], out[8]);
    out[6] = gpt_mpsi(out[3]);
    out[10] = gpt_mpsi(out[5]);
    out[12] = gpt_mpsi(out[6]);
    out[14] = gpt_mpsi(out[7]);
}

// the window digit a + 4 b of window w of the GLV halves k0, k1, and the position digit of bit i of
// the four GLS digits
FPG_DEV int glv_window(const uint32_t* k0, const uint32_t* k1, int w) {
    return (int)(((k0[w >> 4] >> (2 * (w & 15))) & 3) | (((k1[w >> 4] >> (2 * (w & 15))) & 3) << 2));
}
FPG_DEV int gls_position(const uint32_t (*d)[2], int i) {
    return bit_of(d[0], i) | (bit_of(d[1], i) << 1) | (bit_of(d[2], i) << 2) | (bit_of(d[3], i) << 3);
}

// Jacobian (x = X / Z^2, y = Y / Z^3) <-> homogeneous projective (x = X / Z, y = Y / Z), the
// identity to the identity (a Jacobian point with Z = 0, whatever X and Y, maps to (0 : 1 : 0))
template <typename F>
FPG_DEV GPt<F> jac_to_proj(const jac<F>& p) {
    const F z2 = f_sqr(p.Z);
    F one;
    f_set_one(one);
    return {f_mul(p.X, p.Z), f_sel(f_is_zero(p.Z), one, p.Y), f_mul(z2, p.Z)};
}
template <typename F>
FPG_DEV jac<F> proj_to_jac(const GPt<F>& p) {
    return {f_mul(p.X, p.Z), f_mul(p.Y, f_sqr(p.Z)), p.Z};
}
