/*
 * Oracle groups: G1 = E(Fq): y^2 = x^3 + 4, G2 on the sextic twist E'(Fq2): y^2 = x^3 + 4(1+u),
 * Jacobian coordinates with the textbook formulas, plain MSB-first double-and-add scalar
 * multiplication, and the optimal-ate pairing with affine Miller steps.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's bilinear group ("Bilinear Group", Sec. 2) is Type-3 with A*B = prod e(A_i, B_i);
 * this file supplies e for BLS12-381.
 */
#include "oracle.h"
#include <string.h>

g1 G1_GEN;
g2 G2_GEN;
static fe B1;          /* 4 */
static fq2 B2;         /* 4 (1 + u) */

/* standard BLS12-381 generators (affine, big-endian hex); checked at start-up */
static const char* G1X = "17f1d3a73197d7942695638c4fa9ac0fc3688c4f9774b905a14e3a3f171bac586c55e83ff97a1aeffb3af00adb22c6bb";
static const char* G1Y = "08b3f481e3aaa0f1a09e30ed741d8ae4fcf5e095d5d00af600db18cb2c04b3edd03cc744a2888ae40caa232946c5e7e1";
static const char* G2X0 = "024aa2b2f08f0a91260805272dc51051c6e47ad4fa403b02b4510b647ae3d1770bac0326a805bbefd48056c8c121bdb8";
static const char* G2X1 = "13e02b6052719f607dacd3a088274f65596bd0d09920b61ab5da61bbdc7f5049334cf11213945d57e5ac7d055d042b7e";
static const char* G2Y0 = "0ce5d527727d6e118cc9cdc6da2e351aadfd9baa8cbdd3a76d429a695160d12c923ac9cc3baca289e193548608b82801";
static const char* G2Y1 = "0606c4a02ea734cc32acd2b02bc28b99cb3e287e85a763af267492ab572e99ab3f370d275cec1da1aaa9075ff05f79be";

static int hexval(char c) {
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    return -1;
}
static int fq_from_hex(fe* out, const char* h) {
    u8 be[48];
    for (int i = 0; i < 48; i++) be[i] = (u8)(hexval(h[2 * i]) * 16 + hexval(h[2 * i + 1]));
    return f_from_be(&FQ, out, be, 48);
}

/* ------------------------------- G1 -------------------------------------------- */
void g1_set_inf(g1* p) { memset(p, 0, sizeof *p); p->X = FQ.one; p->Y = FQ.one; }
int g1_is_inf(const g1* p) { return f_is_zero(&FQ, &p->Z); }

void g1_dbl(g1* r, const g1* p) {
    if (g1_is_inf(p) || f_is_zero(&FQ, &p->Y)) { g1_set_inf(r); return; }
    fe A, B, C, D, E, F, t, X3, Y3, Z3;
    f_mul(&FQ, &A, &p->X, &p->X);                     /* A = X^2 */
    f_mul(&FQ, &B, &p->Y, &p->Y);                     /* B = Y^2 */
    f_mul(&FQ, &C, &B, &B);                           /* C = B^2 */
    f_add(&FQ, &t, &p->X, &B);                        /* D = 2((X+B)^2 - A - C) */
    f_mul(&FQ, &t, &t, &t);
    f_sub(&FQ, &t, &t, &A);
    f_sub(&FQ, &t, &t, &C);
    f_add(&FQ, &D, &t, &t);
    f_add(&FQ, &E, &A, &A);                           /* E = 3A */
    f_add(&FQ, &E, &E, &A);
    f_mul(&FQ, &F, &E, &E);                           /* F = E^2 */
    f_sub(&FQ, &X3, &F, &D);                          /* X3 = F - 2D */
    f_sub(&FQ, &X3, &X3, &D);
    f_sub(&FQ, &t, &D, &X3);                          /* Y3 = E(D - X3) - 8C */
    f_mul(&FQ, &Y3, &E, &t);
    f_add(&FQ, &C, &C, &C); f_add(&FQ, &C, &C, &C); f_add(&FQ, &C, &C, &C);
    f_sub(&FQ, &Y3, &Y3, &C);
    f_mul(&FQ, &Z3, &p->Y, &p->Z);                    /* Z3 = 2YZ */
    f_add(&FQ, &Z3, &Z3, &Z3);
    r->X = X3; r->Y = Y3; r->Z = Z3;
}

void g1_add(g1* r, const g1* p, const g1* q) {
    if (g1_is_inf(p)) { *r = *q; return; }
    if (g1_is_inf(q)) { *r = *p; return; }
    fe Z1Z1, Z2Z2, U1, U2, S1, S2, H, R, H2, H3, U1H2, X3, Y3, Z3, t;
    f_mul(&FQ, &Z1Z1, &p->Z, &p->Z);
    f_mul(&FQ, &Z2Z2, &q->Z, &q->Z);
    f_mul(&FQ, &U1, &p->X, &Z2Z2);                    /* U1 = X1 Z2^2 */
    f_mul(&FQ, &U2, &q->X, &Z1Z1);                    /* U2 = X2 Z1^2 */
    f_mul(&FQ, &S1, &p->Y, &Z2Z2); f_mul(&FQ, &S1, &S1, &q->Z);   /* S1 = Y1 Z2^3 */
    f_mul(&FQ, &S2, &q->Y, &Z1Z1); f_mul(&FQ, &S2, &S2, &p->Z);   /* S2 = Y2 Z1^3 */
    if (f_eq(&FQ, &U1, &U2)) {
        if (f_eq(&FQ, &S1, &S2)) { g1_dbl(r, p); return; }
        g1_set_inf(r); return;
    }
    f_sub(&FQ, &H, &U2, &U1);
    f_sub(&FQ, &R, &S2, &S1);
    f_mul(&FQ, &H2, &H, &H);
    f_mul(&FQ, &H3, &H2, &H);
    f_mul(&FQ, &U1H2, &U1, &H2);
    f_mul(&FQ, &X3, &R, &R);                           /* X3 = R^2 - H^3 - 2 U1 H^2 */
    f_sub(&FQ, &X3, &X3, &H3);
    f_sub(&FQ, &X3, &X3, &U1H2);
    f_sub(&FQ, &X3, &X3, &U1H2);
    f_sub(&FQ, &t, &U1H2, &X3);                        /* Y3 = R(U1 H^2 - X3) - S1 H^3 */
    f_mul(&FQ, &Y3, &R, &t);
    f_mul(&FQ, &t, &S1, &H3);
    f_sub(&FQ, &Y3, &Y3, &t);
    f_mul(&FQ, &Z3, &H, &p->Z); f_mul(&FQ, &Z3, &Z3, &q->Z);       /* Z3 = H Z1 Z2 */
    r->X = X3; r->Y = Y3; r->Z = Z3;
}
void g1_neg(g1* r, const g1* p) { *r = *p; f_neg(&FQ, &r->Y, &p->Y); }

void g1_mul(g1* r, const g1* p, const fe* k) {
    u64 l[FE_LIMBS] = {0}; f_to_canon(&FR, l, k);
    g1_mul_limbs(r, p, l);
}
static u64 OR_OPS[OR_OP_KINDS];
void or_op_count(int kind) { __atomic_fetch_add(&OR_OPS[kind], 1, __ATOMIC_RELAXED); }
void or_ops_reset(void) { for (int i = 0; i < OR_OP_KINDS; i++) __atomic_store_n(&OR_OPS[i], 0, __ATOMIC_RELAXED); }
void or_ops_get(u64 out[OR_OP_KINDS]) { for (int i = 0; i < OR_OP_KINDS; i++) out[i] = __atomic_load_n(&OR_OPS[i], __ATOMIC_RELAXED); }

void g1_mul_limbs(g1* r, const g1* p, const u64 l[4]) {
    or_op_count(OR_OP_G1_MUL);
    g1 acc; g1_set_inf(&acc);
    for (int i = 255; i >= 0; i--) {
        g1_dbl(&acc, &acc);
        if ((l[i / 64] >> (i % 64)) & 1) g1_add(&acc, &acc, p);
    }
    *r = acc;
}
void g1_affine(fe* x, fe* y, const g1* p) {
    fe zi, zi2, zi3;
    f_inv(&FQ, &zi, &p->Z);
    f_mul(&FQ, &zi2, &zi, &zi);
    f_mul(&FQ, &zi3, &zi2, &zi);
    f_mul(&FQ, x, &p->X, &zi2);
    f_mul(&FQ, y, &p->Y, &zi3);
}
int g1_eq(const g1* p, const g1* q) {
    if (g1_is_inf(p) || g1_is_inf(q)) return g1_is_inf(p) && g1_is_inf(q);
    fe x1, y1, x2, y2;
    g1_affine(&x1, &y1, p); g1_affine(&x2, &y2, q);
    return f_eq(&FQ, &x1, &x2) && f_eq(&FQ, &y1, &y2);
}
int g1_on_curve(const g1* p) {
    if (g1_is_inf(p)) return 1;
    fe x, y, l, r;
    g1_affine(&x, &y, p);
    f_mul(&FQ, &l, &y, &y);
    f_mul(&FQ, &r, &x, &x); f_mul(&FQ, &r, &r, &x); f_add(&FQ, &r, &r, &B1);
    return f_eq(&FQ, &l, &r);
}
void g1_to_bytes(u8 out[96], const g1* p) {
    if (g1_is_inf(p)) { memset(out, 0, 96); return; }
    fe x, y; g1_affine(&x, &y, p);
    f_to_be(&FQ, out, 48, &x);
    f_to_be(&FQ, out + 48, 48, &y);
}
int g1_from_bytes(g1* p, const u8 in[96]) {
    int zero = 1;
    for (int i = 0; i < 96; i++) if (in[i]) { zero = 0; break; }
    if (zero) { g1_set_inf(p); return 0; }
    if (f_from_be(&FQ, &p->X, in, 48) || f_from_be(&FQ, &p->Y, in + 48, 48)) return -1;
    p->Z = FQ.one;
    return g1_on_curve(p) ? 0 : -1;
}

/* ------------------------------- G2 -------------------------------------------- */
void g2_set_inf(g2* p) { memset(p, 0, sizeof *p); fq2_set_one(&p->X); fq2_set_one(&p->Y); }
int g2_is_inf(const g2* p) { return fq2_is_zero(&p->Z); }

void g2_dbl(g2* r, const g2* p) {
    if (g2_is_inf(p) || fq2_is_zero(&p->Y)) { g2_set_inf(r); return; }
    fq2 A, B, C, D, E, F, t, X3, Y3, Z3;
    fq2_mul(&A, &p->X, &p->X);
    fq2_mul(&B, &p->Y, &p->Y);
    fq2_mul(&C, &B, &B);
    fq2_add(&t, &p->X, &B);
    fq2_mul(&t, &t, &t);
    fq2_sub(&t, &t, &A);
    fq2_sub(&t, &t, &C);
    fq2_add(&D, &t, &t);
    fq2_add(&E, &A, &A);
    fq2_add(&E, &E, &A);
    fq2_mul(&F, &E, &E);
    fq2_sub(&X3, &F, &D);
    fq2_sub(&X3, &X3, &D);
    fq2_sub(&t, &D, &X3);
    fq2_mul(&Y3, &E, &t);
    fq2_add(&C, &C, &C); fq2_add(&C, &C, &C); fq2_add(&C, &C, &C);
    fq2_sub(&Y3, &Y3, &C);
    fq2_mul(&Z3, &p->Y, &p->Z);
    fq2_add(&Z3, &Z3, &Z3);
    r->X = X3; r->Y = Y3; r->Z = Z3;
}
void g2_add(g2* r, const g2* p, const g2* q) {
    if (g2_is_inf(p)) { *r = *q; return; }
    if (g2_is_inf(q)) { *r = *p; return; }
    fq2 Z1Z1, Z2Z2, U1, U2, S1, S2, H, R, H2, H3, U1H2, X3, Y3, Z3, t;
    fq2_mul(&Z1Z1, &p->Z, &p->Z);
    fq2_mul(&Z2Z2, &q->Z, &q->Z);
    fq2_mul(&U1, &p->X, &Z2Z2);
    fq2_mul(&U2, &q->X, &Z1Z1);
    fq2_mul(&S1, &p->Y, &Z2Z2); fq2_mul(&S1, &S1, &q->Z);
    fq2_mul(&S2, &q->Y, &Z1Z1); fq2_mul(&S2, &S2, &p->Z);
    if (fq2_eq(&U1, &U2)) {
        if (fq2_eq(&S1, &S2)) { g2_dbl(r, p); return; }
        g2_set_inf(r); return;
    }
    fq2_sub(&H, &U2, &U1);
    fq2_sub(&R, &S2, &S1);
    fq2_mul(&H2, &H, &H);
    fq2_mul(&H3, &H2, &H);
    fq2_mul(&U1H2, &U1, &H2);
    fq2_mul(&X3, &R, &R);
    fq2_sub(&X3, &X3, &H3);
    fq2_sub(&X3, &X3, &U1H2);
    fq2_sub(&X3, &X3, &U1H2);
    fq2_sub(&t, &U1H2, &X3);
    fq2_mul(&Y3, &R, &t);
    fq2_mul(&t, &S1, &H3);
    fq2_sub(&Y3, &Y3, &t);
    fq2_mul(&Z3, &H, &p->Z); fq2_mul(&Z3, &Z3, &q->Z);
    r->X = X3; r->Y = Y3; r->Z = Z3;
}
void g2_neg(g2* r, const g2* p) { *r = *p; fq2_neg(&r->Y, &p->Y); }
void g2_mul(g2* r, const g2* p, const fe* k) {
    u64 l[FE_LIMBS] = {0}; f_to_canon(&FR, l, k);
    g2_mul_limbs(r, p, l);
}
void g2_mul_limbs(g2* r, const g2* p, const u64 l[4]) {
    or_op_count(OR_OP_G2_MUL);
    g2 acc; g2_set_inf(&acc);
    for (int i = 255; i >= 0; i--) {
        g2_dbl(&acc, &acc);
        if ((l[i / 64] >> (i % 64)) & 1) g2_add(&acc, &acc, p);
    }
    *r = acc;
}
void g2_affine(fq2* x, fq2* y, const g2* p) {
    fq2 zi, zi2, zi3;
    fq2_inv(&zi, &p->Z);
    fq2_mul(&zi2, &zi, &zi);
    fq2_mul(&zi3, &zi2, &zi);
    fq2_mul(x, &p->X, &zi2);
    fq2_mul(y, &p->Y, &zi3);
}
int g2_eq(const g2* p, const g2* q) {
    if (g2_is_inf(p) || g2_is_inf(q)) return g2_is_inf(p) && g2_is_inf(q);
    fq2 x1, y1, x2, y2;
    g2_affine(&x1, &y1, p); g2_affine(&x2, &y2, q);
    return fq2_eq(&x1, &x2) && fq2_eq(&y1, &y2);
}
int g2_on_curve(const g2* p) {
    if (g2_is_inf(p)) return 1;
    fq2 x, y, l, r;
    g2_affine(&x, &y, p);
    fq2_mul(&l, &y, &y);
    fq2_mul(&r, &x, &x); fq2_mul(&r, &r, &x); fq2_add(&r, &r, &B2);
    return fq2_eq(&l, &r);
}
void g2_to_bytes(u8 out[192], const g2* p) {
    if (g2_is_inf(p)) { memset(out, 0, 192); return; }
    fq2 x, y; g2_affine(&x, &y, p);
    f_to_be(&FQ, out, 48, &x.c0);
    f_to_be(&FQ, out + 48, 48, &x.c1);
    f_to_be(&FQ, out + 96, 48, &y.c0);
    f_to_be(&FQ, out + 144, 48, &y.c1);
}
int g2_from_bytes(g2* p, const u8 in[192]) {
    int zero = 1;
    for (int i = 0; i < 192; i++) if (in[i]) { zero = 0; break; }
    if (zero) { g2_set_inf(p); return 0; }
    if (f_from_be(&FQ, &p->X.c0, in, 48) || f_from_be(&FQ, &p->X.c1, in + 48, 48) ||
        f_from_be(&FQ, &p->Y.c0, in + 96, 48) || f_from_be(&FQ, &p->Y.c1, in + 144, 48)) return -1;
    fq2_set_one(&p->Z);
    return g2_on_curve(p) ? 0 : -1;
}

/* ------------------------------- pairing --------------------------------------------
 * Untwisting psi: E'(Fq2) -> E(Fq12), (x', y') -> (x' w^-2, y' w^-3), since w^6 = 1 + u.
 * For T, Q on the twist with slope lam' (tangent: 3x'^2/(2y'), chord: (yQ'-yT')/(xQ'-xT')),
 * the slope on E is lam' w^-1 and the line through psi(T) evaluated at P = (xP, yP) in E(Fq) is
 *     l(P) = yP - yT' w^-3 - lam' w^-1 (xP - xT' w^-2)
 *          = w^-3 ( (lam' xT' - yT') - lam' xP w^2 + yP w^3 ).
 * The common factor w^-3 satisfies (w^-3)^((p^12-1)/r) = 1 (w^(p^6) = -w and p^2 + 1 is even),
 * so the Miller loop multiplies by the bracket only.  f_{x,Q} with x < 0 equals
 * 1/(f_{|x|,Q} v_{[|x|]Q}) and the vertical line lies in Fq6, so after the final exponentiation
 * the pairing is (conj f_{|x|,Q}(P))^((p^12-1)/r).
 * --------------------------------------------------------------------------------- */
static void line_mul(fq12* f, const fq2* lam, const fq2* xT, const fq2* yT, const fe* xP, const fe* yP) {
    fq12 l; memset(&l, 0, sizeof l);
    fq2 t;
    fq2_mul(&t, lam, xT);
    fq2_sub(&l.c[0], &t, yT);                 /* w^0: lam' xT' - yT' */
    fq2_mul_fq(&t, lam, xP);
    fq2_neg(&l.c[2], &t);                     /* w^2: -lam' xP */
    l.c[3].c0 = *yP;                          /* w^3: yP */
    fq12_mul(f, f, &l);
}

void miller_loop(fq12* f, const g1* P, const g2* Q) {
    or_op_count(OR_OP_MILLER);
    fq12_one(f);
    if (g1_is_inf(P) || g2_is_inf(Q)) return;
    fe xP, yP; g1_affine(&xP, &yP, P);
    fq2 xQ, yQ; g2_affine(&xQ, &yQ, Q);
    fq2 xT = xQ, yT = yQ;
    const u64 ax = 0xd201000000010000ull;
    for (int i = 62; i >= 0; i--) {
        /* doubling step: f <- f^2 l_{T,T}(P), T <- 2T */
        fq2 lam, num, den, t, x3, y3;
        fq2_mul(&num, &xT, &xT);
        fq2_add(&t, &num, &num); fq2_add(&num, &t, &num);       /* 3 xT^2 */
        fq2_add(&den, &yT, &yT);                                /* 2 yT */
        fq2_inv(&t, &den);
        fq2_mul(&lam, &num, &t);
        fq12_mul(f, f, f);
        line_mul(f, &lam, &xT, &yT, &xP, &yP);
        fq2_mul(&x3, &lam, &lam);
        fq2_sub(&x3, &x3, &xT); fq2_sub(&x3, &x3, &xT);         /* x3 = lam^2 - 2 xT */
        fq2_sub(&t, &xT, &x3);
        fq2_mul(&y3, &lam, &t); fq2_sub(&y3, &y3, &yT);         /* y3 = lam (xT - x3) - yT */
        xT = x3; yT = y3;
        if ((ax >> i) & 1) {
            /* addition step: f <- f l_{T,Q}(P), T <- T + Q */
            fq2_sub(&num, &yQ, &yT);
            fq2_sub(&den, &xQ, &xT);
            fq2_inv(&t, &den);
            fq2_mul(&lam, &num, &t);
            line_mul(f, &lam, &xT, &yT, &xP, &yP);
            fq2_mul(&x3, &lam, &lam);
            fq2_sub(&x3, &x3, &xT); fq2_sub(&x3, &x3, &xQ);     /* x3 = lam^2 - xT - xQ */
            fq2_sub(&t, &xT, &x3);
            fq2_mul(&y3, &lam, &t); fq2_sub(&y3, &y3, &yT);
            xT = x3; yT = y3;
        }
    }
    fq12_conj(f, f);
}

void final_exp(fq12* r, const fq12* f) {
    or_op_count(OR_OP_FINAL_EXP);
    fq12_pow_words(r, f, OR_EXP_FINAL, OR_EXP_FINAL_WORDS);
}

void pairing(fq12* r, const g1* P, const g2* Q) {
    fq12 f; miller_loop(&f, P, Q); final_exp(r, &f);
}

int or_curves_init(void) {
    f_from_u64(&FQ, &B1, 4);
    fq2 four; fq2_set_zero(&four); four.c0 = B1; four.c1 = B1;       /* 4 + 4u */
    B2 = four;
    if (fq_from_hex(&G1_GEN.X, G1X) || fq_from_hex(&G1_GEN.Y, G1Y)) return -10;
    G1_GEN.Z = FQ.one;
    if (fq_from_hex(&G2_GEN.X.c0, G2X0) || fq_from_hex(&G2_GEN.X.c1, G2X1) ||
        fq_from_hex(&G2_GEN.Y.c0, G2Y0) || fq_from_hex(&G2_GEN.Y.c1, G2Y1)) return -11;
    fq2_set_one(&G2_GEN.Z);
    if (!g1_on_curve(&G1_GEN)) return -12;
    if (!g2_on_curve(&G2_GEN)) return -13;
    return 0;
}
