/*
 * Oracle arithmetic: a small bignum used only to derive the BLS12-381 constants, generic
 * Montgomery residues for Fq and Fr, Fq2 = Fq[u]/(u^2+1) and a FLAT Fq12 = Fq2[w]/(w^6-(1+u)).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The curve family is BLS12 with seed x = -0xd201000000010000:
 *     r = x^4 - x^2 + 1,   p = (x-1)^2 r / 3 + x,   #E(Fq) = p + 1 - (x + 1) = p - x = h1 r,
 * with h1 = (x-1)^2/3.  The paper instantiates its bilinear group with mcl/BN_SNARK1
 * (Sec. 5); this build reads the group as BLS12-381 and derives everything from x here.
 */
#include "oracle.h"
#include <string.h>

field FQ, FR;
u32 OR_EXP_FINAL[160];
int OR_EXP_FINAL_WORDS;

/* ---------------------------------------------------------------------------------
 * Plain bignum (little-endian 32-bit words), only for deriving constants at start-up.
 * ------------------------------------------------------------------------------- */
#define BW 320
typedef struct { int n; u32 w[BW]; } big;

static void big_norm(big* a) { while (a->n > 0 && a->w[a->n - 1] == 0) a->n--; }
static void big_set_u64(big* a, u64 x) {
    memset(a, 0, sizeof *a);
    a->w[0] = (u32)x; a->w[1] = (u32)(x >> 32); a->n = 2; big_norm(a);
}
static int big_cmp(const big* a, const big* b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; i--)
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    return 0;
}
static void big_add(big* c, const big* a, const big* b) {
    big t; memset(&t, 0, sizeof t);
    int n = a->n > b->n ? a->n : b->n; u64 carry = 0;
    for (int i = 0; i < n; i++) {
        carry += (u64)(i < a->n ? a->w[i] : 0) + (i < b->n ? b->w[i] : 0);
        t.w[i] = (u32)carry; carry >>= 32;
    }
    t.w[n] = (u32)carry; t.n = n + 1; big_norm(&t); *c = t;
}
static void big_sub(big* c, const big* a, const big* b) {      /* requires a >= b */
    big t; memset(&t, 0, sizeof t);
    int64_t borrow = 0;
    for (int i = 0; i < a->n; i++) {
        int64_t d = (int64_t)a->w[i] - (i < b->n ? b->w[i] : 0) - borrow;
        borrow = d < 0; if (d < 0) d += ((int64_t)1 << 32);
        t.w[i] = (u32)d;
    }
    t.n = a->n; big_norm(&t); *c = t;
}
static void big_mul(big* c, const big* a, const big* b) {
    big t; memset(&t, 0, sizeof t);
    for (int i = 0; i < a->n; i++) {
        u64 carry = 0;
        for (int j = 0; j < b->n; j++) {
            carry += (u64)a->w[i] * b->w[j] + t.w[i + j];
            t.w[i + j] = (u32)carry; carry >>= 32;
        }
        t.w[i + b->n] = (u32)carry;
    }
    t.n = a->n + b->n; big_norm(&t); *c = t;
}
static int big_bit(const big* a, int i) { return (i / 32 < a->n) ? (a->w[i / 32] >> (i % 32)) & 1 : 0; }
static int big_bits(const big* a) {
    if (a->n == 0) return 0;
    int b = 32 * (a->n - 1); u32 top = a->w[a->n - 1];
    while (top) { b++; top >>= 1; }
    return b;
}
/* schoolbook binary long division: q = a / d, rem = a mod d */
static void big_divmod(big* q, big* rem, const big* a, const big* d) {
    big Q, R; memset(&Q, 0, sizeof Q); memset(&R, 0, sizeof R);
    for (int i = big_bits(a) - 1; i >= 0; i--) {
        /* R = 2R + bit */
        u32 carry = (u32)big_bit(a, i);
        for (int k = 0; k <= R.n; k++) {
            u32 nc = R.w[k] >> 31; R.w[k] = (R.w[k] << 1) | carry; carry = nc;
        }
        R.n++; big_norm(&R);
        if (big_cmp(&R, d) >= 0) { big_sub(&R, &R, d); Q.w[i / 32] |= 1u << (i % 32); }
    }
    Q.n = BW; big_norm(&Q);
    if (q) *q = Q;
    if (rem) *rem = R;
}
static void big_to_u64(u64* out, int n, const big* a) {
    for (int i = 0; i < n; i++)
        out[i] = (u64)(2 * i < a->n ? a->w[2 * i] : 0) | ((u64)(2 * i + 1 < a->n ? a->w[2 * i + 1] : 0) << 32);
}

/* ---------------------------------------------------------------------------------
 * Generic Montgomery arithmetic (CIOS), R = 2^(64 n).
 * ------------------------------------------------------------------------------- */
static int limbs_geq(const u64* a, const u64* b, int n) {
    for (int i = n - 1; i >= 0; i--) if (a[i] != b[i]) return a[i] > b[i];
    return 1;
}
static u64 limbs_sub(u64* c, const u64* a, const u64* b, int n) {
    u64 borrow = 0;
    for (int i = 0; i < n; i++) {
        u128 d = (u128)a[i] - b[i] - borrow;
        c[i] = (u64)d; borrow = (u64)(d >> 64) & 1;
    }
    return borrow;
}
static u64 limbs_add(u64* c, const u64* a, const u64* b, int n) {
    u64 carry = 0;
    for (int i = 0; i < n; i++) {
        u128 s = (u128)a[i] + b[i] + carry;
        c[i] = (u64)s; carry = (u64)(s >> 64);
    }
    return carry;
}

void f_zero(fe* a) { memset(a, 0, sizeof *a); }

void f_add(const field* F, fe* c, const fe* a, const fe* b) {
    fe t; f_zero(&t);
    u64 carry = limbs_add(t.v, a->v, b->v, F->n);
    if (carry || limbs_geq(t.v, F->mod, F->n)) limbs_sub(t.v, t.v, F->mod, F->n);
    *c = t;
}
void f_sub(const field* F, fe* c, const fe* a, const fe* b) {
    fe t; f_zero(&t);
    if (limbs_sub(t.v, a->v, b->v, F->n)) limbs_add(t.v, t.v, F->mod, F->n);
    *c = t;
}
void f_neg(const field* F, fe* c, const fe* a) { fe z; f_zero(&z); f_sub(F, c, &z, a); }

void f_mul(const field* F, fe* c, const fe* a, const fe* b) {
    const int n = F->n;
    u64 t[FE_LIMBS + 2] = {0};
    for (int i = 0; i < n; i++) {
        u128 acc = 0;
        for (int j = 0; j < n; j++) {
            acc += (u128)a->v[j] * b->v[i] + t[j];
            t[j] = (u64)acc; acc >>= 64;
        }
        acc += t[n]; t[n] = (u64)acc; t[n + 1] = (u64)(acc >> 64);
        u64 m = t[0] * F->ninv;
        acc = ((u128)m * F->mod[0] + t[0]) >> 64;
        for (int j = 1; j < n; j++) {
            acc += (u128)m * F->mod[j] + t[j];
            t[j - 1] = (u64)acc; acc >>= 64;
        }
        acc += t[n]; t[n - 1] = (u64)acc; t[n] = t[n + 1] + (u64)(acc >> 64);
    }
    fe r; f_zero(&r);
    memcpy(r.v, t, sizeof(u64) * n);
    if (t[n] || limbs_geq(r.v, F->mod, n)) limbs_sub(r.v, r.v, F->mod, n);
    *c = r;
}

int f_is_zero(const field* F, const fe* a) {
    for (int i = 0; i < F->n; i++) if (a->v[i]) return 0;
    return 1;
}
int f_eq(const field* F, const fe* a, const fe* b) {
    for (int i = 0; i < F->n; i++) if (a->v[i] != b->v[i]) return 0;
    return 1;
}
void f_from_canon(const field* F, fe* c, const u64* limbs) {
    fe t; f_zero(&t); memcpy(t.v, limbs, sizeof(u64) * F->n);
    f_mul(F, c, &t, &F->r2);
}
void f_to_canon(const field* F, u64* limbs, const fe* a) {
    fe one; f_zero(&one); one.v[0] = 1;
    fe t; f_mul(F, &t, a, &one);
    memcpy(limbs, t.v, sizeof(u64) * F->n);
}
void f_from_u64(const field* F, fe* c, u64 x) {
    u64 l[FE_LIMBS] = {0}; l[0] = x; f_from_canon(F, c, l);
}
/* plain exponentiation by a little-endian limb exponent, left to right */
static void f_pow_limbs(const field* F, fe* c, const fe* a, const u64* e, int n) {
    fe acc = F->one;
    for (int i = 64 * n - 1; i >= 0; i--) {
        f_mul(F, &acc, &acc, &acc);
        if ((e[i / 64] >> (i % 64)) & 1) f_mul(F, &acc, &acc, a);
    }
    *c = acc;
}
void f_inv(const field* F, fe* c, const fe* a) {
    u64 e[FE_LIMBS]; u64 two[FE_LIMBS] = {2};
    limbs_sub(e, F->mod, two, F->n);
    f_pow_limbs(F, c, a, e, F->n);
}
int f_from_be(const field* F, fe* c, const u8* be, int nbytes) {
    u64 l[FE_LIMBS] = {0};
    for (int i = 0; i < nbytes; i++) {
        int bit = 8 * (nbytes - 1 - i);
        if (bit / 64 >= FE_LIMBS) { if (be[i]) return -1; continue; }
        l[bit / 64] |= (u64)be[i] << (bit % 64);
    }
    for (int i = F->n; i < FE_LIMBS; i++) if (l[i]) return -1;
    if (limbs_geq(l, F->mod, F->n)) return -1;
    f_from_canon(F, c, l);
    return 0;
}
void f_to_be(const field* F, u8* be, int nbytes, const fe* a) {
    u64 l[FE_LIMBS] = {0};
    f_to_canon(F, l, a);
    for (int i = 0; i < nbytes; i++) {
        int bit = 8 * (nbytes - 1 - i);
        be[i] = bit / 64 < FE_LIMBS ? (u8)(l[bit / 64] >> (bit % 64)) : 0;
    }
}
/* Horner over bytes: value = sum be[i] 256^(len-1-i) reduced mod r */
void fr_from_be_wide(fe* c, const u8* be, int nbytes) {
    fe acc; f_zero(&acc);
    fe b256; f_from_u64(&FR, &b256, 256);
    for (int i = 0; i < nbytes; i++) {
        fe d; f_from_u64(&FR, &d, be[i]);
        f_mul(&FR, &acc, &acc, &b256);
        f_add(&FR, &acc, &acc, &d);
    }
    *c = acc;
}

static void field_setup(field* F, const big* m) {
    memset(F, 0, sizeof *F);
    F->bits = big_bits(m);
    F->n = (F->bits + 63) / 64;
    big_to_u64(F->mod, F->n, m);
    u64 inv = 1;                       /* Newton: inv = m0^{-1} mod 2^64 */
    for (int i = 0; i < 7; i++) inv *= 2 - F->mod[0] * inv;
    F->ninv = (u64)0 - inv;
    big R, R2, rem;
    big_set_u64(&R, 1);
    for (int i = 0; i < 64 * F->n; i++) big_add(&R, &R, &R);
    big_divmod(NULL, &rem, &R, m);
    big_to_u64(F->one.v, F->n, &rem);
    big_mul(&R2, &R, &R);
    big_divmod(NULL, &rem, &R2, m);
    big_to_u64(F->r2.v, F->n, &rem);
}

/* Miller-Rabin with the first twelve primes as bases (deterministic far beyond need
 * is not claimed; a composite passing all twelve is astronomically unlikely). */
static int is_probable_prime(const big* m) {
    field F; field_setup(&F, m);
    u64 mm1[FE_LIMBS] = {0}, one[FE_LIMBS] = {1};
    limbs_sub(mm1, F.mod, one, F.n);
    int s = 0; u64 d[FE_LIMBS]; memcpy(d, mm1, sizeof d);
    while (!(d[0] & 1)) {
        for (int i = 0; i < F.n; i++) d[i] = (d[i] >> 1) | (i + 1 < F.n ? d[i + 1] << 63 : 0);
        s++;
    }
    fe minus_one; f_from_canon(&F, &minus_one, mm1);
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int b = 0; b < 12; b++) {
        fe a, x; f_from_u64(&F, &a, bases[b]);
        f_pow_limbs(&F, &x, &a, d, F.n);
        if (f_eq(&F, &x, &F.one) || f_eq(&F, &x, &minus_one)) continue;
        int ok = 0;
        for (int k = 1; k < s; k++) {
            f_mul(&F, &x, &x, &x);
            if (f_eq(&F, &x, &minus_one)) { ok = 1; break; }
        }
        if (!ok) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------------------------------
 * Fq2 = Fq[u]/(u^2 + 1)
 * ------------------------------------------------------------------------------- */
void fq2_add(fq2* c, const fq2* a, const fq2* b) { f_add(&FQ, &c->c0, &a->c0, &b->c0); f_add(&FQ, &c->c1, &a->c1, &b->c1); }
void fq2_sub(fq2* c, const fq2* a, const fq2* b) { f_sub(&FQ, &c->c0, &a->c0, &b->c0); f_sub(&FQ, &c->c1, &a->c1, &b->c1); }
void fq2_neg(fq2* c, const fq2* a) { f_neg(&FQ, &c->c0, &a->c0); f_neg(&FQ, &c->c1, &a->c1); }
void fq2_mul(fq2* c, const fq2* a, const fq2* b) {
    fe t0, t1, t2, t3;
    f_mul(&FQ, &t0, &a->c0, &b->c0);
    f_mul(&FQ, &t1, &a->c1, &b->c1);
    f_mul(&FQ, &t2, &a->c0, &b->c1);
    f_mul(&FQ, &t3, &a->c1, &b->c0);
    f_sub(&FQ, &c->c0, &t0, &t1);
    f_add(&FQ, &c->c1, &t2, &t3);
}
void fq2_mul_fq(fq2* c, const fq2* a, const fe* b) { f_mul(&FQ, &c->c0, &a->c0, b); f_mul(&FQ, &c->c1, &a->c1, b); }
void fq2_inv(fq2* c, const fq2* a) {          /* (a0 - a1 u) / (a0^2 + a1^2) */
    fe n0, n1, inv;
    f_mul(&FQ, &n0, &a->c0, &a->c0);
    f_mul(&FQ, &n1, &a->c1, &a->c1);
    f_add(&FQ, &n0, &n0, &n1);
    f_inv(&FQ, &inv, &n0);
    fq2 t; t.c0 = a->c0; f_neg(&FQ, &t.c1, &a->c1);
    fq2_mul_fq(c, &t, &inv);
}
int fq2_is_zero(const fq2* a) { return f_is_zero(&FQ, &a->c0) && f_is_zero(&FQ, &a->c1); }
int fq2_eq(const fq2* a, const fq2* b) { return f_eq(&FQ, &a->c0, &b->c0) && f_eq(&FQ, &a->c1, &b->c1); }
void fq2_set_zero(fq2* a) { memset(a, 0, sizeof *a); }
void fq2_set_one(fq2* a) { fq2_set_zero(a); a->c0 = FQ.one; }

/* xi = 1 + u: (a0 + a1 u)(1 + u) = (a0 - a1) + (a0 + a1) u */
static void fq2_mul_xi(fq2* c, const fq2* a) {
    fq2 t;
    f_sub(&FQ, &t.c0, &a->c0, &a->c1);
    f_add(&FQ, &t.c1, &a->c0, &a->c1);
    *c = t;
}

/* ---------------------------------------------------------------------------------
 * Fq12 = Fq2[w]/(w^6 - xi), flat coefficients of w^0..w^5.
 * ------------------------------------------------------------------------------- */
void fq12_one(fq12* a) { memset(a, 0, sizeof *a); fq2_set_one(&a->c[0]); }

void fq12_mul(fq12* c, const fq12* a, const fq12* b) {
    fq2 t[11];
    for (int k = 0; k < 11; k++) fq2_set_zero(&t[k]);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            fq2 p; fq2_mul(&p, &a->c[i], &b->c[j]);
            fq2_add(&t[i + j], &t[i + j], &p);
        }
    for (int k = 10; k >= 6; k--) {            /* w^k = xi w^(k-6) */
        fq2 s; fq2_mul_xi(&s, &t[k]);
        fq2_add(&t[k - 6], &t[k - 6], &s);
    }
    for (int k = 0; k < 6; k++) c->c[k] = t[k];
}
/* the p^6-power Frobenius: w -> -w (v = w^2 is a non-square in Fq6) */
void fq12_conj(fq12* c, const fq12* a) {
    fq12 t = *a;
    fq2_neg(&t.c[1], &a->c[1]); fq2_neg(&t.c[3], &a->c[3]); fq2_neg(&t.c[5], &a->c[5]);
    *c = t;
}
int fq12_eq(const fq12* a, const fq12* b) {
    for (int k = 0; k < 6; k++) if (!fq2_eq(&a->c[k], &b->c[k])) return 0;
    return 1;
}
void fq12_pow_words(fq12* c, const fq12* a, const u32* e, int nwords) {
    fq12 acc; fq12_one(&acc);
    int top = 32 * nwords - 1;
    while (top >= 0 && !((e[top / 32] >> (top % 32)) & 1)) top--;
    for (int i = top; i >= 0; i--) {
        fq12_mul(&acc, &acc, &acc);
        if ((e[i / 32] >> (i % 32)) & 1) fq12_mul(&acc, &acc, a);
    }
    *c = acc;
}
void fq12_pow_fr(fq12* c, const fq12* a, const fe* k) {
    u64 l[FE_LIMBS] = {0}; f_to_canon(&FR, l, k);
    u32 w[8];
    for (int i = 0; i < 4; i++) { w[2 * i] = (u32)l[i]; w[2 * i + 1] = (u32)(l[i] >> 32); }
    fq12_pow_words(c, a, w, 8);
}
/* Tower order: Fq12 = Fq6 + Fq6 w with Fq6 = Fq2 + Fq2 v + Fq2 v^2, v = w^2, so the tower
 * coefficients (c0.c0, c0.c1, c0.c2, c1.c0, c1.c1, c1.c2) are the flat w^0, w^2, w^4, w^1, w^3, w^5. */
static const int TOWER_TO_FLAT[6] = {0, 2, 4, 1, 3, 5};
void fq12_to_bytes(u8 out[576], const fq12* a) {
    for (int t = 0; t < 6; t++) {
        const fq2* e = &a->c[TOWER_TO_FLAT[t]];
        f_to_be(&FQ, out + 96 * t, 48, &e->c0);
        f_to_be(&FQ, out + 96 * t + 48, 48, &e->c1);
    }
}
int fq12_from_bytes(fq12* a, const u8 in[576]) {
    for (int t = 0; t < 6; t++) {
        fq2* e = &a->c[TOWER_TO_FLAT[t]];
        if (f_from_be(&FQ, &e->c0, in + 96 * t, 48)) return -1;
        if (f_from_be(&FQ, &e->c1, in + 96 * t + 48, 48)) return -1;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Derivation of p, r and the final exponent from x, with the checks.
 * ------------------------------------------------------------------------------- */
static int g_inited = 0;
int or_curves_init(void);

int or_init(void) {
    if (g_inited) return 0;
    big ax, ax2, ax4, r, one, t, p, three, q, rem, h1;
    big_set_u64(&ax, 0xd201000000010000ull);          /* |x|, x = -|x| */
    big_set_u64(&one, 1);
    big_set_u64(&three, 3);
    big_mul(&ax2, &ax, &ax);
    big_mul(&ax4, &ax2, &ax2);
    big_sub(&r, &ax4, &ax2);                           /* r = x^4 - x^2 + 1 */
    big_add(&r, &r, &one);
    big_add(&t, &ax, &one);                            /* (x - 1)^2 = (|x| + 1)^2 */
    big_mul(&t, &t, &t);
    big_divmod(&h1, &rem, &t, &three);                 /* h1 = (x-1)^2 / 3 */
    if (rem.n != 0) return -1;
    big_mul(&p, &h1, &r);                              /* p = (x-1)^2 r / 3 + x */
    big_sub(&p, &p, &ax);
    if (!is_probable_prime(&p) || !is_probable_prime(&r)) return -2;
    if (big_bits(&p) != 381 || big_bits(&r) != 255) return -3;
    /* #E(Fq) = p + 1 - t with trace t = x + 1, i.e. p - x = p + |x| must equal h1 r */
    big_add(&t, &p, &ax);
    big_mul(&q, &h1, &r);
    if (big_cmp(&t, &q) != 0) return -4;
    field_setup(&FQ, &p);
    field_setup(&FR, &r);
    /* (p^12 - 1) / r, exactly */
    big p12; big_set_u64(&p12, 1);
    for (int i = 0; i < 12; i++) big_mul(&p12, &p12, &p);
    big_sub(&p12, &p12, &one);
    big_divmod(&q, &rem, &p12, &r);
    if (rem.n != 0) return -5;                         /* r | p^12 - 1 */
    memset(OR_EXP_FINAL, 0, sizeof OR_EXP_FINAL);
    for (int i = 0; i < q.n; i++) OR_EXP_FINAL[i] = q.w[i];
    OR_EXP_FINAL_WORDS = q.n;
    int rc = or_curves_init();
    if (rc) return rc;
    g_inited = 1;
    return 0;
}
