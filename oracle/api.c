/*
 * Byte-level entry points of the oracle for the test-suite (ctypes).  Every value crosses as
 * canonical big-endian bytes (Fq 48, Fr 32, G1 96, G2 192, GT 576).  Scalars for group
 * multiplications are plain 256-bit big-endian integers (not reduced), so the tests can
 * multiply by r itself.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"
#include <string.h>

int or_status(void) { return or_init(); }

static void be_to_limbs(u64 l[4], const u8 be[32]) {
    for (int i = 0; i < 4; i++) {
        l[i] = 0;
        for (int k = 0; k < 8; k++) l[i] |= (u64)be[31 - 8 * i - k] << (8 * k);
    }
}

/* which: 0 = p (48 B), 1 = r (32 B), 2 = final exponent (little-endian u32 words; returns count) */
int or_const(int which, u8* out) {
    if (or_init()) return -1;
    if (which == 0) { for (int i = 0; i < 48; i++) out[i] = (u8)(FQ.mod[(47 - i) / 8] >> (8 * ((47 - i) % 8))); return 48; }
    if (which == 1) { for (int i = 0; i < 32; i++) out[i] = (u8)(FR.mod[(31 - i) / 8] >> (8 * ((31 - i) % 8))); return 32; }
    if (which == 2) { memcpy(out, OR_EXP_FINAL, 4 * (size_t)OR_EXP_FINAL_WORDS); return OR_EXP_FINAL_WORDS; }
    return -1;
}

int or_fq_op(int op, const u8* a, const u8* b, u8* out) {
    fe x, y, z;
    if (f_from_be(&FQ, &x, a, 48)) return -1;
    if (op <= 2 && f_from_be(&FQ, &y, b, 48)) return -1;
    switch (op) {
        case 0: f_add(&FQ, &z, &x, &y); break;
        case 1: f_sub(&FQ, &z, &x, &y); break;
        case 2: f_mul(&FQ, &z, &x, &y); break;
        case 3: f_inv(&FQ, &z, &x); break;
        default: return -1;
    }
    f_to_be(&FQ, out, 48, &z);
    return 0;
}
int or_fr_op(int op, const u8* a, const u8* b, u8* out) {
    fe x, y, z;
    if (f_from_be(&FR, &x, a, 32)) return -1;
    if (op <= 2 && f_from_be(&FR, &y, b, 32)) return -1;
    switch (op) {
        case 0: f_add(&FR, &z, &x, &y); break;
        case 1: f_sub(&FR, &z, &x, &y); break;
        case 2: f_mul(&FR, &z, &x, &y); break;
        case 3: f_inv(&FR, &z, &x); break;
        default: return -1;
    }
    f_to_be(&FR, out, 32, &z);
    return 0;
}
/* Fq2 multiply: a, b are c0||c1 (96 B) */
int or_fq2_mul(const u8* a, const u8* b, u8* out) {
    fq2 x, y, z;
    if (f_from_be(&FQ, &x.c0, a, 48) || f_from_be(&FQ, &x.c1, a + 48, 48)) return -1;
    if (f_from_be(&FQ, &y.c0, b, 48) || f_from_be(&FQ, &y.c1, b + 48, 48)) return -1;
    fq2_mul(&z, &x, &y);
    f_to_be(&FQ, out, 48, &z.c0); f_to_be(&FQ, out + 48, 48, &z.c1);
    return 0;
}
int or_fr_wide(const u8* be, int n, u8* out) { fe z; fr_from_be_wide(&z, be, n); f_to_be(&FR, out, 32, &z); return 0; }

int or_fq12_mul(const u8* a, const u8* b, u8* out) {
    fq12 x, y, z;
    if (fq12_from_bytes(&x, a) || fq12_from_bytes(&y, b)) return -1;
    fq12_mul(&z, &x, &y); fq12_to_bytes(out, &z);
    return 0;
}
/* exponent: little-endian u32 words */
int or_fq12_pow(const u8* a, const u32* e, int nwords, u8* out) {
    fq12 x, z;
    if (fq12_from_bytes(&x, a)) return -1;
    fq12_pow_words(&z, &x, e, nwords); fq12_to_bytes(out, &z);
    return 0;
}
int or_fq12_conj(const u8* a, u8* out) {
    fq12 x; if (fq12_from_bytes(&x, a)) return -1;
    fq12_conj(&x, &x); fq12_to_bytes(out, &x);
    return 0;
}

int or_g1_gen(u8* out) { if (or_init()) return -1; g1_to_bytes(out, &G1_GEN); return 0; }
int or_g2_gen(u8* out) { if (or_init()) return -1; g2_to_bytes(out, &G2_GEN); return 0; }
int or_g1_mul(const u8* p, const u8* k, u8* out) {
    g1 P, Q; if (g1_from_bytes(&P, p)) return -1;
    u64 l[4]; be_to_limbs(l, k); g1_mul_limbs(&Q, &P, l); g1_to_bytes(out, &Q);
    return 0;
}
int or_g1_add(const u8* p, const u8* q, u8* out) {
    g1 P, Q, S; if (g1_from_bytes(&P, p) || g1_from_bytes(&Q, q)) return -1;
    g1_add(&S, &P, &Q); g1_to_bytes(out, &S);
    return 0;
}
int or_g1_dbl(const u8* p, u8* out) {
    g1 P, S; if (g1_from_bytes(&P, p)) return -1;
    g1_dbl(&S, &P); g1_to_bytes(out, &S);
    return 0;
}
int or_g2_mul(const u8* p, const u8* k, u8* out) {
    g2 P, Q; if (g2_from_bytes(&P, p)) return -1;
    u64 l[4]; be_to_limbs(l, k); g2_mul_limbs(&Q, &P, l); g2_to_bytes(out, &Q);
    return 0;
}
int or_g2_add(const u8* p, const u8* q, u8* out) {
    g2 P, Q, S; if (g2_from_bytes(&P, p) || g2_from_bytes(&Q, q)) return -1;
    g2_add(&S, &P, &Q); g2_to_bytes(out, &S);
    return 0;
}
/* validity of serialised points: 1 if on the curve (or identity), 0 otherwise */
int or_g1_valid(const u8* p) { g1 P; return g1_from_bytes(&P, p) == 0; }
int or_g2_valid(const u8* p) { g2 P; return g2_from_bytes(&P, p) == 0; }

int or_pairing(const u8* p, const u8* q, u8* out) {
    g1 P; g2 Q; if (g1_from_bytes(&P, p) || g2_from_bytes(&Q, q)) return -1;
    fq12 e; pairing(&e, &P, &Q); fq12_to_bytes(out, &e);
    return 0;
}
int or_miller(const u8* p, const u8* q, u8* out) {
    g1 P; g2 Q; if (g1_from_bytes(&P, p) || g2_from_bytes(&Q, q)) return -1;
    fq12 e; miller_loop(&e, &P, &Q); fq12_to_bytes(out, &e);
    return 0;
}
int or_final_exp(const u8* f, u8* out) {
    fq12 x, e; if (fq12_from_bytes(&x, f)) return -1;
    final_exp(&e, &x); fq12_to_bytes(out, &e);
    return 0;
}
/* naive multi-scalar multiplication sum k_i P_i (double-and-add per term) */
int or_g1_msm(const u8* pts, const u8* ks, u32 n, u8* out) {
    g1 acc; g1_set_inf(&acc);
    for (u32 i = 0; i < n; i++) {
        g1 P, T; if (g1_from_bytes(&P, pts + 96 * (size_t)i)) return -1;
        u64 l[4]; be_to_limbs(l, ks + 32 * (size_t)i);
        g1_mul_limbs(&T, &P, l); g1_add(&acc, &acc, &T);
    }
    g1_to_bytes(out, &acc);
    return 0;
}

int or_sha256(const u8* msg, size_t len, u8* out) { sha256(out, msg, len); return 0; }
int or_hfr(const char* tag, const u8* data, size_t len, u8* out) {
    if (or_init()) return -1;
    fe z; hfr(&z, tag, data, len); f_to_be(&FR, out, 32, &z);
    return 0;
}
/* n rejection-sampled Fr draws of SplitMix64 seeded with `seed`, canonical LE limbs */
int or_splitmix_fr(u64 seed, u32 n, u64* out) {
    if (or_init()) return -1;
    splitmix s = {seed};
    for (u32 i = 0; i < n; i++) splitmix_fr(&s, out + 4 * (size_t)i);
    return 0;
}
