/*
 * FlexProofs CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded-per-call CPU restatement of what the FlexProofs
 * ProveAll path computes, written from the paper (arXiv 2601.03031):
 *   - the bilinear group (BLS12-381 here; the paper used BN_SNARK1, Sec. 5),
 *   - PST multilinear commitments with HyperEval (Sec. 2.2),
 *   - the functional commitment FC.Setup/Commit/BOpen/BVerify (Sec. 3, Eq. folding,
 *     Eq. comy, "Faster verification"),
 *   - VC.Setup/Commit (Sec. 4.1, Eqs. vcpp, genCi, genC), OpenAll (Protocol 1 and the
 *     Sub-protocol, Sec. 4.2), the unit-vector shortcut (Sec. 4.3, Eq. b_l), and the
 *     verifier-side combination (Appendix C, correctness proof).
 *
 * Only the tests, the package's smoke() and bench.py's CPU-baseline leg may load this
 * library.  It shares no code, header, table or constant generator with the CUDA path.
 *
 * Arithmetic: generic Montgomery residues over 64-bit limbs; p and r are DERIVED from
 * the BLS12-381 seed x = -0xd201000000010000 at start-up and checked (primality,
 * r | p^12 - 1, #E(Fq) = p - x = h1 * r).  Fq12 is kept FLAT as Fq2[w]/(w^6 - (1+u)),
 * which is isomorphic to the usual tower (v = w^2); serialisation maps it to tower order.
 * The pairing is the optimal-ate Miller loop f_{|x|,Q}(P) with affine line functions,
 * conjugated (x < 0), raised by plain square-and-multiply to exactly (p^12-1)/r.
 */
#ifndef FLEXPROOFS_ORACLE_H
#define FLEXPROOFS_ORACLE_H

#include <stddef.h>
#include <stdint.h>

typedef uint64_t u64;
typedef uint32_t u32;
typedef uint8_t u8;
typedef unsigned __int128 u128;

#define FE_LIMBS 6

/* A residue (Montgomery form) of FQ or FR, little-endian 64-bit limbs. */
typedef struct { u64 v[FE_LIMBS]; } fe;

typedef struct {
    int n;              /* 64-bit limbs in use (6 for Fq, 4 for Fr) */
    int bits;           /* bit length of the modulus */
    u64 mod[FE_LIMBS];
    u64 ninv;           /* -mod^{-1} mod 2^64 */
    fe r2;              /* 2^(128 n) mod m (plain integer) */
    fe one;             /* Montgomery form of 1 */
} field;

extern field FQ, FR;

typedef struct { fe c0, c1; } fq2;          /* c0 + c1 u, u^2 = -1 */
typedef struct { fq2 c[6]; } fq12;          /* sum c[k] w^k, w^6 = 1 + u */

typedef struct { fe X, Y, Z; } g1;          /* Jacobian; Z = 0 is the identity */
typedef struct { fq2 X, Y, Z; } g2;

/* --- derived constants ------------------------------------------------------ */
int  or_init(void);                                     /* 0 on success */
extern u32 OR_EXP_FINAL[160];                           /* (p^12-1)/r, little-endian 32-bit words */
extern int OR_EXP_FINAL_WORDS;

/* --- operation counters ---------------------------------------------------------
 * Miller loops, final exponentiations and G1 / G2 scalar multiplications since the last reset,
 * over all threads: the efficiency statements of Sec. 3 (pairings and exponentiations per
 * algorithm) are checked against them. */
enum { OR_OP_MILLER = 0, OR_OP_FINAL_EXP = 1, OR_OP_G1_MUL = 2, OR_OP_G2_MUL = 3, OR_OP_KINDS = 4 };
void or_op_count(int kind);
void or_ops_reset(void);
void or_ops_get(u64 out[OR_OP_KINDS]);

/* --- field ------------------------------------------------------------------- */
void f_add(const field* F, fe* c, const fe* a, const fe* b);
void f_sub(const field* F, fe* c, const fe* a, const fe* b);
void f_neg(const field* F, fe* c, const fe* a);
void f_mul(const field* F, fe* c, const fe* a, const fe* b);
void f_inv(const field* F, fe* c, const fe* a);         /* a^(m-2); 0 -> 0 */
int  f_is_zero(const field* F, const fe* a);
int  f_eq(const field* F, const fe* a, const fe* b);
void f_zero(fe* a);
void f_from_canon(const field* F, fe* c, const u64* limbs);   /* limbs < m */
void f_to_canon(const field* F, u64* limbs, const fe* a);
void f_from_u64(const field* F, fe* c, u64 x);
int  f_from_be(const field* F, fe* c, const u8* be, int nbytes);   /* -1 if >= m */
void f_to_be(const field* F, u8* be, int nbytes, const fe* a);
void fr_from_be_wide(fe* c, const u8* be, int nbytes);             /* any length, mod r */

void fq2_add(fq2* c, const fq2* a, const fq2* b);
void fq2_sub(fq2* c, const fq2* a, const fq2* b);
void fq2_neg(fq2* c, const fq2* a);
void fq2_mul(fq2* c, const fq2* a, const fq2* b);
void fq2_mul_fq(fq2* c, const fq2* a, const fe* b);
void fq2_inv(fq2* c, const fq2* a);
int  fq2_is_zero(const fq2* a);
int  fq2_eq(const fq2* a, const fq2* b);
void fq2_set_zero(fq2* a);
void fq2_set_one(fq2* a);

void fq12_one(fq12* a);
void fq12_mul(fq12* c, const fq12* a, const fq12* b);
void fq12_conj(fq12* c, const fq12* a);
int  fq12_eq(const fq12* a, const fq12* b);
void fq12_pow_words(fq12* c, const fq12* a, const u32* e, int nwords);
void fq12_pow_fr(fq12* c, const fq12* a, const fe* k);      /* k an Fr residue */
void fq12_to_bytes(u8 out[576], const fq12* a);               /* tower order, BE */
int  fq12_from_bytes(fq12* a, const u8 in[576]);

/* --- curves -------------------------------------------------------------------- */
extern g1 G1_GEN;
extern g2 G2_GEN;
void g1_set_inf(g1* p);
int  g1_is_inf(const g1* p);
void g1_dbl(g1* r, const g1* p);
void g1_add(g1* r, const g1* p, const g1* q);
void g1_neg(g1* r, const g1* p);
void g1_mul(g1* r, const g1* p, const fe* k);                /* k an Fr residue */
void g1_mul_limbs(g1* r, const g1* p, const u64 l[4]);       /* plain 256-bit integer */
void g1_affine(fe* x, fe* y, const g1* p);
int  g1_eq(const g1* p, const g1* q);
int  g1_on_curve(const g1* p);
void g1_to_bytes(u8 out[96], const g1* p);
int  g1_from_bytes(g1* p, const u8 in[96]);

void g2_set_inf(g2* p);
int  g2_is_inf(const g2* p);
void g2_dbl(g2* r, const g2* p);
void g2_add(g2* r, const g2* p, const g2* q);
void g2_neg(g2* r, const g2* p);
void g2_mul(g2* r, const g2* p, const fe* k);
void g2_mul_limbs(g2* r, const g2* p, const u64 l[4]);
void g2_affine(fq2* x, fq2* y, const g2* p);
int  g2_eq(const g2* p, const g2* q);
int  g2_on_curve(const g2* p);
void g2_to_bytes(u8 out[192], const g2* p);
int  g2_from_bytes(g2* p, const u8 in[192]);

void miller_loop(fq12* f, const g1* P, const g2* Q);         /* conjugated f_{|x|,Q}(P) */
void final_exp(fq12* r, const fq12* f);                       /* f^((p^12-1)/r) */
void pairing(fq12* r, const g1* P, const g2* Q);

/* --- hashing ----------------------------------------------------------------- */
void sha256(u8 out[32], const u8* msg, size_t len);
void hfr(fe* out, const char* tag, const u8* data, size_t len);   /* Fr residue */
void hfr_nonzero(fe* out, const char* tag, const u8* data, size_t len);

/* --- PRNG (SplitMix64) ------------------------------------------------------------ */
typedef struct { u64 state; } splitmix;
u64  splitmix_next(splitmix* s);
void splitmix_fr(splitmix* s, u64 limbs[4]);                  /* canonical, rejection-sampled */

#endif
