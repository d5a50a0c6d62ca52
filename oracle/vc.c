/*
 * Oracle protocol layer: PST (Sec. 2.2 with HyperEval), FC (Sec. 3), FlexProofs VC
 * (Sec. 4: Setup, Commit, OpenAll = Protocol 1 + Sub-protocol + the Fiat-Shamir Merkle tree,
 * the unit-vector shortcut of Sec. 4.3, and Verify as in the correctness proof of Appendix C).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Exported entry points are prefixed or_ and take
 * canonical big-endian byte strings, so the tests can drive them through ctypes.
 *
 * Notation: N = 2^n, R = 2^floor(n/2) rows (FC length, l_R = log R), M = 2^ceil(n/2) columns
 * (PST variables l_c = log M), i = j M + a, blocks S_k = [k b, min((k+1) b, R)).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - serialisation: Fr 32 B, G1 96 B (x||y), G2 192 B (x.c0||x.c1||y.c0||y.c1), GT 576 B in
 *     tower order, all canonical big-endian; the identity is all-zero bytes;
 *   - the FC statement hashed for r_a is C || u32be(k) || u32be(b) || u32be(|S_k|) || D_k with D_k
 *     the root of a binary tree over the block's C_a (leaves SHA256("FP-sleaf"||C_a) in row order,
 *     nodes SHA256("FP-snode"||left||right) pairing each level left to right, an odd last node
 *     carried up unchanged), and r_a = HFr("FP-r", SHA256(statement) || u32be(a));
 *   - x_j = HFr("FP-x", x_{j-1} || L_j.T || L_j.1 || R_j.T || R_j.1), x_0 the empty string;
 *   - v_l is proven KZG-style in G2: z = HFr("FP-z", x_l || v_l),
 *     W = g2^{(P(beta)-P(z))/(beta-z)}, P(X) = prod_j (1 + x_j^{-1} X^{2^{l_R-j+1}});
 *   - the Step-2 Merkle tree is two-level: element leaves SHA256("FP-leaf"||u64be(i)||m_i),
 *     per-row trees, row leaves SHA256("FP-row"||s_j||C_j), a tree over the rows;
 *     nodes SHA256("FP-node"||left||right); r_j = HFr("FP-rho", root || u32be(j));
 *   - PST: variable x_t pairs with bit t of the column index; Lambda_t[c] = g1^{eq_t(c, tau)}.
 */
#include "oracle.h"
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* Memo of verifier sub-checks (FC.BVerify per block, PST.Verify per column), keyed by the
 * SHA-256 of every input the sub-check reads, so a tampered input can never hit a stale entry. */
#define MEMO_SLOTS (1u << 16)
static pthread_mutex_t memo_mu = PTHREAD_MUTEX_INITIALIZER;
static struct { u8 key[32]; u8 used, val; } memo[MEMO_SLOTS];
static int memo_get(const u8 key[32], int* val) {
    int hit = 0;
    pthread_mutex_lock(&memo_mu);
    u32 h = ((u32)key[0] << 8 | key[1]) & (MEMO_SLOTS - 1);
    for (u32 p = 0; p < 64; p++) {
        u32 s = (h + p) & (MEMO_SLOTS - 1);
        if (!memo[s].used) break;
        if (!memcmp(memo[s].key, key, 32)) { *val = memo[s].val; hit = 1; break; }
    }
    pthread_mutex_unlock(&memo_mu);
    return hit;
}
static void memo_put(const u8 key[32], int val) {
    pthread_mutex_lock(&memo_mu);
    u32 h = ((u32)key[0] << 8 | key[1]) & (MEMO_SLOTS - 1);
    for (u32 p = 0; p < 64; p++) {
        u32 s = (h + p) & (MEMO_SLOTS - 1);
        if (!memo[s].used || !memcmp(memo[s].key, key, 32)) {
            memcpy(memo[s].key, key, 32); memo[s].used = 1; memo[s].val = (u8)val; break;
        }
    }
    pthread_mutex_unlock(&memo_mu);
}
static void memo_key(u8 out[32], const char* kind, const void* pp_id, size_t pp_len,
                     const u8* a, size_t al, const u8* b, size_t bl, const u8* c, size_t cl) {
    size_t kl = strlen(kind), n = kl + pp_len + al + bl + cl;
    u8* buf = (u8*)malloc(n ? n : 1); size_t o = 0;
    memcpy(buf + o, kind, kl); o += kl;
    memcpy(buf + o, pp_id, pp_len); o += pp_len;
    if (al) { memcpy(buf + o, a, al); o += al; }
    if (bl) { memcpy(buf + o, b, bl); o += bl; }
    if (cl) { memcpy(buf + o, c, cl); o += cl; }
    sha256(out, buf, o);
    free(buf);
}

/* ------------------------------------------------------------------------------- */
typedef struct {
    int log_n, log_r, log_c;
    u32 R, M;
    u64 seed;
    fe beta, tau[32];
    g1* lam;           /* Lambda_t at offset 2^t - 1, t = 0..l_c; 2M - 1 points */
    g1 g1beta;
    g2* g2pow;         /* g2^{beta^i}, i < 2R - 1; v_i = g2pow[2 i] */
    g2* g2tau;         /* g2^{tau_t}, t < l_c */
} or_pp;

static void be32(u8* o, u32 x) { o[0] = (u8)(x >> 24); o[1] = (u8)(x >> 16); o[2] = (u8)(x >> 8); o[3] = (u8)x; }
static void be64(u8* o, u64 x) { for (int i = 0; i < 8; i++) o[i] = (u8)(x >> (56 - 8 * i)); }
static void fr_to_bytes(u8 o[32], const fe* a) { f_to_be(&FR, o, 32, a); }

static const g1* LAM(const or_pp* pp, int t) { return pp->lam + ((1u << t) - 1); }

/* multi-pairing prod_i e(P_i, Q_i) = (prod_i f_i)^((p^12-1)/r): one final exponentiation */
static void multi_pairing(fq12* out, const g1* P, const g2* Q, int n, int stride_q) {
    fq12 acc; fq12_one(&acc);
    for (int i = 0; i < n; i++) {
        fq12 f; miller_loop(&f, &P[i], &Q[(size_t)i * stride_q]);
        fq12_mul(&acc, &acc, &f);
    }
    final_exp(out, &acc);
}

/* eq_t(c, tau) = prod_{s<t} (c_s tau_s + (1 - c_s)(1 - tau_s)) -- Eq. multi-extension's basis */
static void eq_weight(fe* w, const or_pp* pp, int t, u32 c) {
    fe acc = FR.one;
    for (int s = 0; s < t; s++) {
        fe f;
        if ((c >> s) & 1) f = pp->tau[s];
        else f_sub(&FR, &f, &FR.one, &pp->tau[s]);
        f_mul(&FR, &acc, &acc, &f);
    }
    *w = acc;
}

/* VC.Setup (Eq. vcpp): pp_PC for l_c variables (Lambda tables, g2^tau) and pp_FC of size R
 * with the faster-verification extras (all g2^{beta^i}, i < 2R - 1, and g1^beta).  R = 2^l_R
 * segments of M = 2^l_c elements (OpenAll for sub-arrays, Sec. 4.4, partitions m into any number
 * of equal segments); or_setup takes l_R = floor(n/2).  The trapdoor stream draws beta, then
 * tau_0, tau_1, ...: the tables of a smaller split are prefixes of a larger split's. */
or_pp* or_setup_split(u32 log_r, u32 log_c, u64 seed) {
    if (or_init()) return NULL;
    if (log_r < 1 || log_c < 1 || log_r > 13 || log_r + log_c > 26) return NULL;
    or_pp* pp = (or_pp*)calloc(1, sizeof *pp);
    pp->log_n = (int)(log_r + log_c); pp->log_r = (int)log_r; pp->log_c = (int)log_c;
    pp->R = 1u << pp->log_r; pp->M = 1u << pp->log_c; pp->seed = seed;
    splitmix s = {seed ^ 0x5eed5eedull};
    u64 l[4];
    splitmix_fr(&s, l); f_from_canon(&FR, &pp->beta, l);
    for (int t = 0; t < pp->log_c; t++) { splitmix_fr(&s, l); f_from_canon(&FR, &pp->tau[t], l); }
    pp->lam = (g1*)calloc(2 * (size_t)pp->M - 1, sizeof(g1));
    for (int t = 0; t <= pp->log_c; t++)
        for (u32 c = 0; c < (1u << t); c++) {
            fe w; eq_weight(&w, pp, t, c);
            g1_mul(&pp->lam[(1u << t) - 1 + c], &G1_GEN, &w);
        }
    g1_mul(&pp->g1beta, &G1_GEN, &pp->beta);
    pp->g2pow = (g2*)calloc(2 * (size_t)pp->R - 1, sizeof(g2));
    fe bp = FR.one;
    for (u32 i = 0; i < 2 * pp->R - 1; i++) {
        g2_mul(&pp->g2pow[i], &G2_GEN, &bp);
        f_mul(&FR, &bp, &bp, &pp->beta);
    }
    pp->g2tau = (g2*)calloc((size_t)pp->log_c + 1, sizeof(g2));
    for (int t = 0; t < pp->log_c; t++) g2_mul(&pp->g2tau[t], &G2_GEN, &pp->tau[t]);
    return pp;
}
or_pp* or_setup(u32 log_n, u64 seed) {
    if (log_n < 2 || log_n > 26) return NULL;
    return or_setup_split(log_n / 2, log_n - log_n / 2, seed);
}
void or_pp_free(or_pp* pp) {
    if (!pp) return;
    free(pp->lam); free(pp->g2pow); free(pp->g2tau); free(pp);
}
void or_pp_info(const or_pp* pp, u32 out[4]) { out[0] = (u32)pp->log_n; out[1] = pp->R; out[2] = pp->M; out[3] = (u32)pp->log_c; }
/* serialised pp: Lambda (2M-1)x96 || g1beta 96 || g2pow (2R-1)x192 || g2tau l_c x192 */
size_t or_pp_bytes(const or_pp* pp, u8* out) {
    size_t n = 0;
    for (u32 i = 0; i < 2 * pp->M - 1; i++) { if (out) g1_to_bytes(out + n, &pp->lam[i]); n += 96; }
    if (out) g1_to_bytes(out + n, &pp->g1beta);
    n += 96;
    for (u32 i = 0; i < 2 * pp->R - 1; i++) { if (out) g2_to_bytes(out + n, &pp->g2pow[i]); n += 192; }
    for (int t = 0; t < pp->log_c; t++) { if (out) g2_to_bytes(out + n, &pp->g2tau[t]); n += 192; }
    return n;
}
/* the trapdoor, for closed-form tests only: beta || tau_0 .. tau_{l_c-1}, 32 B each */
void or_pp_trapdoor(const or_pp* pp, u8* out) {
    fr_to_bytes(out, &pp->beta);
    for (int t = 0; t < pp->log_c; t++) fr_to_bytes(out + 32 * (t + 1), &pp->tau[t]);
}

/* m is N x 4 little-endian u64 canonical limbs */
static int load_m(fe* out, const u64* m, size_t N) {
    for (size_t i = 0; i < N; i++) {
        const u64* l = m + 4 * i;
        for (int k = 3; k >= 0; k--) {
            if (l[k] != FR.mod[k]) { if (l[k] > FR.mod[k]) return -1; break; }
            if (k == 0) return -1;        /* equal to r */
        }
        f_from_canon(&FR, &out[i], l);
    }
    return 0;
}

/* ------------------------------------------------------------------------------
 * VC.Commit (Eqs. genCi, genC): C_j = PC.Commit(f_j) = sum_a m[jM + a] Lambda_{l_c}[a] (naive
 * double-and-add per term), C = FC.Commit(C) = prod_j e(C_j, v_j).
 * ------------------------------------------------------------------------------ */
int or_commit(const or_pp* pp, const u64* m, u8* C_out, u8* rows_out) {
    size_t N = (size_t)pp->R * pp->M;
    fe* mm = (fe*)malloc(N * sizeof(fe));
    if (load_m(mm, m, N)) { free(mm); return -1; }
    g1* rows = (g1*)malloc(pp->R * sizeof(g1));
    const g1* L = LAM(pp, pp->log_c);
    for (u32 j = 0; j < pp->R; j++) {
        g1 acc; g1_set_inf(&acc);
        for (u32 a = 0; a < pp->M; a++) {
            g1 t; g1_mul(&t, &L[a], &mm[(size_t)j * pp->M + a]);
            g1_add(&acc, &acc, &t);
        }
        rows[j] = acc;
        g1_to_bytes(rows_out + 96 * (size_t)j, &acc);
    }
    fq12 C; multi_pairing(&C, rows, pp->g2pow, (int)pp->R, 2);
    fq12_to_bytes(C_out, &C);
    free(rows); free(mm);
    return 0;
}

/* ------------------------------------------------------------------------------
 * FC.BOpen for block k (Sec. 3, Eq. b and Eq. folding; Protocol 1 Step 1, Eq. genFCBatchProof)
 * with b = sum_{a in S_k} r_a u_a, plus the faster-verification proof of v_l.
 * Output layout: per round j = 1..l_R: L_j.T(576) L_j.1(96) R_j.T(576) R_j.1(96);
 * then A_l(96) v_l(192) W(192).
 * If invariant_fail is non-NULL the FC correctness invariant C_j = (A_j*v_j, <A_j, b_j>) of
 * the correctness proof (Sec. 3) is checked after every round (slow).
 * ------------------------------------------------------------------------------ */
size_t or_bopen_len(const or_pp* pp) { return (size_t)pp->log_r * 1344 + 480; }

/* D_k: the tree over the nk >= 1 row commitments ca[0 .. nk - 1] (96 bytes each), level by level */
static void stmt_rows_root(u8 out[32], const u8* ca, u32 nk) {
    u8* lv = (u8*)malloc(32 * (size_t)nk);
    for (u32 t = 0; t < nk; t++) {
        u8 buf[8 + 96];
        memcpy(buf, "FP-sleaf", 8);
        memcpy(buf + 8, ca + 96 * (size_t)t, 96);
        sha256(lv + 32 * (size_t)t, buf, sizeof buf);
    }
    for (u32 n = nk; n > 1;) {
        u32 m = 0;
        for (u32 i = 0; i + 1 < n; i += 2, m++) {
            u8 buf[8 + 64];
            memcpy(buf, "FP-snode", 8);
            memcpy(buf + 8, lv + 32 * (size_t)i, 64);
            sha256(lv + 32 * (size_t)m, buf, sizeof buf);
        }
        if (n & 1) { memmove(lv + 32 * (size_t)m, lv + 32 * (size_t)(n - 1), 32); m++; }
        n = m;
    }
    memcpy(out, lv, 32);
    free(lv);
}

static void block_challenges(fe* r_out, const u8* C, const u8* rows, u32 R, u32 b, u32 k, u32* nk_out) {
    u32 lo = k * b, hi = (k + 1) * b < R ? (k + 1) * b : R, nk = hi - lo;
    u8 stmt[576 + 12 + 32];
    memcpy(stmt, C, 576);
    be32(stmt + 576, k); be32(stmt + 580, b); be32(stmt + 584, nk);
    stmt_rows_root(stmt + 588, rows + 96 * (size_t)lo, nk);
    u8 buf[36];
    sha256(buf, stmt, sizeof stmt);
    for (u32 a = lo; a < hi; a++) {
        be32(buf + 32, a);
        hfr(&r_out[a - lo], "FP-r", buf, 36);
    }
    *nk_out = nk;
}

/* FC.BOpen rounds, y's opening and the faster-verification proof for the combined vector bv (R
 * entries) over A = the row commitments, v_i = g2^{beta^{2i}}; A, v, bv are consumed. */
static int fc_bopen_core(const or_pp* pp, const u8* C_bytes, g1* A, g2* v, fe* bv, u8* out, int check_invariant) {
    const u32 R = pp->R; const int lr = pp->log_r;
    /* invariant state: C_0 = (C, y) with y = <A, b> */
    fq12 invT; g1 inv1;
    if (check_invariant) {
        fq12_from_bytes(&invT, C_bytes);
        g1_set_inf(&inv1);
        for (u32 i = 0; i < R; i++) { g1 t; g1_mul(&t, &A[i], &bv[i]); g1_add(&inv1, &inv1, &t); }
    }
    int bad = 0;

    u8 xprev[32]; size_t xl = 0;
    fe xs[32], xinv[32];
    u8* o = out;
    for (int j = 1; j <= lr; j++) {
        u32 h = R >> j;
        fq12 LT, RT; g1 L1, R1;
        multi_pairing(&LT, A + h, v, (int)h, 1);           /* (A_R) * (v_L) */
        multi_pairing(&RT, A, v + h, (int)h, 1);           /* (A_L) * (v_R) */
        g1_set_inf(&L1); g1_set_inf(&R1);
        for (u32 i = 0; i < h; i++) {
            g1 t;
            g1_mul(&t, &A[h + i], &bv[i]); g1_add(&L1, &L1, &t);     /* <A_R, b_L> */
            g1_mul(&t, &A[i], &bv[h + i]); g1_add(&R1, &R1, &t);     /* <A_L, b_R> */
        }
        u8 tr[32 + 576 + 96 + 576 + 96];
        size_t tl = 0;
        memcpy(tr, xprev, xl); tl += xl;
        fq12_to_bytes(tr + tl, &LT); tl += 576;
        g1_to_bytes(tr + tl, &L1); tl += 96;
        fq12_to_bytes(tr + tl, &RT); tl += 576;
        g1_to_bytes(tr + tl, &R1); tl += 96;
        memcpy(o, tr + xl, 1344); o += 1344;
        fe x; hfr_nonzero(&x, "FP-x", tr, tl);
        fe xi; f_inv(&FR, &xi, &x);
        xs[j - 1] = x; xinv[j - 1] = xi;
        fr_to_bytes(xprev, &x); xl = 32;
        for (u32 i = 0; i < h; i++) {
            g1 t; g1_mul(&t, &A[h + i], &x); g1_add(&A[i], &A[i], &t);          /* A_L o A_R^x */
            g2 u; g2_mul(&u, &v[h + i], &xi); g2_add(&v[i], &v[i], &u);         /* v_L o v_R^{1/x} */
            fe w; f_mul(&FR, &w, &bv[h + i], &xi); f_add(&FR, &bv[i], &bv[i], &w); /* b_L + b_R / x */
        }
        if (check_invariant) {
            /* C_j = L_j^{x_j} o C_{j-1} o R_j^{1/x_j} must equal (A_j * v_j, <A_j, b_j>) */
            fq12 t1, t2; fq12_pow_fr(&t1, &LT, &x); fq12_pow_fr(&t2, &RT, &xi);
            fq12_mul(&invT, &invT, &t1); fq12_mul(&invT, &invT, &t2);
            g1 s1, s2; g1_mul(&s1, &L1, &x); g1_mul(&s2, &R1, &xi);
            g1_add(&inv1, &inv1, &s1); g1_add(&inv1, &inv1, &s2);
            fq12 lhsT; multi_pairing(&lhsT, A, v, (int)h, 1);
            g1 lhs1; g1_set_inf(&lhs1);
            for (u32 i = 0; i < h; i++) { g1 t; g1_mul(&t, &A[i], &bv[i]); g1_add(&lhs1, &lhs1, &t); }
            if (!fq12_eq(&lhsT, &invT) || !g1_eq(&lhs1, &inv1)) bad = 1;
        }
    }
    g1_to_bytes(o, &A[0]); o += 96;
    g2_to_bytes(o, &v[0]); o += 192;

    /* faster verification: z = H'(x_l, v_l), W = g2^{q(beta)}, q = (P - P(z)) / (X - z) */
    u8 zb[32 + 192];
    memcpy(zb, xprev, 32); g2_to_bytes(zb + 32, &v[0]);
    fe z; hfr(&z, "FP-z", zb, sizeof zb);
    u32 deg = 2 * R - 2;
    fe* P = (fe*)calloc(deg + 1, sizeof(fe));
    P[0] = FR.one;
    u32 cur = 0;                                            /* current degree */
    for (int j = 1; j <= lr; j++) {                         /* P *= (1 + x_j^{-1} X^{2^{l_R-j+1}}) */
        u32 e = 1u << (lr - j + 1);
        for (int d = (int)cur; d >= 0; d--) {
            fe t; f_mul(&FR, &t, &P[d], &xinv[j - 1]);
            f_add(&FR, &P[d + e], &P[d + e], &t);
        }
        cur += e;
    }
    fe* q = (fe*)calloc(deg > 0 ? deg : 1, sizeof(fe));
    if (deg > 0) {                                          /* synthetic division by (X - z) */
        q[deg - 1] = P[deg];
        for (int i = (int)deg - 1; i >= 1; i--) {
            fe t; f_mul(&FR, &t, &z, &q[i]);
            f_add(&FR, &q[i - 1], &P[i], &t);
        }
    }
    g2 W; g2_set_inf(&W);
    for (u32 i = 0; i < deg; i++) { g2 t; g2_mul(&t, &pp->g2pow[i], &q[i]); g2_add(&W, &W, &t); }
    g2_to_bytes(o, &W); o += 192;
    (void)xs;
    free(P); free(q);
    return bad ? 1 : 0;
}

int or_bopen(const or_pp* pp, const u8* C_bytes, const u8* rows_bytes, u32 b, u32 k, u8* out, int check_invariant) {
    const u32 R = pp->R;
    if (b < 1 || b > R || k * b >= R) return -1;
    g1* A = (g1*)malloc(R * sizeof(g1));
    g2* v = (g2*)malloc(R * sizeof(g2));
    fe* bv = (fe*)calloc(R, sizeof(fe));
    fe* rr = (fe*)malloc(b * sizeof(fe));
    for (u32 i = 0; i < R; i++) {
        if (g1_from_bytes(&A[i], rows_bytes + 96 * (size_t)i)) { free(A); free(v); free(bv); free(rr); return -2; }
        v[i] = pp->g2pow[2 * i];
    }
    u32 nk;
    block_challenges(rr, C_bytes, rows_bytes, R, b, k, &nk);
    for (u32 a = 0; a < nk; a++) bv[k * b + a] = rr[a];
    int rc = fc_bopen_core(pp, C_bytes, A, v, bv, out, check_invariant);
    free(A); free(v); free(bv); free(rr);
    return rc;
}

/* ------------------------------------------------------------------------------
 * Step 2 (Protocol 1 Step 2, Sub-protocol, Fiat-Shamir Merkle tree) and assembly.
 * ------------------------------------------------------------------------------ */
typedef struct {
    const or_pp* pp;
    u32 b, K;
    u8 C[576];
    u8* rows;          /* R x 96 */
    fe* m;             /* N residues */
    u64* m_raw;        /* N x 4 canonical */
    u8* blocks;        /* K x bopen_len */
    u8* blk_done;
    u8* row_tree;      /* R x (2M-1) digests: level l at offset (2M - 2M/2^l) */
    u8* top_tree;      /* (2R-1) digests, same level layout */
    fe* rj;            /* R */
    fe* gt;            /* fold tables, level h node s at ((2R - 2R/2^h) + s) x M */
    g1* D;             /* fold commitments, same node order */
    g1* pst;           /* HyperEval: level t prefix p at ((M/2^(t+1)) - 1 ... ) see pst_index */
    int step2_done;
} or_prover;

static size_t lvl_off(u32 leaves, int l) { return 2 * (size_t)leaves - 2 * (size_t)(leaves >> l); }
static size_t pst_index(u32 M, int t, u32 prefix) {
    /* level t has M / 2^(t+1) prefixes; levels stored from t = 0 upward */
    size_t off = 0;
    for (int s = 0; s < t; s++) off += M >> (s + 1);
    return off + prefix;
}

static void node_hash(u8 out[32], const u8 l[32], const u8 r[32]) {
    u8 buf[7 + 64]; memcpy(buf, "FP-node", 7); memcpy(buf + 7, l, 32); memcpy(buf + 39, r, 32);
    sha256(out, buf, sizeof buf);
}
static void leaf_hash(u8 out[32], u64 i, const u8 mi[32]) {
    u8 buf[7 + 8 + 32]; memcpy(buf, "FP-leaf", 7); be64(buf + 7, i); memcpy(buf + 15, mi, 32);
    sha256(out, buf, sizeof buf);
}
static void row_hash(u8 out[32], const u8 s[32], const u8 Cj[96]) {
    u8 buf[6 + 32 + 96]; memcpy(buf, "FP-row", 6); memcpy(buf + 6, s, 32); memcpy(buf + 38, Cj, 96);
    sha256(out, buf, sizeof buf);
}
/* build all levels of a binary tree whose leaves (count n) are at tree[0..n) */
static void build_tree(u8* tree, u32 n) {
    int levels = 0; while ((1u << levels) < n) levels++;
    for (int l = 1; l <= levels; l++) {
        u8* prev = tree + 32 * lvl_off(n, l - 1);
        u8* cur = tree + 32 * lvl_off(n, l);
        for (u32 s = 0; s < (n >> l); s++) node_hash(cur + 32 * s, prev + 64 * s, prev + 64 * s + 32);
    }
}

or_prover* or_prover_new(const or_pp* pp, const u64* m, const u8* C, const u8* rows, u32 b) {
    if (b < 1 || b > pp->R) return NULL;
    size_t N = (size_t)pp->R * pp->M;
    or_prover* P = (or_prover*)calloc(1, sizeof *P);
    P->pp = pp; P->b = b; P->K = (pp->R + b - 1) / b;
    memcpy(P->C, C, 576);
    P->rows = (u8*)malloc(96 * (size_t)pp->R); memcpy(P->rows, rows, 96 * (size_t)pp->R);
    P->m = (fe*)malloc(N * sizeof(fe));
    if (load_m(P->m, m, N)) { free(P->rows); free(P->m); free(P); return NULL; }
    P->m_raw = (u64*)malloc(N * 32); memcpy(P->m_raw, m, N * 32);
    P->blocks = (u8*)calloc(P->K, or_bopen_len(pp));
    P->blk_done = (u8*)calloc(P->K, 1);
    return P;
}
void or_prover_free(or_prover* P) {
    if (!P) return;
    free(P->rows); free(P->m); free(P->m_raw); free(P->blocks); free(P->blk_done);
    free(P->row_tree); free(P->top_tree); free(P->rj); free(P->gt); free(P->D); free(P->pst);
    free(P);
}
/* Step 1 for one block (independent of every other block; callers may run blocks on threads) */
int or_prover_block(or_prover* P, u32 k) {
    if (k >= P->K) return -1;
    int rc = or_bopen(P->pp, P->C, P->rows, P->b, k, P->blocks + or_bopen_len(P->pp) * k, 0);
    if (rc == 0) P->blk_done[k] = 1;
    return rc;
}
const u8* or_prover_block_bytes(const or_prover* P, u32 k) { return P->blocks + or_bopen_len(P->pp) * k; }

int or_prover_step2(or_prover* P) {
    const or_pp* pp = P->pp; const u32 R = pp->R, M = pp->M;
    if (R < 2 || M < 2) return -1;
    /* Merkle tree (Fiat-Shamir of [ZXH+22] as used in Sec. 4.2) */
    P->row_tree = (u8*)malloc((size_t)R * (2 * M - 1) * 32);
    for (u32 j = 0; j < R; j++) {
        u8* t = P->row_tree + (size_t)j * (2 * M - 1) * 32;
        for (u32 a = 0; a < M; a++) {
            u8 mi[32]; fr_to_bytes(mi, &P->m[(size_t)j * M + a]);
            leaf_hash(t + 32 * a, (u64)j * M + a, mi);
        }
        build_tree(t, M);
    }
    P->top_tree = (u8*)malloc((2 * (size_t)R - 1) * 32);
    for (u32 j = 0; j < R; j++) {
        const u8* s = P->row_tree + ((size_t)j * (2 * M - 1) + 2 * M - 2) * 32;
        row_hash(P->top_tree + 32 * j, s, P->rows + 96 * (size_t)j);
    }
    build_tree(P->top_tree, R);
    const u8* root = P->top_tree + 32 * (2 * (size_t)R - 2);
    /* r_j, g_j = r_j f_j, D_j = C_j^{r_j} (Eq. ProverRand) */
    P->rj = (fe*)malloc(R * sizeof(fe));
    P->gt = (fe*)malloc((2 * (size_t)R - 1) * M * sizeof(fe));
    P->D = (g1*)malloc((2 * (size_t)R - 1) * sizeof(g1));
    for (u32 j = 0; j < R; j++) {
        u8 buf[36]; memcpy(buf, root, 32); be32(buf + 32, j);
        hfr(&P->rj[j], "FP-rho", buf, 36);
        for (u32 a = 0; a < M; a++) f_mul(&FR, &P->gt[(size_t)j * M + a], &P->rj[j], &P->m[(size_t)j * M + a]);
        g1 Cj; g1_from_bytes(&Cj, P->rows + 96 * (size_t)j);
        g1_mul(&P->D[j], &Cj, &P->rj[j]);
    }
    /* fold tree (Sub-protocol): g_w = g_wl + g_wr, D_w = D_wl D_wr; every node kept */
    for (int h = 1; h <= pp->log_r; h++)
        for (u32 s = 0; s < (R >> h); s++) {
            size_t w = lvl_off(R, h) + s, wl = lvl_off(R, h - 1) + 2 * s, wr = wl + 1;
            for (u32 a = 0; a < M; a++) f_add(&FR, &P->gt[w * M + a], &P->gt[wl * M + a], &P->gt[wr * M + a]);
            g1_add(&P->D[w], &P->D[wl], &P->D[wr]);
        }
    /* HyperEval on g* (PST, all hypercube points): at level t the quotient for the prefix p
     * (top bits a_{l_c-1..t+1}) is Q[c] = g*[(2p+1)2^t + c] - g*[(2p)2^t + c], committed
     * against Lambda_t. */
    const fe* gs = P->gt + (2 * (size_t)R - 2) * M;
    P->pst = (g1*)malloc(M * sizeof(g1));
    for (int t = 0; t < pp->log_c; t++) {
        u32 np = M >> (t + 1), w = 1u << t;
        for (u32 p = 0; p < np; p++) {
            g1 acc; g1_set_inf(&acc);
            for (u32 c = 0; c < w; c++) {
                fe q; f_sub(&FR, &q, &gs[(2 * (size_t)p + 1) * w + c], &gs[(2 * (size_t)p) * w + c]);
                g1 tt; g1_mul(&tt, &LAM(pp, t)[c], &q); g1_add(&acc, &acc, &tt);
            }
            P->pst[pst_index(M, t, p)] = acc;
        }
    }
    P->step2_done = 1;
    return 0;
}

size_t or_proof_len(const or_pp* pp, u32 b, u32 k) {
    u32 lo = k * b, hi = (k + 1) * b < pp->R ? (k + 1) * b : pp->R;
    return 96 * (size_t)(hi - lo) + or_bopen_len(pp) + 32 * (size_t)pp->log_n + 128 * (size_t)pp->log_r + 96 * (size_t)pp->log_c;
}

/* pi_i = block (C_a)_{a in S_k} || pi_{C_k} || Merkle path (l_c row-tree digests, then l_R
 * top-tree digests, leaf-up) || l_R sibling pairs (D_w, g_w[a]) leaf-up || PST proof
 * (pi_{l_c-1}, ..., pi_0). */
int or_prover_proof(const or_prover* P, u64 i, u8* out, size_t cap, size_t* len) {
    const or_pp* pp = P->pp; const u32 R = pp->R, M = pp->M;
    if (i >= (u64)R * M || !P->step2_done) return -1;
    u32 j = (u32)(i / M), a = (u32)(i % M), k = j / P->b;
    if (!P->blk_done[k]) return -2;
    size_t L = or_proof_len(pp, P->b, k);
    *len = L;
    if (cap < L) return -3;
    u8* o = out;
    u32 lo = k * P->b, hi = (k + 1) * P->b < R ? (k + 1) * P->b : R;
    memcpy(o, P->rows + 96 * (size_t)lo, 96 * (size_t)(hi - lo)); o += 96 * (size_t)(hi - lo);
    memcpy(o, or_prover_block_bytes(P, k), or_bopen_len(pp)); o += or_bopen_len(pp);
    const u8* rt = P->row_tree + (size_t)j * (2 * M - 1) * 32;
    for (int l = 0; l < pp->log_c; l++) { memcpy(o, rt + 32 * (lvl_off(M, l) + ((a >> l) ^ 1)), 32); o += 32; }
    for (int l = 0; l < pp->log_r; l++) { memcpy(o, P->top_tree + 32 * (lvl_off(R, l) + ((j >> l) ^ 1)), 32); o += 32; }
    for (int h = 0; h < pp->log_r; h++) {
        size_t w = lvl_off(R, h) + ((j >> h) ^ 1);
        g1_to_bytes(o, &P->D[w]); o += 96;
        fr_to_bytes(o, &P->gt[w * M + a]); o += 32;
    }
    for (int t = pp->log_c - 1; t >= 0; t--) { g1_to_bytes(o, &P->pst[pst_index(M, t, a >> (t + 1))]); o += 96; }
    return 0;
}

/* The whole shared proof state in one byte string (test access; the layout of the GPU library's
 * state export): K block records (zeros for blocks not run) || R row trees || the top tree || r_j ||
 * D_w for every fold-tree node || g_w for every node || the PST quotient commitments.  Returns the
 * size; out may be NULL to query it. */
size_t or_prover_state(const or_prover* P, u8* out) {
    const or_pp* pp = P->pp; const u32 R = pp->R, M = pp->M;
    const size_t nb = (size_t)P->K * or_bopen_len(pp), nrt = (size_t)R * (2 * M - 1) * 32, ntt = (2 * (size_t)R - 1) * 32;
    const size_t nw = 2 * (size_t)R - 1;
    const size_t total = nb + nrt + ntt + 32 * (size_t)R + 96 * nw + 32 * nw * M + 96 * ((size_t)M - 1);
    if (!out) return total;
    if (!P->step2_done) return 0;
    u8* o = out;
    memcpy(o, P->blocks, nb); o += nb;
    memcpy(o, P->row_tree, nrt); o += nrt;
    memcpy(o, P->top_tree, ntt); o += ntt;
    for (u32 j = 0; j < R; j++) { fr_to_bytes(o, &P->rj[j]); o += 32; }
    for (size_t w = 0; w < nw; w++) { g1_to_bytes(o, &P->D[w]); o += 96; }
    for (size_t q = 0; q < nw * M; q++) { fr_to_bytes(o, &P->gt[q]); o += 32; }
    for (u32 q = 0; q + 1 < M; q++) { g1_to_bytes(o, &P->pst[q]); o += 96; }
    return total;
}

/* digest of the whole shared proof state (Merkle root, r_j, fold tables, D, PST) for tests */
void or_prover_step2_parts(const or_prover* P, u8* root, u8* rj, u8* gstar, u8* dstar) {
    const u32 R = P->pp->R, M = P->pp->M;
    if (root) memcpy(root, P->top_tree + 32 * (2 * (size_t)R - 2), 32);
    if (rj) for (u32 j = 0; j < R; j++) fr_to_bytes(rj + 32 * j, &P->rj[j]);
    if (gstar) for (u32 a = 0; a < M; a++) fr_to_bytes(gstar + 32 * a, &P->gt[(2 * (size_t)R - 2) * M + a]);
    if (dstar) g1_to_bytes(dstar, &P->D[2 * (size_t)R - 2]);
}

/* ------------------------------------------------------------------------------
 * ProveOne: pi_i rebuilt from scratch with no shared state (brute force, O(N) per index):
 * BOpen on its block alone, the full Merkle tree, siblings as direct sums over their
 * subtrees, and PST.Open(g*, a) by the plain restriction chain.
 * ------------------------------------------------------------------------------ */
int or_prove_one(const or_pp* pp, const u64* m, const u8* C, const u8* rows, u32 b, u64 i, u8* out, size_t cap, size_t* len) {
    const u32 R = pp->R, M = pp->M;
    if (b < 1 || b > R || i >= (u64)R * M) return -1;
    u32 j = (u32)(i / M), a = (u32)(i % M), k = j / b;
    size_t L = or_proof_len(pp, b, k);
    *len = L;
    if (cap < L) return -3;
    size_t N = (size_t)R * M;
    fe* mm = (fe*)malloc(N * sizeof(fe));
    if (load_m(mm, m, N)) { free(mm); return -1; }
    u8* o = out;
    u32 lo = k * b, hi = (k + 1) * b < R ? (k + 1) * b : R;
    memcpy(o, rows + 96 * (size_t)lo, 96 * (size_t)(hi - lo)); o += 96 * (size_t)(hi - lo);
    int rc = or_bopen(pp, C, rows, b, k, o, 0);
    if (rc) { free(mm); return rc; }
    o += or_bopen_len(pp);
    /* whole Merkle tree */
    u8* rowt = (u8*)malloc((2 * (size_t)M - 1) * 32);
    u8* top = (u8*)malloc((2 * (size_t)R - 1) * 32);
    u8* mypath = (u8*)malloc(32 * (size_t)pp->log_c);
    for (u32 jj = 0; jj < R; jj++) {
        for (u32 aa = 0; aa < M; aa++) {
            u8 mi[32]; fr_to_bytes(mi, &mm[(size_t)jj * M + aa]);
            leaf_hash(rowt + 32 * aa, (u64)jj * M + aa, mi);
        }
        build_tree(rowt, M);
        if (jj == j)
            for (int l = 0; l < pp->log_c; l++) memcpy(mypath + 32 * l, rowt + 32 * (lvl_off(M, l) + ((a >> l) ^ 1)), 32);
        row_hash(top + 32 * jj, rowt + 32 * (2 * (size_t)M - 2), rows + 96 * (size_t)jj);
    }
    build_tree(top, R);
    memcpy(o, mypath, 32 * (size_t)pp->log_c); o += 32 * (size_t)pp->log_c;
    for (int l = 0; l < pp->log_r; l++) { memcpy(o, top + 32 * (lvl_off(R, l) + ((j >> l) ^ 1)), 32); o += 32; }
    fe* rj = (fe*)malloc(R * sizeof(fe));
    for (u32 jj = 0; jj < R; jj++) {
        u8 buf[36]; memcpy(buf, top + 32 * (2 * (size_t)R - 2), 32); be32(buf + 32, jj);
        hfr(&rj[jj], "FP-rho", buf, 36);
    }
    /* siblings as direct sums */
    for (int h = 0; h < pp->log_r; h++) {
        u32 s = (j >> h) ^ 1;
        g1 D; g1_set_inf(&D); fe y; f_zero(&y);
        for (u32 jj = s << h; jj < ((s + 1) << h); jj++) {
            g1 Cj; g1_from_bytes(&Cj, rows + 96 * (size_t)jj);
            g1 t; g1_mul(&t, &Cj, &rj[jj]); g1_add(&D, &D, &t);
            fe w; f_mul(&FR, &w, &rj[jj], &mm[(size_t)jj * M + a]); f_add(&FR, &y, &y, &w);
        }
        g1_to_bytes(o, &D); o += 96;
        fr_to_bytes(o, &y); o += 32;
    }
    /* PST.Open(g*, a) */
    fe* T = (fe*)calloc(M, sizeof(fe));
    for (u32 c = 0; c < M; c++)
        for (u32 jj = 0; jj < R; jj++) {
            fe w; f_mul(&FR, &w, &rj[jj], &mm[(size_t)jj * M + c]); f_add(&FR, &T[c], &T[c], &w);
        }
    for (int t = pp->log_c - 1; t >= 0; t--) {
        u32 w = 1u << t;
        g1 acc; g1_set_inf(&acc);
        for (u32 c = 0; c < w; c++) {
            fe q; f_sub(&FR, &q, &T[w + c], &T[c]);
            g1 tt; g1_mul(&tt, &LAM(pp, t)[c], &q); g1_add(&acc, &acc, &tt);
        }
        g1_to_bytes(o, &acc); o += 96;
        if ((a >> t) & 1) memmove(T, T + w, w * sizeof(fe));   /* T_t = a_t ? hi : lo */
    }
    free(T); free(rj); free(rowt); free(top); free(mypath); free(mm);
    return 0;
}

/* FC.BVerify checks after C_0 = (C, c1) and the weights rr of positions lo .. lo + n - 1 are known:
 * the rounds' folds of C_0, b_l from the weights (Eq. b_l), e(A_l, v_l) and b_l A_l against the
 * folded C_0, and the faster-verification check of v_l.  Returns 1 if accepted. */
static int fc_bverify_core(const or_pp* pp, const fq12* Cg, g1 c1, const fe* rr, u32 lo, u32 n, const u8* fc) {
    const int lr = pp->log_r;
    int ok = 1;
    fq12 cT = *Cg;
    u8 xprev[32]; size_t xl = 0;
    fe xinv[32];
    for (int jj = 1; jj <= lr; jj++) {
        const u8* rd = fc + 1344 * (size_t)(jj - 1);
        fq12 LT, RT; g1 L1, R1;
        if (fq12_from_bytes(&LT, rd) || g1_from_bytes(&L1, rd + 576) ||
            fq12_from_bytes(&RT, rd + 672) || g1_from_bytes(&R1, rd + 1248)) { ok = 0; break; }
        u8 tr[32 + 1344]; memcpy(tr, xprev, xl); memcpy(tr + xl, rd, 1344);
        fe x; hfr_nonzero(&x, "FP-x", tr, xl + 1344);
        fe xi; f_inv(&FR, &xi, &x); xinv[jj - 1] = xi;
        fr_to_bytes(xprev, &x); xl = 32;
        fq12 t1, t2; fq12_pow_fr(&t1, &LT, &x); fq12_pow_fr(&t2, &RT, &xi);
        fq12_mul(&cT, &cT, &t1); fq12_mul(&cT, &cT, &t2);      /* L^x o C o R^{1/x} */
        g1 s1, s2; g1_mul(&s1, &L1, &x); g1_mul(&s2, &R1, &xi);
        g1_add(&c1, &c1, &s1); g1_add(&c1, &c1, &s2);
    }
    if (ok) {
        const u8* tail = fc + 1344 * (size_t)lr;
        g1 Al; g2 vl, W;
        if (g1_from_bytes(&Al, tail) || g2_from_bytes(&vl, tail + 96) || g2_from_bytes(&W, tail + 288)) ok = 0;
        if (ok) {
            /* b_l = sum_a r_a prod_k (1/x_k)^{a_{l-k}} (Eq. b_l) */
            fe bl; f_zero(&bl);
            for (u32 t = 0; t < n; t++) {
                u32 aa = lo + t; fe w = rr[t];
                for (int kk = 1; kk <= lr; kk++) if ((aa >> (lr - kk)) & 1) f_mul(&FR, &w, &w, &xinv[kk - 1]);
                f_add(&FR, &bl, &bl, &w);
            }
            fq12 eAv; pairing(&eAv, &Al, &vl);
            g1 bA; g1_mul(&bA, &Al, &bl);
            if (!fq12_eq(&eAv, &cT) || !g1_eq(&bA, &c1)) ok = 0;
            /* v_l check: e(g1^beta - z g1, W) = e(g1, v_l - P(z) g2) */
            u8 zb[32 + 192]; memcpy(zb, xprev, 32); memcpy(zb + 32, tail + 96, 192);
            fe z; hfr(&z, "FP-z", zb, sizeof zb);
            fe Pz = FR.one, zp = z;                 /* zp runs through z^(2^e) */
            fe zpow[34]; zpow[0] = z;
            for (int e = 1; e <= lr + 1; e++) f_mul(&FR, &zpow[e], &zpow[e - 1], &zpow[e - 1]);
            for (int jj = 1; jj <= lr; jj++) {
                fe t; f_mul(&FR, &t, &xinv[jj - 1], &zpow[lr - jj + 1]);
                f_add(&FR, &t, &t, &FR.one);
                f_mul(&FR, &Pz, &Pz, &t);
            }
            (void)zp;
            g1 lhsP, zg; g1_mul(&zg, &G1_GEN, &z); g1_neg(&zg, &zg); g1_add(&lhsP, &pp->g1beta, &zg);
            g2 rhsQ, pg; g2_mul(&pg, &G2_GEN, &Pz); g2_neg(&pg, &pg); g2_add(&rhsQ, &vl, &pg);
            fq12 e1, e2; pairing(&e1, &lhsP, &W); pairing(&e2, &G1_GEN, &rhsQ);
            if (!fq12_eq(&e1, &e2)) ok = 0;
        }
    }
    return ok;
}

/* FC.BVerify of block k (Sec. 3, with the b_l shortcut of Sec. 4.3 and the faster-verification
 * check of v_l) for the block's row commitments Ca (decoded from blk) and pi_{C_k} at fc.
 * Returns 1 if accepted.  The memo key covers every input, the split included. */
static int fc_bverify(const or_pp* pp, const fq12* Cgp, const u8* C, u32 b, u32 k, const u8* blk, const g1* Ca,
                      u32 nk, const u8* fc, int use_memo) {
    const u32 R = pp->R;
    const u32 lo = k * b;
    const fq12 Cg = *Cgp;
    int ok = 1;
    u32 pid[5] = {(u32)pp->log_n, (u32)pp->seed, (u32)(pp->seed >> 32), b, (u32)pp->log_r};
    u8 hdr[576 + 4]; memcpy(hdr, C, 576); be32(hdr + 576, k);
    u8 bkey[32]; int cached = 0, cval = 0;
    if (use_memo) {
        memo_key(bkey, "bverify-t", pid, sizeof pid, hdr, sizeof hdr, blk, 96 * (size_t)nk, fc, or_bopen_len(pp));
        cached = memo_get(bkey, &cval);
        if (cached) ok = cval;
    }
    if (!cached) {
        /* r_a exactly as in BOpen: the statement needs the block's C_a in place */
        u8* rows_view = (u8*)calloc(R, 96);
        memcpy(rows_view + 96 * (size_t)lo, blk, 96 * (size_t)nk);
        fe* rr = (fe*)malloc(nk * sizeof(fe)); u32 nk2;
        block_challenges(rr, C, rows_view, R, b, k, &nk2);
        free(rows_view);
        /* C_0 = (C, y), y = prod_a C_a^{r_a} (Eq. comy) */
        g1 c1; g1_set_inf(&c1);
        for (u32 t = 0; t < nk; t++) { g1 sm; g1_mul(&sm, &Ca[t], &rr[t]); g1_add(&c1, &c1, &sm); }
        ok = fc_bverify_core(pp, &Cg, c1, rr, lo, nk, fc);
        free(rr);
        if (use_memo) memo_put(bkey, ok);
    }
    return ok;
}

/* ------------------------------------------------------------------------------
 * VC.Verify (Protocol 1 verifier steps; the combination D* = r_j C_j + sum D_w,
 * y* = r_j m_i + sum y_w of Appendix C; FC.BVerify with the b_l shortcut of Eq. b_l and the
 * faster-verification check; PST.Verify).  Returns 1 if the proof is accepted, 0 if not.
 * ------------------------------------------------------------------------------ */
int or_verify(const or_pp* pp, const u8* C, u32 b, u64 i, const u8 mi_be[32], const u8* proof, size_t len, int use_memo) {
    const u32 R = pp->R, M = pp->M; const int lr = pp->log_r, lc = pp->log_c;
    if (b < 1 || b > R || i >= (u64)R * M) return 0;
    u32 j = (u32)(i / M), a = (u32)(i % M), k = j / b;
    if (len != or_proof_len(pp, b, k)) return 0;
    fe mi; if (f_from_be(&FR, &mi, mi_be, 32)) return 0;
    u32 lo = k * b, hi = (k + 1) * b < R ? (k + 1) * b : R, nk = hi - lo;
    const u8* blk = proof;
    const u8* fc = blk + 96 * (size_t)nk;
    const u8* path = fc + or_bopen_len(pp);
    const u8* sib = path + 32 * (size_t)pp->log_n;
    const u8* pst = sib + 128 * (size_t)lr;
    fq12 Cg; if (fq12_from_bytes(&Cg, C)) return 0;
    u32 pid[5] = {(u32)pp->log_n, (u32)pp->seed, (u32)(pp->seed >> 32), b, (u32)pp->log_r};

    /* --- FC.BVerify --- */
    g1* Ca = (g1*)malloc(nk * sizeof(g1));
    for (u32 t = 0; t < nk; t++) if (g1_from_bytes(&Ca[t], blk + 96 * (size_t)t)) { free(Ca); return 0; }
    int ok = fc_bverify(pp, &Cg, C, b, k, blk, Ca, nk, fc, use_memo);
    if (!ok) { free(Ca); return 0; }
    g1 Cj = Ca[j - lo];
    free(Ca);

    /* --- Merkle path -> root -> r_j --- */
    u8 cur[32]; leaf_hash(cur, i, mi_be);
    for (int l = 0; l < lc; l++) {
        u8 nxt[32];
        if ((a >> l) & 1) node_hash(nxt, path + 32 * l, cur); else node_hash(nxt, cur, path + 32 * l);
        memcpy(cur, nxt, 32);
    }
    u8 Cjb[96]; g1_to_bytes(Cjb, &Cj);
    u8 rl[32]; row_hash(rl, cur, Cjb); memcpy(cur, rl, 32);
    for (int l = 0; l < lr; l++) {
        u8 nxt[32];
        if ((j >> l) & 1) node_hash(nxt, path + 32 * (lc + l), cur); else node_hash(nxt, cur, path + 32 * (lc + l));
        memcpy(cur, nxt, 32);
    }
    u8 buf[36]; memcpy(buf, cur, 32); be32(buf + 32, j);
    fe r; hfr(&r, "FP-rho", buf, 36);

    /* --- D*, y* (Eq. VerifierRand and the Sub-protocol's sums) --- */
    g1 Ds; g1_mul(&Ds, &Cj, &r);
    fe ys; f_mul(&FR, &ys, &r, &mi);
    for (int h = 0; h < lr; h++) {
        g1 D; fe y;
        if (g1_from_bytes(&D, sib + 128 * h) || f_from_be(&FR, &y, sib + 128 * h + 96, 32)) return 0;
        g1_add(&Ds, &Ds, &D); f_add(&FR, &ys, &ys, &y);
    }
    /* --- PST.Verify: e(D* - y* g1, g2) = prod_t e(pi_t, g2^{tau_t} - a_t g2) --- */
    u8 pkey[32], dsb[96 + 32 + 4];
    if (use_memo) {
        g1_to_bytes(dsb, &Ds); fr_to_bytes(dsb + 96, &ys); be32(dsb + 128, a);
        memo_key(pkey, "pst", pid, sizeof pid, dsb, sizeof dsb, pst, 96 * (size_t)lc, NULL, 0);
        int v; if (memo_get(pkey, &v)) return v;
    }
    g1 lhs, yg; g1_mul(&yg, &G1_GEN, &ys); g1_neg(&yg, &yg); g1_add(&lhs, &Ds, &yg);
    fq12 el; pairing(&el, &lhs, &G2_GEN);
    fq12 acc; fq12_one(&acc);
    for (int idx = 0; idx < lc; idx++) {
        int t = lc - 1 - idx;
        g1 pi; if (g1_from_bytes(&pi, pst + 96 * idx)) return 0;
        g2 q = pp->g2tau[t];
        if ((a >> t) & 1) { g2 ng; g2_neg(&ng, &G2_GEN); g2_add(&q, &q, &ng); }
        fq12 f; miller_loop(&f, &pi, &q); fq12_mul(&acc, &acc, &f);
    }
    fq12 er; final_exp(&er, &acc);
    int res = fq12_eq(&el, &er) ? 1 : 0;
    if (use_memo) memo_put(pkey, res);
    return res;
}

/* ------------------------------------------------------------------------------
 * OpenAll for sub-arrays (Sec. 4.4): the proof for segment j is its block's row commitments
 * (C_a)_{a in S_k} and pi_{C_k} (Step 1 only).  Verifier V_j recomputes C_j from its segment m_j
 * (the MLE commitment of m_j, as in VC.Commit) and checks it against the block's entry, then runs
 * FC.BVerify of the block.  m_j: M x 4 little-endian u64.  Returns 1 if accepted, 0 if not.
 * ------------------------------------------------------------------------------ */
size_t or_segment_proof_len(const or_pp* pp, u32 b, u32 k) {
    u32 lo = k * b, hi = (k + 1) * b < pp->R ? (k + 1) * b : pp->R;
    return 96 * (size_t)(hi - lo) + or_bopen_len(pp);
}
int or_verify_segment(const or_pp* pp, const u8* C, u32 b, u32 j, const u64* m_j, const u8* proof, size_t len) {
    const u32 R = pp->R, M = pp->M;
    if (b < 1 || b > R || j >= R) return 0;
    const u32 k = j / b, lo = k * b, hi = (k + 1) * b < R ? (k + 1) * b : R, nk = hi - lo;
    if (len != or_segment_proof_len(pp, b, k)) return 0;
    fe* mm = (fe*)malloc(M * sizeof(fe));
    if (load_m(mm, m_j, M)) { free(mm); return 0; }
    const g1* L = LAM(pp, pp->log_c);
    g1 Cj; g1_set_inf(&Cj);
    for (u32 a = 0; a < M; a++) { g1 t; g1_mul(&t, &L[a], &mm[a]); g1_add(&Cj, &Cj, &t); }
    free(mm);
    fq12 Cg; if (fq12_from_bytes(&Cg, C)) return 0;
    g1* Ca = (g1*)malloc(nk * sizeof(g1));
    for (u32 t = 0; t < nk; t++) if (g1_from_bytes(&Ca[t], proof + 96 * (size_t)t)) { free(Ca); return 0; }
    int ok = g1_eq(&Ca[j - lo], &Cj);
    if (ok) ok = fc_bverify(pp, &Cg, C, b, k, proof, Ca, nk, proof + 96 * (size_t)nk, 0);
    free(Ca);
    return ok;
}

/* ------------------------------------------------------------------------------
 * Evaluation proof of f_m at a point r (Sec. 4.4, "Compatibility with a family of zkSNARKs"),
 * r = (r_0 .. r_{log N - 1}) with variable k <-> bit k of i = j M + a, so the column variables
 * r_R = (r_0 .. r_{l_c - 1}) and the row variables r_L = (r_{l_c} .. r_{log N - 1}):
 *   T_j = prod_{s < l_R} (j_s r_{l_c + s} + (1 - j_s)(1 - r_{l_c + s}))   (T_{j, log mu}(r_L))
 *   F = sum_j T_j f_j (a table over the M columns), y = F(r_R) = f_m(r)  (Eq. fANDfj)
 *   step 1: C_F = prod_j C_j^{T_j};
 *   step 2: FC.BOpen(C, C, {b^(0) = T}, {y_0 = C_F}) with t = 1: r_0 = HFr("FP-r", SHA256(stmt) ||
 *           u32be(0)), stmt = "FP-eval" || C || u32be(log N) || r_0 .. r_{log N - 1} || C_F, b = r_0 T;
 *   step 3: PST.Eval(F, r_R): for t = l_c - 1 .. 0, q_t[c] = F[2^t + c] - F[c] (c < 2^t),
 *           pi_t = sum_c q_t[c] Lambda_t[c], then F[c] <- F[c] + r_t q_t[c].
 * Proof: y (32) || C_F (96) || pi_FC (or_bopen_len) || pi_{l_c-1} .. pi_0 (96 each).
 * The verifier checks FC.BVerify with C_0 = (C, C_F^{r_0}) and weights r_0 T, and
 * e(C_F - y g1, g2) = prod_t e(pi_t, g2^{tau_t} - r_t g2).
 * ------------------------------------------------------------------------------ */
size_t or_eval_proof_len(const or_pp* pp) { return 32 + 96 + or_bopen_len(pp) + 96 * (size_t)pp->log_c; }

static int load_point(fe* r, const or_pp* pp, const u8* r_be) {
    for (int k = 0; k < pp->log_n; k++)
        if (f_from_be(&FR, &r[k], r_be + 32 * (size_t)k, 32)) return -1;
    return 0;
}
static void eval_weights(fe* T, const or_pp* pp, const fe* r) {
    for (u32 j = 0; j < pp->R; j++) {
        fe acc = FR.one;
        for (int s = 0; s < pp->log_r; s++) {
            fe f = r[pp->log_c + s];
            if (!((j >> s) & 1)) f_sub(&FR, &f, &FR.one, &f);
            f_mul(&FR, &acc, &acc, &f);
        }
        T[j] = acc;
    }
}
static void eval_r0(fe* r0, const or_pp* pp, const u8* C, const u8* r_be, const u8* CF_bytes) {
    size_t sl = 7 + 576 + 4 + 32 * (size_t)pp->log_n + 96;
    u8* stmt = (u8*)malloc(sl);
    size_t o = 0;
    memcpy(stmt + o, "FP-eval", 7); o += 7;
    memcpy(stmt + o, C, 576); o += 576;
    be32(stmt + o, (u32)pp->log_n); o += 4;
    memcpy(stmt + o, r_be, 32 * (size_t)pp->log_n); o += 32 * (size_t)pp->log_n;
    memcpy(stmt + o, CF_bytes, 96);
    u8 buf[36];
    sha256(buf, stmt, sl);
    free(stmt);
    be32(buf + 32, 0);
    hfr(r0, "FP-r", buf, 36);
}

int or_eval_prove(const or_pp* pp, const u64* m, const u8* C, const u8* rows_bytes, const u8* r_be, u8* out) {
    const u32 R = pp->R, M = pp->M; const int lc = pp->log_c;
    const size_t N = (size_t)R * M;
    fe r[32];
    if (load_point(r, pp, r_be)) return -1;
    fe* mm = (fe*)malloc(N * sizeof(fe));
    if (load_m(mm, m, N)) { free(mm); return -1; }
    fe* T = (fe*)malloc(R * sizeof(fe));
    eval_weights(T, pp, r);
    fe* F = (fe*)calloc(M, sizeof(fe));
    for (u32 a = 0; a < M; a++)
        for (u32 j = 0; j < R; j++) { fe w; f_mul(&FR, &w, &T[j], &mm[(size_t)j * M + a]); f_add(&FR, &F[a], &F[a], &w); }
    g1* A = (g1*)malloc(R * sizeof(g1));
    g2* v = (g2*)malloc(R * sizeof(g2));
    g1 CF; g1_set_inf(&CF);
    for (u32 j = 0; j < R; j++) {
        if (g1_from_bytes(&A[j], rows_bytes + 96 * (size_t)j)) { free(mm); free(T); free(F); free(A); free(v); return -2; }
        v[j] = pp->g2pow[2 * j];
        g1 t; g1_mul(&t, &A[j], &T[j]); g1_add(&CF, &CF, &t);
    }
    u8* o = out + 32;
    g1_to_bytes(o, &CF); o += 96;
    fe r0; eval_r0(&r0, pp, C, r_be, out + 32);
    fe* bv = (fe*)malloc(R * sizeof(fe));
    for (u32 j = 0; j < R; j++) f_mul(&FR, &bv[j], &r0, &T[j]);
    fc_bopen_core(pp, C, A, v, bv, o, 0);
    o += or_bopen_len(pp);
    for (int t = lc - 1; t >= 0; t--) {
        const u32 w = 1u << t;
        g1 acc; g1_set_inf(&acc);
        for (u32 c = 0; c < w; c++) {
            fe q; f_sub(&FR, &q, &F[w + c], &F[c]);
            g1 tt; g1_mul(&tt, &LAM(pp, t)[c], &q); g1_add(&acc, &acc, &tt);
            fe s; f_mul(&FR, &s, &r[t], &q); f_add(&FR, &F[c], &F[c], &s);
        }
        g1_to_bytes(o, &acc); o += 96;
    }
    fr_to_bytes(out, &F[0]);
    free(mm); free(T); free(F); free(A); free(v); free(bv);
    return 0;
}

int or_eval_verify(const or_pp* pp, const u8* C, const u8* r_be, const u8* proof, size_t len) {
    const u32 R = pp->R; const int lc = pp->log_c;
    if (len != or_eval_proof_len(pp)) return 0;
    fe r[32];
    if (load_point(r, pp, r_be)) return 0;
    fe y; if (f_from_be(&FR, &y, proof, 32)) return 0;
    g1 CF; if (g1_from_bytes(&CF, proof + 32)) return 0;
    fq12 Cg; if (fq12_from_bytes(&Cg, C)) return 0;
    fe* T = (fe*)malloc(R * sizeof(fe));
    eval_weights(T, pp, r);
    fe r0; eval_r0(&r0, pp, C, r_be, proof + 32);
    for (u32 j = 0; j < R; j++) f_mul(&FR, &T[j], &T[j], &r0);
    g1 c1; g1_mul(&c1, &CF, &r0);
    int ok = fc_bverify_core(pp, &Cg, c1, T, 0, R, proof + 128);
    free(T);
    if (!ok) return 0;
    /* PST.Verify at r_R */
    const u8* pst = proof + 128 + or_bopen_len(pp);
    g1 lhsP, yg; g1_mul(&yg, &G1_GEN, &y); g1_neg(&yg, &yg); g1_add(&lhsP, &CF, &yg);
    fq12 lhs; pairing(&lhs, &lhsP, &G2_GEN);
    fq12 rhs; int first = 1;
    for (int idx = 0; idx < lc; idx++) {
        const int t = lc - 1 - idx;
        g1 pi; if (g1_from_bytes(&pi, pst + 96 * (size_t)idx)) return 0;
        g2 rg, Q; g2_mul(&rg, &G2_GEN, &r[t]); g2_neg(&rg, &rg); g2_add(&Q, &pp->g2tau[t], &rg);
        fq12 e; pairing(&e, &pi, &Q);
        if (first) { rhs = e; first = 0; } else fq12_mul(&rhs, &rhs, &e);
    }
    if (first) fq12_one(&rhs);
    return fq12_eq(&lhs, &rhs);
}
