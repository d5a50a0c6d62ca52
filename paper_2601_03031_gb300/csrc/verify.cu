// VC.Verify on the GPU (Sec. 4.2, Protocol 1 verification; FC.BVerify of Sec. 3 with the b_l
// shortcut of Sec. 4.3 and the fast verification of v_l; PST.Verify), for one proof (verify_one)
// and for all N proofs of an OpenAll output (verify_all).
//
// A proof of element i = j M + a (row j, column a, block k = j / b) consists of
//   the block part:   the block's row commitments C_a and pi_{C_k} (the same for all of block k),
//   the element part: the Merkle path of (i, m_i) and the fold-tree siblings (D_w, y_w),
//   the column part:  the PST proof of g* at a (the same for all of column a).
// Checks, in three groups:
//   block:   statement hash, x_j, z, P(z); C_0's G1 part sum_a r_a C_a and the rounds'
//            x_j L_j.1 + x_j^-1 R_j.1 (one 8-lane group per term, pairwise sums);
//            b_l = sum_a r_a prod_k x_k^-(bit l - k of a); the GT fold C L_1^x1 R_1^(1/x1) ...
//            (one 128-thread block per exponentiation); e(A_l, v_l) against the folded C,
//            e(g1^beta - z g1, W) e(-g1, v_l - P(z) g2) = 1, and b_l A_l against the folded G1 part;
//   element: the Merkle path to the root, r_j = H(root, j), D* = r_j C_j + sum_w D_w and
//            y* = r_j m_i + sum_w y_w (Eq. VerifierRand and the Sub-protocol);
//   PST:     e(D* - y* g1, g2) prod_t e(-pi_t, g2^tau_t - a_t g2) = 1 (PST.Verify at Bin(a)).
// Every serialised element is decoded with its checks (canonical coordinates, on the curve); a
// failed decode rejects the proof.  A proof is accepted iff no check of any group fails.
//
// verify_all runs each block check once per block (every proof of a block carries the same block
// part) and one PST check per column for the proofs whose PST inputs (a, D*, y*) equal those of
// the column's row-0 proof, which holds when the Merkle roots, the rows' D* and the y* agree.
// Every other proof gets a PST check of its own, so each result is the one verify_one gives for
// that proof's bytes.
#include <algorithm>

#include "group_ec.cuh"
#include "k_common.cuh"
#include "warp12.cuh"

namespace fpk {

// ------------------------------------------------------------------------------ decoding
FPG_DEV bool fq_from_be48(const uint8_t* b, fq& out) {
    fq c;
    for (int w = 0; w < 12; w++) {
        const uint8_t* q = b + (11 - w) * 4;
        c.v[w] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
    }
    if (!mp::lt<12>(c.v, FQ_P)) return false;
    out = fq_to_mont(c);
    return true;
}
FPG_DEV bool fr_from_be32(const uint8_t* b, fr& out) {
    fr c;
    for (int w = 0; w < 8; w++) {
        const uint8_t* q = b + (7 - w) * 4;
        c.v[w] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
    }
    if (!mp::lt<8>(c.v, FR_P)) return false;
    out = fr_to_mont(c);
    return true;
}
FPG_DEV bool all_zero(const uint8_t* b, int n) {
    for (int i = 0; i < n; i++)
        if (b[i]) return false;
    return true;
}
// y^2 = x^3 + 4 on G1, y^2 = x^3 + 4 (1 + u) on the twist; all-zero bytes = identity
FPG_DEV bool g1_decode(const uint8_t* b, g1a& p) {
    fq_zero(p.x);
    fq_zero(p.y);
    if (all_zero(b, 96)) return true;
    if (!fq_from_be48(b, p.x) || !fq_from_be48(b + 48, p.y)) return false;
    fq four;
    fq_one(four);
    four = fq_dbl(fq_dbl(four));
    return fq_eq(fq_sqr(p.y), fq_add(fq_mul(fq_sqr(p.x), p.x), four));
}
FPG_DEV bool g2_decode(const uint8_t* b, g2a& p) {
    fq2_zero(p.x);
    fq2_zero(p.y);
    if (all_zero(b, 192)) return true;
    if (!fq_from_be48(b, p.x.c0) || !fq_from_be48(b + 48, p.x.c1) || !fq_from_be48(b + 96, p.y.c0) ||
        !fq_from_be48(b + 144, p.y.c1))
        return false;
    fq2 bp;
    fq_one(bp.c0);
    fq_zero(bp.c1);
    bp = fq2_dbl(fq2_dbl(fq2_mul_xi(bp)));             // 4 (1 + u)
    return fq2_eq(fq2_sqr(p.y), fq2_add(fq2_mul(fq2_sqr(p.x), p.x), bp));
}
// GT element: 12 Fq in tower order
FPG_DEV bool fq12_decode(const uint8_t* b, fq12& f) {
    fq* c = reinterpret_cast<fq*>(&f);
    for (int t = 0; t < 12; t++)
        if (!fq_from_be48(b + 48 * t, c[t])) return false;
    return true;
}
FPG_DEV g1j g1j_neg(const g1j& p) { g1j r = p; r.Y = fq_neg(p.Y); return r; }
FPG_DEV bool g1a_same(const g1a& a, const g1a& b) { return fq_eq(a.x, b.x) && fq_eq(a.y, b.y); }
FPG_DEV bool jac_eq(const g1j& p, const g1j& q) { return g1a_same(g1_affine(p), g1_affine(q)); }
FPG_DEV bool fr_same(const fr& a, const fr& b) {
    for (int w = 0; w < 8; w++)
        if (a.v[w] != b.v[w]) return false;
    return true;
}
FPG_DEV bool digest_same(const uint8_t* a, const uint8_t* b) {
    for (int q = 0; q < 32; q++)
        if (a[q] != b[q]) return false;
    return true;
}
FPG_DEV g2a g2a_negate(const g2a& p) { return g2a_is_inf(p) ? p : g2a{p.x, fq2_neg(p.y)}; }
// homogeneous projective (X : Y : Z) -> Jacobian (X Z, Y Z^2, Z)
FPG_DEV g1j proj_to_jac(const GPt<fq>& r) {
    g1j o;
    o.X = fq_mul(r.X, r.Z);
    o.Y = fq_mul(r.Y, fq_sqr(r.Z));
    o.Z = r.Z;
    return o;
}
FPG_DEV g2j proj_to_jac(const GPt<fq2>& r) {
    g2j o;
    o.X = fq2_mul(r.X, r.Z);
    o.Y = fq2_mul(r.Y, fq2_sqr(r.Z));
    o.Z = r.Z;
    return o;
}
// k P on one 8-lane group (GLV, 2-bit joint windows); every lane of the group must call it
FPG_DEV g1j g1_mul8(GEc<fq>& sm, int lane, const g1a& P, const fr& k_mont) {
    uint32_t kw[8];
    fr_canon_words(kw, k_mont);
    return proj_to_jac(gec_g1_mul_proj_w2(sm, lane, P, kw));
}
// r_j = HFr("FP-rho", root || u32be(j))
FPG_DEV fr row_rho(const uint8_t* root, uint32_t j) {
    uint8_t rb[36];
    for (int q = 0; q < 32; q++) rb[q] = root[q];
    put_be32(rb + 32, j);
    return hash_to_fr("FP-rho", 6, rb, 36, nullptr, 0, nullptr, 0);
}
// one step up a Merkle path: SHA256("FP-node" || left || right), cur the right child if `right`
FPG_DEV void node_hash(uint8_t* cur, const uint8_t* sib, bool right) {
    uint8_t buf[7 + 64];
    for (int q = 0; q < 7; q++) buf[q] = (uint8_t)"FP-node"[q];
    for (int q = 0; q < 32; q++) {
        buf[7 + q] = right ? sib[q] : cur[q];
        buf[39 + q] = right ? cur[q] : sib[q];
    }
    sha256(cur, buf, 7 + 64);
}
// element leaf SHA256("FP-leaf" || u64be(i) || m_i)
FPG_DEV void leaf_hash(uint8_t* cur, uint64_t i, const uint8_t* mi_be) {
    uint8_t buf[7 + 8 + 32];
    for (int q = 0; q < 7; q++) buf[q] = (uint8_t)"FP-leaf"[q];
    put_be64(buf + 7, i);
    for (int q = 0; q < 32; q++) buf[15 + q] = mi_be[q];
    sha256(cur, buf, sizeof buf);
}
// row leaf SHA256("FP-row" || s_j || C_j), s_j = cur
FPG_DEV void row_leaf_hash(uint8_t* cur, const uint8_t* Cj_be) {
    uint8_t buf[6 + 32 + 96];
    for (int q = 0; q < 6; q++) buf[q] = (uint8_t)"FP-row"[q];
    for (int q = 0; q < 32; q++) buf[6 + q] = cur[q];
    for (int q = 0; q < 96; q++) buf[38 + q] = Cj_be[q];
    sha256(cur, buf, sizeof buf);
}

// ------------------------------------------------------------------------------ block checks
// FC.BVerify state of one block
struct VBlk {
    uint32_t bad;
    uint8_t hstmt[32];
    fr x[32], xinv[32];            // Montgomery
    fr z, Pz, bl;                  // Montgomery
    g1a Al;
    g2a vl, W;
    g1j blA, zg;
    g2j Pzg;
};

// blocks q = 0 .. nb - 1 (block k0 + q): row commitments at blk + q blk_stride, pi_{C_k} at
// fc + q fc_stride
struct VSrc {
    const uint8_t* blk;
    size_t blk_stride;
    const uint8_t* fc;
    size_t fc_stride;
    uint32_t k0, nb, b, R;
    int lr;
    __host__ __device__ uint32_t lo(uint32_t q) const { return (k0 + q) * b; }
    __host__ __device__ uint32_t nk(uint32_t q) const { return lo(q) + b < R ? b : R - lo(q); }
};

__global__ void k_v_cdec(const uint8_t* C_be, fq12* Cd, uint32_t* cbad) {
    if (gtid() != 0) return;
    *cbad = fq12_decode(C_be, *Cd) ? 0u : 1u;
}

// D_k, the tree root over the nk >= 1 row commitments at blk (96 bytes each), on one thread: the
// leaves SHA256("FP-sleaf" || C_a) go in order onto a stack of subtree roots, two subtrees of equal
// height merge as SHA256("FP-snode" || left || right) as soon as they meet, and the stack is then
// folded from the top; this is the level-by-level tree with an odd last node carried up
FPG_DEV void stmt_rows_root(const uint8_t* blk, uint32_t nk, uint8_t* out) {
    uint8_t st[33][32];
    int hgt[33];
    int sp = 0;
    auto node = [&](int l) {                           // st[l] <- H(st[l] || st[l + 1])
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, (const uint8_t*)"FP-snode", 8);
        sha256_update(c, st[l], 32);
        sha256_update(c, st[l + 1], 32);
        sha256_final(c, st[l]);
    };
    for (uint32_t t = 0; t < nk; t++) {
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, (const uint8_t*)"FP-sleaf", 8);
        sha256_update(c, blk + (size_t)t * 96, 96);
        sha256_final(c, st[sp]);
        hgt[sp++] = 0;
        while (sp >= 2 && hgt[sp - 1] == hgt[sp - 2]) {
            node(sp - 2);
            hgt[sp - 2]++;
            sp--;
        }
    }
    while (sp >= 2) {
        node(sp - 2);
        sp--;
    }
    for (int q = 0; q < 32; q++) out[q] = st[0][q];
}

// statement hash, x_j and x_j^-1, A_l, v_l, W, z and P(z) = prod_j (1 + x_j^-1 z^(2^(l - j + 1)))
__global__ void k_vb_transcript(VSrc S, const uint8_t* C_be, VBlk* st) {
    const uint64_t q = gtid();
    if (q >= S.nb) return;
    VBlk& B = st[q];
    const uint32_t k = S.k0 + (uint32_t)q, nk = S.nk((uint32_t)q);
    const uint8_t* blk = S.blk + q * S.blk_stride;
    const uint8_t* fc = S.fc + q * S.fc_stride;
    const int lr = S.lr;
    uint32_t bad = 0;
    if (S.blk) {                                       // the evaluation proof has no block statement
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, C_be, 576);
        uint8_t hdr[12];
        put_be32(hdr, k); put_be32(hdr + 4, S.b); put_be32(hdr + 8, nk);
        sha256_update(c, hdr, 12);
        uint8_t root[32];
        stmt_rows_root(blk, nk, root);
        sha256_update(c, root, 32);
        sha256_final(c, B.hstmt);
    }
    uint8_t xprev[32];
    for (int j = 1; j <= lr; j++) {
        const uint8_t* rd = fc + (size_t)(j - 1) * ROUND_BYTES;
        const fr x = hash_to_fr_nonzero("FP-x", 4, xprev, j > 1 ? 32 : 0, rd, ROUND_BYTES, nullptr, 0);
        B.x[j - 1] = x;
        B.xinv[j - 1] = fr_inv(x);
        fr_to_be(xprev, x);
    }
    const uint8_t* tail = fc + (size_t)lr * ROUND_BYTES;
    if (!g1_decode(tail, B.Al) || !g2_decode(tail + G1_SER, B.vl) || !g2_decode(tail + G1_SER + G2_SER, B.W))
        bad |= 2;
    const fr z = hash_to_fr("FP-z", 4, xprev, 32, tail + G1_SER, G2_SER, nullptr, 0);
    B.z = z;
    fr zp[34];
    zp[0] = z;
    for (int e = 1; e <= lr + 1; e++) zp[e] = fr_mul(zp[e - 1], zp[e - 1]);
    fr one, Pz;
    fr_one(one);
    Pz = one;
    for (int j = 1; j <= lr; j++) Pz = fr_mul(Pz, fr_add(one, fr_mul(B.xinv[j - 1], zp[lr - j + 1])));
    B.Pz = Pz;
    B.bad = bad;
}

// per block tpb term slots (a power of two): r_a C_a for its nk rows, then x_j L_j.1 and
// x_j^-1 R_j.1; the b_l summands r_a prod_k x_k^-(bit l - k of a) at wt[q b + t].  One 8-lane
// group per slot (16 per block); unused slots keep the identity the caller cleared them to.
__global__ void __launch_bounds__(128) k_vb_terms(VSrc S, VBlk* st, uint32_t tpb, g1j* T, fr* wt) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t t = (uint64_t)blockIdx.x * 16 + grp;
    const int lr = S.lr;
    uint32_t q = 0, u = 0, nk = 0;
    bool valid = t < (uint64_t)S.nb * tpb;
    if (valid) {
        q = (uint32_t)(t / tpb);
        u = (uint32_t)(t % tpb);
        nk = S.nk(q);
        valid = u < nk + 2 * (uint32_t)lr;
    }
    g1a P;                                             // identity and k = 0 for the idle groups
    fq_zero(P.x);
    fq_zero(P.y);
    fr k;
    fr_zero(k);
    if (valid) {
        VBlk& B = st[q];
        if (u < nk) {
            const uint32_t a = S.lo(q) + u;
            if (!g1_decode(S.blk + q * S.blk_stride + 96 * (size_t)u, P) && lane == 0) atomicOr(&B.bad, 32u);
            uint8_t buf[36];
            for (int c = 0; c < 32; c++) buf[c] = B.hstmt[c];
            put_be32(buf + 32, a);
            k = hash_to_fr("FP-r", 4, buf, 36, nullptr, 0, nullptr, 0);
            if (lane == 0) {
                fr w = k;
                for (int kk = 1; kk <= lr; kk++)
                    if ((a >> (lr - kk)) & 1) w = fr_mul(w, B.xinv[kk - 1]);
                wt[(size_t)q * S.b + u] = w;
            }
        } else {
            const int v = (int)(u - nk), jj = v >> 1, side = v & 1;
            const uint8_t* rd = S.fc + q * S.fc_stride + (size_t)jj * ROUND_BYTES;
            if (!g1_decode(rd + (side ? GT_SER + G1_SER + GT_SER : GT_SER), P) && lane == 0) atomicOr(&B.bad, 64u);
            k = side ? B.xinv[jj] : B.x[jj];
        }
    }
    const g1j r = g1_mul8(sm[grp], lane, P, k);
    if (valid && lane == 0) T[t] = r;
}

__global__ void k_vb_scalars(VSrc S, const fr* wt, VBlk* st) {
    const uint64_t q = gtid();
    if (q >= S.nb) return;
    fr s;
    fr_zero(s);
    const uint32_t nk = S.nk((uint32_t)q);
    for (uint32_t u = 0; u < nk; u++) s = fr_add(s, wt[q * S.b + u]);
    st[q].bl = s;
}

// per block: P(z) g2 on one warp (the first nb2 CTAs, four blocks each), b_l A_l and z g1 on
// 8-lane groups (16 per CTA)
union VMulSmem {
    GEcW g2[4];
    GEc<fq> g1[16];
};
__global__ void __launch_bounds__(128) k_vb_muls(VBlk* st, uint32_t nb, uint32_t nb2) {
    __shared__ VMulSmem sm;
    if (blockIdx.x < nb2) {
        const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
        const uint64_t q = (uint64_t)blockIdx.x * 4 + w;
        if (q >= nb) return;                                  // warp-uniform
        VBlk& B = st[q];
        uint32_t kw[8];
        fr_canon_words(kw, B.Pz);
        const GPt<fq2> r = gecw_g2_mul_proj(sm.g2[w], L, g2_generator(), kw);
        if (L == 0) B.Pzg = proj_to_jac(r);
        return;
    }
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t t0 = (uint64_t)(blockIdx.x - nb2) * 16 + grp;
    const bool valid = t0 < 2 * (uint64_t)nb;
    const uint64_t t = valid ? t0 : 0;
    VBlk& B = st[t >> 1];
    const bool zg = t & 1;
    const g1j r = g1_mul8(sm.g1[grp], lane, zg ? g1_generator() : B.Al, zg ? B.z : B.bl);
    if (valid && lane == 0) {
        if (zg) B.zg = r;
        else B.blA = r;
    }
}

// block q's pairs at 3q: (A_l, v_l), (g1^beta - z g1, W), (-g1, v_l - P(z) g2); and b_l A_l
// against the folded G1 part c1[q]
__global__ void k_vb_pairs(uint32_t nb, const g1a* g1beta, const g1j* c1, VBlk* st, g1a* P, g2a* Q) {
    const uint64_t q = gtid();
    if (q >= nb) return;
    VBlk& B = st[q];
    if (!jac_eq(c1[q], B.blA)) atomicOr(&B.bad, 128u);
    P[3 * q] = B.Al;
    Q[3 * q] = B.vl;
    P[3 * q + 1] = g1_affine(g1_madd(g1j_neg(B.zg), g1beta[0]));
    Q[3 * q + 1] = B.W;
    P[3 * q + 2] = g1a_neg(g1_generator());
    Q[3 * q + 2] = g2_affine(g2_madd(g2j{B.Pzg.X, fq2_neg(B.Pzg.Y), B.Pzg.Z}, B.vl));
}

// one 128-thread block per pair
__global__ void __launch_bounds__(128) k_v_miller(const g1a* P, const g2a* Q, fq12* out) {
    __shared__ WMill S;
    const int L = threadIdx.x;
    const uint64_t j = blockIdx.x;
    w_miller<4>(S, P[j], Q[j]);
    if (L < 12) reinterpret_cast<fq*>(&out[j])[2 * w_tower_pos(L >> 1) + (L & 1)] = S.f[L];
}

// L_j.T^(x_j) and R_j.T^(1/x_j) of block q at 2 lr q + 2 (j - 1) + side
__global__ void __launch_bounds__(128) k_vb_gt(VSrc S, VBlk* st, fq12* out) {
    __shared__ W12 W;
    const int L = threadIdx.x;
    const int per = 2 * S.lr;
    const uint32_t q = blockIdx.x / per;
    const int jj = (blockIdx.x % per) >> 1, side = blockIdx.x & 1;
    VBlk& B = st[q];
    const uint8_t* rd = S.fc + q * S.fc_stride + (size_t)jj * ROUND_BYTES + (side ? GT_SER + G1_SER : 0);
    if (L < 12) {
        const int pos = 2 * w_tower_pos(L >> 1) + (L & 1);
        fq v;
        if (!fq_from_be48(rd + 48 * pos, v)) {
            atomicOr(&B.bad, 1024u);
            fq_zero(v);
        }
        W.s[0][L] = v;
    }
    __syncthreads();
    uint32_t kw[8];
    fr_canon_words(kw, side ? B.xinv[jj] : B.x[jj]);
    w_exp<4>(W, W.s[1], W.s[0], kw, 256);
    if (L < 12) reinterpret_cast<fq*>(&out[blockIdx.x])[2 * w_tower_pos(L >> 1) + (L & 1)] = W.s[1][L];
}

// per block: the folded C, and the inputs of its two final exponentiations (e(A_l, v_l) and the
// fast-verification product) at fe_in[2q], fe_in[2q + 1]
__global__ void k_vb_prod(const fq12* ml, const fq12* ge, const fq12* Cd, uint32_t nb, int lr, fq12* fe_in,
                          fq12* cT) {
    const uint64_t q = gtid();
    if (q >= nb) return;
    fq12 c = *Cd;
    for (int t = 0; t < 2 * lr; t++) c = fq12_mul(c, ge[q * 2 * lr + t]);
    cT[q] = c;
    fe_in[2 * q] = ml[3 * q];
    fe_in[2 * q + 1] = fq12_mul(ml[3 * q + 1], ml[3 * q + 2]);
}

__global__ void k_vb_check(const fq12* fe_out, const fq12* cT, const uint32_t* cbad, const VBlk* st, uint32_t nb,
                           uint32_t* res) {
    const uint64_t q = gtid();
    if (q >= nb) return;
    fq12 one;
    fq12_one(one);
    uint32_t bad = st[q].bad | *cbad;
    if (!fq12_eq(fe_out[2 * q], cT[q])) bad |= 2048;
    if (!fq12_eq(fe_out[2 * q + 1], one)) bad |= 4096;
    res[q] = bad;
}

// ------------------------------------------------------------------------------ PST checks
// A PST job q checks e(E_q, g2) prod_t e(-pi_t, g2^tau_t - a_t g2) = 1 for column a_q, with
// E_q = D* - y* g1.  pi_t comes from one proof's PST part (idx = l_c - 1 - t, contiguous) or from
// the stored table of HyperEval proofs (level t at offset sum_{u<t} M / 2^(u+1), node a >> (t+1)).
struct PiSrc {
    const uint8_t* base;
    int table;
    uint32_t M;
    int lc;
    FPG_DEV const uint8_t* at(uint32_t a, int idx) const {
        if (!table) return base + 96 * (size_t)idx;
        const int t = lc - 1 - idx;
        uint64_t off = 0;
        for (int u = 0; u < t; u++) off += M >> (u + 1);
        return base + (off + (a >> (t + 1))) * G1_SER;
    }
};

// pairs of job q at (lc + 1) q: idx < lc: (-pi_idx, g2^tau_t - a_t g2); idx = lc: (E_q, g2)
__global__ void k_vp_pairs(PiSrc pi, const uint32_t* job_a, uint32_t a0, const g1a* E, uint32_t nj,
                           const g2a* g2tau, uint32_t* job_bad, g1a* P, g2a* Q) {
    const uint64_t t = gtid();
    const int lc = pi.lc;
    if (t >= (uint64_t)nj * (lc + 1)) return;
    const uint32_t q = (uint32_t)(t / (lc + 1));
    const int idx = (int)(t % (lc + 1));
    const uint32_t a = job_a ? job_a[q] : a0 + q;
    if (idx == lc) {
        P[t] = E[q];
        Q[t] = g2_generator();
        return;
    }
    const int tt = lc - 1 - idx;
    g1a p;
    if (!g1_decode(pi.at(a, idx), p)) atomicOr(&job_bad[q], 512u);
    P[t] = g1a_neg(p);
    g2a v = g2tau[tt];
    if ((a >> tt) & 1) v = g2_affine(g2_madd(g2_from_affine(v), g2a_negate(g2_generator())));
    Q[t] = v;
}

// out[q] = prod_{u < per} ml[per q + u]
__global__ void k_vp_prod(const fq12* ml, uint32_t per, uint32_t nj, fq12* out) {
    const uint64_t q = gtid();
    if (q >= nj) return;
    fq12 p = ml[q * per];
    for (uint32_t u = 1; u < per; u++) p = fq12_mul(p, ml[q * per + u]);
    out[q] = p;
}

// job q's result (decode failures | the pairing check) at res[idx ? idx[q0 + q] : q]
__global__ void k_vp_check(const fq12* fe_out, const uint32_t* job_bad, uint32_t nj, const uint32_t* idx, uint32_t q0,
                           uint32_t* res) {
    const uint64_t q = gtid();
    if (q >= nj) return;
    fq12 one;
    fq12_one(one);
    uint32_t bad = job_bad[q];
    if (!fq12_eq(fe_out[q], one)) bad |= 8192;
    res[idx ? idx[q0 + q] : q] = bad;
}

// ------------------------------------------------------------------------------ one proof
struct VElem {
    uint32_t bad;
    fr rj, ys;
    g1a Cj;
    g1j ysg, rjCj;
};

// offsets inside a proof of block size nk: block | pi_Ck | path | siblings | pst
struct VLayout {
    uint32_t nk;
    int lr, lc;
    __host__ __device__ size_t fc() const { return 96 * (size_t)nk; }
    __host__ __device__ size_t path() const { return fc() + (size_t)lr * ROUND_BYTES + G1_SER + 2 * G2_SER; }
    __host__ __device__ size_t sib() const { return path() + 32 * (size_t)(lr + lc); }
    __host__ __device__ size_t pst() const { return sib() + 128 * (size_t)lr; }
};

// Merkle path of (i, m_i) up the row tree, the row leaf with C_j, up the top tree; r_j; y*
__global__ void k_v_elem(const uint8_t* proof, const uint8_t* mi_be, VLayout Ly, uint64_t i, uint32_t M, uint32_t lo,
                         VElem* e) {
    if (gtid() != 0) return;
    uint32_t bad = 0;
    const int lr = Ly.lr, lc = Ly.lc;
    const uint32_t j = (uint32_t)(i / M), a = (uint32_t)(i % M);
    const uint8_t* Cj_be = proof + 96 * (size_t)(j - lo);
    const uint8_t* path = proof + Ly.path();
    uint8_t cur[32];
    leaf_hash(cur, i, mi_be);
    for (int l = 0; l < lc; l++) node_hash(cur, path + 32 * l, (a >> l) & 1);
    row_leaf_hash(cur, Cj_be);
    for (int l = 0; l < lr; l++) node_hash(cur, path + 32 * (lc + l), (j >> l) & 1);
    e->rj = row_rho(cur, j);
    fr mi, ys;
    if (!fr_from_be32(mi_be, mi)) bad |= 4;
    ys = fr_mul(e->rj, mi);
    const uint8_t* sib = proof + Ly.sib();
    for (int h = 0; h < lr; h++) {
        fr y;
        if (!fr_from_be32(sib + 128 * h + 96, y)) bad |= 8;
        ys = fr_add(ys, y);
    }
    e->ys = ys;
    if (!g1_decode(Cj_be, e->Cj)) bad |= 16;
    e->bad = bad;
}

// group 0: y* g1, group 1: r_j C_j (groups 2 and 3 idle)
__global__ void __launch_bounds__(32) k_v_elem_muls(VElem* e) {
    __shared__ GEc<fq> sm[4];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const bool yg = grp == 0;
    const g1j r = g1_mul8(sm[grp], lane, yg ? g1_generator() : e->Cj, yg ? e->ys : e->rj);
    if (lane == 0 && grp < 2) {
        if (yg) e->ysg = r;
        else e->rjCj = r;
    }
}

// E = D* - y* g1 with D* = r_j C_j + sum_w D_w
__global__ void k_v_elem_E(const uint8_t* proof, VLayout Ly, VElem* e, g1a* E) {
    if (gtid() != 0) return;
    g1j Ds = e->rjCj;
    const uint8_t* sib = proof + Ly.sib();
    for (int h = 0; h < Ly.lr; h++) {
        g1a D;
        if (!g1_decode(sib + 128 * h, D)) atomicOr(&e->bad, 256u);
        Ds = g1_madd(Ds, D);
    }
    E[0] = g1_affine(jac_add(Ds, g1j_neg(e->ysg)));
}

__global__ void k_v_result(const uint32_t* blk_res, const VElem* e, const uint32_t* pst_res, uint32_t* result) {
    if (gtid() != 0) return;
    result[0] = blk_res[0] | e->bad | pst_res[0];
}

namespace {

// carves a scratch buffer into 256-byte aligned pieces (SizeArena: the same walk, sizes only)
struct Arena {
    uint8_t* p;
    void* take(size_t bytes) {
        uint8_t* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    }
};
struct SizeArena {
    size_t n = 0;
    void* take(size_t bytes) {
        n += (bytes + 255) & ~(size_t)255;
        return nullptr;
    }
};

uint32_t pow2_at_least(uint64_t n) {
    uint32_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

// scratch of the checks of nb blocks of size b
template <class A>
struct BlockBufs {
    VBlk* st; g1j* T; g1j* T2; fr* wt; g1a* P; g2a* Q; fq12* ml; fq12* ge; fq12* fe_in; fq12* fe_out; fq12* cT;
    uint32_t* res;
    BlockBufs(A& ar, uint32_t nb, uint32_t b, int lr) {
        const uint64_t tpb = pow2_at_least(b + 2 * (uint64_t)lr);
        st = (VBlk*)ar.take(nb * sizeof(VBlk));
        T = (g1j*)ar.take(nb * tpb * G1J_BYTES);
        T2 = (g1j*)ar.take((nb * tpb / 2 + 1) * G1J_BYTES);
        wt = (fr*)ar.take((size_t)nb * b * FR_BYTES);
        P = (g1a*)ar.take(3 * (size_t)nb * G1A_BYTES);
        Q = (g2a*)ar.take(3 * (size_t)nb * G2A_BYTES);
        ml = (fq12*)ar.take(3 * (size_t)nb * FQ12_BYTES);
        ge = (fq12*)ar.take(2 * (size_t)lr * nb * FQ12_BYTES);
        fe_in = (fq12*)ar.take(2 * (size_t)nb * FQ12_BYTES);
        fe_out = (fq12*)ar.take(2 * (size_t)nb * FQ12_BYTES);
        cT = (fq12*)ar.take((size_t)nb * FQ12_BYTES);
        res = (uint32_t*)ar.take((size_t)nb * 4);
    }
};

// scratch of nj PST jobs with lc + 1 pairs each
template <class A>
struct JobBufs {
    g1a* E; uint32_t* a; uint32_t* bad; g1a* P; g2a* Q; fq12* ml; fq12* fe_in; fq12* fe_out;
    JobBufs(A& ar, uint32_t nj, int lc) {
        const size_t np = (size_t)nj * (lc + 1);
        E = (g1a*)ar.take((size_t)nj * G1A_BYTES);
        a = (uint32_t*)ar.take((size_t)nj * 4);
        bad = (uint32_t*)ar.take((size_t)nj * 4);
        P = (g1a*)ar.take(np * G1A_BYTES);
        Q = (g2a*)ar.take(np * G2A_BYTES);
        ml = (fq12*)ar.take(np * FQ12_BYTES);
        fe_in = (fq12*)ar.take((size_t)nj * FQ12_BYTES);
        fe_out = (fq12*)ar.take((size_t)nj * FQ12_BYTES);
    }
};

// the block checks up to their pairs (at Bb.P / Bb.Q, three per block)
template <class A>
void block_checks_front(const VSrc& S, const uint8_t* C_be, const g1a* g1beta, BlockBufs<A>& Bb, cudaStream_t s) {
    const uint32_t tpb = pow2_at_least(S.b + 2 * (uint64_t)S.lr);
    const uint64_t nt = (uint64_t)S.nb * tpb;
    cudaMemsetAsync(Bb.T, 0, nt * G1J_BYTES, s);
    FP_KERNEL("k_vb_transcript", s, k_vb_transcript<<<grid_for(S.nb, 32), 32, 0, s>>>(S, C_be, Bb.st));
    FP_KERNEL("k_vb_terms", s, k_vb_terms<<<grid_for(nt, 16), 128, 0, s>>>(S, Bb.st, tpb, Bb.T, Bb.wt));
    g1j* x = Bb.T;
    g1j* y = Bb.T2;
    for (uint64_t n = nt; n > S.nb; n /= 2) {            // per-block sums: tpb is a power of two
        g1_pair_reduce(x, y, n / 2, s);
        std::swap(x, y);
    }
    FP_KERNEL("k_vb_scalars", s, k_vb_scalars<<<grid_for(S.nb, 64), 64, 0, s>>>(S, Bb.wt, Bb.st));
    const uint32_t nb2 = (S.nb + 3) / 4;
    FP_KERNEL("k_vb_muls", s, k_vb_muls<<<nb2 + grid_for(2 * (uint64_t)S.nb, 16), 128, 0, s>>>(Bb.st, S.nb, nb2));
    FP_KERNEL("k_vb_pairs", s, k_vb_pairs<<<grid_for(S.nb, 64), 64, 0, s>>>(S.nb, g1beta, x, Bb.st, Bb.P, Bb.Q));
}

// verify_one's scratch: the block's buffers, the element state, and the pairs of the block's
// three and the PST job's lc + 1 checks (one Miller launch for all)
template <class A>
struct OneBufs {
    fq12* Cd; uint32_t* cbad; VElem* e; BlockBufs<A> Bb; g1a* P; g2a* Q; fq12* ml; fq12* fe_in; fq12* fe_out;
    g1a* E; uint32_t* job_bad; uint32_t* pst_res;
    OneBufs(A& ar, uint32_t b, int lr, int lc)
        : Cd((fq12*)ar.take(FQ12_BYTES)), cbad((uint32_t*)ar.take(4)), e((VElem*)ar.take(sizeof(VElem))),
          Bb(ar, 1, b, lr) {
        const int np = 3 + lc + 1;
        P = (g1a*)ar.take((size_t)np * G1A_BYTES);
        Q = (g2a*)ar.take((size_t)np * G2A_BYTES);
        ml = (fq12*)ar.take((size_t)np * FQ12_BYTES);
        fe_in = (fq12*)ar.take(3 * FQ12_BYTES);
        fe_out = (fq12*)ar.take(3 * FQ12_BYTES);
        E = (g1a*)ar.take(G1A_BYTES);
        job_bad = (uint32_t*)ar.take(4);
        pst_res = (uint32_t*)ar.take(4);
        Bb.P = P;
        Bb.Q = Q;
        Bb.ml = ml;
    }
};

}  // namespace

void verify_one(const void* proof, const void* C_be, const void* mi_be, uint32_t nk, int lr, int lc, uint32_t b,
                uint64_t i, uint32_t M, uint32_t k, uint32_t lo, const void* g1beta, const void* g2tau, void* scratch,
                uint32_t* result, cudaStream_t s) {
    const VLayout Ly{nk, lr, lc};
    const uint8_t* pr = (const uint8_t*)proof;
    const VSrc S{pr, 0, pr + Ly.fc(), 0, k, 1, b, lo + nk, lr};   // R = lo + nk gives nk(0) = nk
    Arena ar{(uint8_t*)scratch};
    OneBufs<Arena> O(ar, b, lr, lc);
    const int np = 3 + lc + 1;
    cudaMemsetAsync(O.job_bad, 0, 4, s);
    FP_KERNEL("k_v_cdec", s, k_v_cdec<<<1, 32, 0, s>>>((const uint8_t*)C_be, O.Cd, O.cbad));
    FP_KERNEL("k_v_elem", s, k_v_elem<<<1, 32, 0, s>>>(pr, (const uint8_t*)mi_be, Ly, i, M, lo, O.e));
    block_checks_front(S, (const uint8_t*)C_be, (const g1a*)g1beta, O.Bb, s);
    FP_KERNEL("k_v_elem_muls", s, k_v_elem_muls<<<1, 32, 0, s>>>(O.e));
    FP_KERNEL("k_v_elem_E", s, k_v_elem_E<<<1, 32, 0, s>>>(pr, Ly, O.e, O.E));
    const PiSrc pi{pr + Ly.pst(), 0, M, lc};
    FP_KERNEL("k_vp_pairs", s, k_vp_pairs<<<1, 32, 0, s>>>(pi, nullptr, (uint32_t)(i % M), O.E, 1,
                                                           (const g2a*)g2tau, O.job_bad, O.P + 3, O.Q + 3));
    FP_KERNEL("k_v_miller", s, k_v_miller<<<np, 128, 0, s>>>(O.P, O.Q, O.ml));
    FP_KERNEL("k_vb_gt", s, k_vb_gt<<<2 * lr, 128, 0, s>>>(S, O.Bb.st, O.Bb.ge));
    FP_KERNEL("k_vb_prod", s, k_vb_prod<<<1, 32, 0, s>>>(O.ml, O.Bb.ge, O.Cd, 1, lr, O.fe_in, O.Bb.cT));
    FP_KERNEL("k_vp_prod", s, k_vp_prod<<<1, 32, 0, s>>>(O.ml + 3, lc + 1, 1, O.fe_in + 2));
    final_exp_group(O.fe_in, 3, O.fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_vb_check", s, k_vb_check<<<1, 32, 0, s>>>(O.fe_out, O.Bb.cT, O.cbad, O.Bb.st, 1, O.Bb.res));
    FP_KERNEL("k_vp_check", s, k_vp_check<<<1, 32, 0, s>>>(O.fe_out + 2, O.job_bad, 1, nullptr, 0, O.pst_res));
    FP_KERNEL("k_v_result", s, k_v_result<<<1, 32, 0, s>>>(O.Bb.res, O.e, O.pst_res, result));
}

size_t verify_scratch_bytes(uint32_t b, int lr, int lc) {
    SizeArena ar;
    OneBufs<SizeArena> O(ar, b, lr, lc);
    (void)O;
    return ar.n + 256;
}

// FC.BVerify of one block on its own (the segment verifier of OpenAll for sub-arrays): result
// word 0 = 0 if the block check accepts
namespace {
template <class A>
struct BlockOnlyBufs {
    fq12* Cd; uint32_t* cbad; BlockBufs<A> Bb;
    BlockOnlyBufs(A& ar, uint32_t b, int lr)
        : Cd((fq12*)ar.take(FQ12_BYTES)), cbad((uint32_t*)ar.take(4)), Bb(ar, 1, b, lr) {}
};
}  // namespace

size_t verify_block_scratch_bytes(uint32_t b, int lr) {
    SizeArena ar;
    BlockOnlyBufs<SizeArena> O(ar, b, lr);
    (void)O;
    return ar.n + 256;
}

void verify_block(const void* blk, const void* fc, const void* C_be, uint32_t nk, int lr, uint32_t b, uint32_t k,
                  uint32_t lo, const void* g1beta, void* scratch, uint32_t* result, cudaStream_t s) {
    const VSrc S{(const uint8_t*)blk, 0, (const uint8_t*)fc, 0, k, 1, b, lo + nk, lr};
    Arena ar{(uint8_t*)scratch};
    BlockOnlyBufs<Arena> O(ar, b, lr);
    FP_KERNEL("k_v_cdec", s, k_v_cdec<<<1, 32, 0, s>>>((const uint8_t*)C_be, O.Cd, O.cbad));
    block_checks_front(S, (const uint8_t*)C_be, (const g1a*)g1beta, O.Bb, s);
    FP_KERNEL("k_v_miller", s, k_v_miller<<<3, 128, 0, s>>>(O.Bb.P, O.Bb.Q, O.Bb.ml));
    FP_KERNEL("k_vb_gt", s, k_vb_gt<<<2 * lr, 128, 0, s>>>(S, O.Bb.st, O.Bb.ge));
    FP_KERNEL("k_vb_prod", s, k_vb_prod<<<1, 32, 0, s>>>(O.Bb.ml, O.Bb.ge, O.Cd, 1, lr, O.Bb.fe_in, O.Bb.cT));
    final_exp_group(O.Bb.fe_in, 2, O.Bb.fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_vb_check", s, k_vb_check<<<1, 32, 0, s>>>(O.Bb.fe_out, O.Bb.cT, O.cbad, O.Bb.st, 1, result));
}

// ------------------------------------------------------------------------------ evaluation proof
// Verifier of the evaluation proof at r (Sec. 4.4): FC.BVerify with C_0 = (C, r_0 C_F) and the
// weights w = r_0 T (one block of all R rows, no block statement), then PST.Verify at r_R:
// e(C_F - y g1, g2) prod_t e(-pi_t, g2^{tau_t} - r_t g2) = 1.  Proof: y | C_F | pi_FC | pi_PST.

// y (canonical) and C_F (on the curve) from the proof; bad |= 1 on a failed decode
__global__ void k_ve_decode(const uint8_t* proof, fr* y, g1a* CF, uint32_t* bad) {
    if (gtid() != 0) return;
    if (!fr_from_be32(proof, *y) || !g1_decode(proof + 32, *CF)) atomicOr(bad, 1u);
}

// slot 0: r_0 C_F; slots 1 .. 2 l_R: x_j L_j.1 and x_j^-1 R_j.1 (one 8-lane group each)
__global__ void __launch_bounds__(128) k_ve_terms(VSrc S, VBlk* st, const g1a* CF, const fr* r0, uint32_t tpb,
                                                  g1j* T) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t u = (uint64_t)blockIdx.x * 16 + grp;
    const int lr = S.lr;
    const bool valid = u < 1 + 2 * (uint64_t)lr && u < tpb;
    VBlk& B = st[0];
    g1a P;
    fq_zero(P.x);
    fq_zero(P.y);
    fr k;
    fr_zero(k);
    if (valid && u == 0) {
        P = *CF;
        k = *r0;
    } else if (valid) {
        const int v = (int)(u - 1), jj = v >> 1, side = v & 1;
        const uint8_t* rd = S.fc + (size_t)jj * ROUND_BYTES;
        if (!g1_decode(rd + (side ? GT_SER + G1_SER + GT_SER : GT_SER), P) && lane == 0) atomicOr(&B.bad, 64u);
        k = side ? B.xinv[jj] : B.x[jj];
    }
    const g1j r = g1_mul8(sm[grp], lane, P, k);
    if (valid && lane == 0) T[u] = r;
}

// b_l summands w_a prod_k x_k^-(bit l - k of a), a < R
__global__ void k_ve_wt(VSrc S, const VBlk* st, const fr* w, fr* wt) {
    const uint64_t a = gtid();
    if (a >= S.R) return;
    fr v = w[a];
    for (int kk = 1; kk <= S.lr; kk++)
        if ((a >> (S.lr - kk)) & 1) v = fr_mul(v, st[0].xinv[kk - 1]);
    wt[a] = v;
}

// E = C_F - y g1 on one 8-lane group
__global__ void __launch_bounds__(32) k_ve_E(const g1a* CF, const fr* y, g1a* E) {
    __shared__ GEc<fq> sm[4];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const g1j yg = g1_mul8(sm[grp], lane, g1_generator(), *y);
    if (threadIdx.x == 0) *E = g1_affine(g1_madd(g1j_neg(yg), *CF));
}

// PST pairs at r: idx < l_c: (-pi_idx, g2^{tau_t} - r_t g2), t = l_c - 1 - idx (r_t g2 on one warp);
// idx = l_c: (E, g2)
__global__ void __launch_bounds__(32) k_ve_pst_pairs(const uint8_t* pst, const fr* r_mont, const g2a* g2tau, int lc,
                                                     const g1a* E, uint32_t* bad, g1a* P, g2a* Q) {
    __shared__ GEcW sm;
    const int idx = blockIdx.x, L = threadIdx.x;
    if (idx == lc) {
        if (L == 0) {
            P[idx] = *E;
            Q[idx] = g2_generator();
        }
        return;
    }
    const int t = lc - 1 - idx;
    uint32_t kw[8];
    fr_canon_words(kw, r_mont[t]);
    const GPt<fq2> rg = gecw_g2_mul_proj(sm, L, g2_generator(), kw);
    if (L == 0) {
        g1a p;
        if (!g1_decode(pst + 96 * (size_t)idx, p)) atomicOr(bad, 512u);
        P[idx] = g1a_neg(p);
        g2a ra;
        gec_to_affine(ra.x, ra.y, rg);
        Q[idx] = g2_affine(g2_madd(g2_from_affine(g2tau[t]), g2a_negate(ra)));
    }
}

__global__ void k_ve_result(const uint32_t* blk_res, const uint32_t* pst_res, const uint32_t* dec_bad,
                            const uint32_t* err, uint32_t* result) {
    if (gtid() != 0) return;
    result[0] = blk_res[0] | pst_res[0] | dec_bad[0] | err[0];
}

namespace {
template <class A>
struct EvalBufs {
    fq12* Cd; uint32_t* cbad; BlockBufs<A> Bb; fr* r_mont; uint32_t* err; fr* Tm; fr* Tc; fr* w; fr* r0; fr* y;
    g1a* CF; g1a* E; uint32_t* dec_bad; g1a* P; g2a* Q; fq12* ml; fq12* fe_in; fq12* fe_out; uint32_t* blk_res;
    uint32_t* pst_res;
    EvalBufs(A& ar, uint32_t R, int lr, int lc, int log_n)
        : Cd((fq12*)ar.take(FQ12_BYTES)), cbad((uint32_t*)ar.take(4)), Bb(ar, 1, R, lr) {
        r_mont = (fr*)ar.take((size_t)log_n * FR_BYTES);
        err = (uint32_t*)ar.take(4);
        Tm = (fr*)ar.take((size_t)R * FR_BYTES);
        Tc = (fr*)ar.take((size_t)R * FR_BYTES);
        w = (fr*)ar.take((size_t)R * FR_BYTES);
        r0 = (fr*)ar.take(FR_BYTES);
        y = (fr*)ar.take(FR_BYTES);
        CF = (g1a*)ar.take(G1A_BYTES);
        E = (g1a*)ar.take(G1A_BYTES);
        dec_bad = (uint32_t*)ar.take(4);
        P = (g1a*)ar.take((size_t)(lc + 1) * G1A_BYTES);
        Q = (g2a*)ar.take((size_t)(lc + 1) * G2A_BYTES);
        ml = (fq12*)ar.take((size_t)(lc + 1) * FQ12_BYTES);
        fe_in = (fq12*)ar.take(FQ12_BYTES);
        fe_out = (fq12*)ar.take(FQ12_BYTES);
        blk_res = (uint32_t*)ar.take(4);
        pst_res = (uint32_t*)ar.take(4);
    }
};
}  // namespace

size_t verify_eval_scratch_bytes(uint32_t R, int lr, int lc, int log_n) {
    SizeArena ar;
    EvalBufs<SizeArena> Eb(ar, R, lr, lc, log_n);
    (void)Eb;
    return ar.n + 256;
}

void verify_eval(const void* proof, const void* C_be, const void* r_be, int log_n, int lr, int lc, uint32_t R,
                 const void* g1beta, const void* g2tau, void* scratch, uint32_t* result, cudaStream_t s) {
    const uint8_t* pr = (const uint8_t*)proof;
    const size_t blen = (size_t)lr * ROUND_BYTES + G1_SER + 2 * G2_SER;
    const VSrc S{nullptr, 0, pr + 128, 0, 0, 1, R, R, lr};
    Arena ar{(uint8_t*)scratch};
    EvalBufs<Arena> O(ar, R, lr, lc, log_n);
    cudaMemsetAsync(O.err, 0, 4, s);
    cudaMemsetAsync(O.dec_bad, 0, 4, s);
    eval_point(r_be, log_n, O.r_mont, O.err, s);
    eval_weights(O.r_mont, lr, lc, O.Tm, O.Tc, s);
    FP_KERNEL("k_ve_decode", s, k_ve_decode<<<1, 32, 0, s>>>(pr, O.y, O.CF, O.dec_bad));
    eval_bvec(C_be, r_be, log_n, pr + 32, O.Tm, R, O.r0, O.w, s);          // r_0 and w = r_0 T
    FP_KERNEL("k_v_cdec", s, k_v_cdec<<<1, 32, 0, s>>>((const uint8_t*)C_be, O.Cd, O.cbad));
    // FC.BVerify front: transcript, the G1 part of C_0 and the rounds, b_l, the three pairs
    const uint32_t tpb = pow2_at_least(1 + 2 * (uint64_t)lr);
    cudaMemsetAsync(O.Bb.T, 0, (size_t)tpb * G1J_BYTES, s);
    FP_KERNEL("k_vb_transcript", s, k_vb_transcript<<<1, 32, 0, s>>>(S, (const uint8_t*)C_be, O.Bb.st));
    FP_KERNEL("k_ve_terms", s, k_ve_terms<<<grid_for(tpb, 16), 128, 0, s>>>(S, O.Bb.st, O.CF, O.r0, tpb, O.Bb.T));
    FP_KERNEL("k_ve_wt", s, k_ve_wt<<<grid_for(R, 64), 64, 0, s>>>(S, O.Bb.st, O.w, O.Bb.wt));
    g1j* x = O.Bb.T;
    g1j* yb = O.Bb.T2;
    for (uint64_t n = tpb; n > 1; n /= 2) {
        g1_pair_reduce(x, yb, n / 2, s);
        std::swap(x, yb);
    }
    FP_KERNEL("k_vb_scalars", s, k_vb_scalars<<<1, 64, 0, s>>>(S, O.Bb.wt, O.Bb.st));
    FP_KERNEL("k_vb_muls", s, k_vb_muls<<<2, 128, 0, s>>>(O.Bb.st, 1, 1));
    FP_KERNEL("k_vb_pairs", s, k_vb_pairs<<<1, 64, 0, s>>>(1, (const g1a*)g1beta, x, O.Bb.st, O.Bb.P, O.Bb.Q));
    FP_KERNEL("k_v_miller", s, k_v_miller<<<3, 128, 0, s>>>(O.Bb.P, O.Bb.Q, O.Bb.ml));
    FP_KERNEL("k_vb_gt", s, k_vb_gt<<<2 * lr, 128, 0, s>>>(S, O.Bb.st, O.Bb.ge));
    FP_KERNEL("k_vb_prod", s, k_vb_prod<<<1, 32, 0, s>>>(O.Bb.ml, O.Bb.ge, O.Cd, 1, lr, O.Bb.fe_in, O.Bb.cT));
    final_exp_group(O.Bb.fe_in, 2, O.Bb.fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_vb_check", s, k_vb_check<<<1, 32, 0, s>>>(O.Bb.fe_out, O.Bb.cT, O.cbad, O.Bb.st, 1, O.blk_res));
    // PST.Verify at r_R
    FP_KERNEL("k_ve_E", s, k_ve_E<<<1, 32, 0, s>>>(O.CF, O.y, O.E));
    FP_KERNEL("k_ve_pst_pairs", s, k_ve_pst_pairs<<<lc + 1, 32, 0, s>>>(pr + 128 + blen, O.r_mont, (const g2a*)g2tau,
                                                                       lc, O.E, O.dec_bad, O.P, O.Q));
    FP_KERNEL("k_v_miller", s, k_v_miller<<<lc + 1, 128, 0, s>>>(O.P, O.Q, O.ml));
    FP_KERNEL("k_vp_prod", s, k_vp_prod<<<1, 32, 0, s>>>(O.ml, lc + 1, 1, O.fe_in));
    final_exp_group(O.fe_in, 1, O.fe_out, nullptr, 1, 0, 0, s);
    cudaMemsetAsync(O.pst_res, 0, 4, s);
    FP_KERNEL("k_vp_check", s, k_vp_check<<<1, 32, 0, s>>>(O.fe_out, O.pst_res, 1, nullptr, 0, O.pst_res));
    FP_KERNEL("k_ve_result", s, k_ve_result<<<1, 32, 0, s>>>(O.blk_res, O.pst_res, O.dec_bad, O.err, result));
}

// ------------------------------------------------------------------------------ all proofs
// Merkle root of every proof (from the stored trees) and the range check of its claimed m_i
// (N x 4 little-endian u64)
__global__ void k_va_paths(ProofLayout L, const uint64_t* m, const uint8_t* row_tree, const uint8_t* top_tree,
                           const uint8_t* rows_ser, uint8_t* roots, uint8_t* mbad) {
    const uint64_t i = gtid();
    if (i >= (uint64_t)L.R * L.M) return;
    const uint32_t j = (uint32_t)(i / L.M), a = (uint32_t)(i % L.M);
    uint8_t mi_be[32];
    uint64_t limb[4];
    for (int w = 0; w < 4; w++) limb[w] = m[4 * i + w];
    for (int w = 0; w < 4; w++) put_be64(mi_be + 8 * (3 - w), limb[w]);
    fr c;
    for (int w = 0; w < 4; w++) {
        c.v[2 * w] = (uint32_t)limb[w];
        c.v[2 * w + 1] = (uint32_t)(limb[w] >> 32);
    }
    mbad[i] = mp::lt<8>(c.v, FR_P) ? 0 : 1;
    uint8_t cur[32];
    leaf_hash(cur, i, mi_be);
    const uint8_t* rt = row_tree + (size_t)j * (2 * (size_t)L.M - 1) * 32;
    for (int l = 0; l < L.log_c; l++) node_hash(cur, rt + 32 * (tree_off(L.M, l) + ((a >> l) ^ 1)), (a >> l) & 1);
    row_leaf_hash(cur, rows_ser + 96 * (size_t)j);
    for (int l = 0; l < L.log_r; l++)
        node_hash(cur, top_tree + 32 * (tree_off(L.R, l) + ((j >> l) ^ 1)), (j >> l) & 1);
    for (int q = 0; q < 32; q++) roots[32 * i + q] = cur[q];
}

// per row, with the root of proof 0: r_j and D*_j = r_j C_j + sum_w D_w (affine); one 8-lane
// group per row
__global__ void __launch_bounds__(128) k_va_rows(ProofLayout L, const uint8_t* roots, const uint8_t* rows_ser,
                                                 const uint8_t* D_ser, fr* rj, g1a* Dstar, uint32_t* row_bad) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t j0 = (uint64_t)blockIdx.x * 16 + grp;
    const bool valid = j0 < L.R;
    const uint32_t j = valid ? (uint32_t)j0 : 0;
    const fr r = row_rho(roots, j);
    g1a Cj;
    const bool cok = g1_decode(rows_ser + 96 * (size_t)j, Cj);
    g1j Ds = g1_mul8(sm[grp], lane, Cj, r);
    if (!valid || lane != 0) return;
    uint32_t bad = cok ? 0u : 16u;
    for (int h = 0; h < L.log_r; h++) {
        g1a D;
        if (!g1_decode(D_ser + G1_SER * (tree_off(L.R, h) + ((j >> h) ^ 1)), D)) bad |= 256;
        Ds = g1_madd(Ds, D);
    }
    rj[j] = r;
    Dstar[j] = g1_affine(Ds);
    row_bad[j] = bad;
}

// y* = r_j m_i + sum_w g_w[a] of every proof, r_j from the proof's own root
__global__ void k_va_y(ProofLayout L, const uint64_t* m, const uint8_t* roots, const fr* rj, const fr* g,
                       const uint8_t* mbad, fr* ys) {
    const uint64_t i = gtid();
    if (i >= (uint64_t)L.R * L.M) return;
    const uint32_t j = (uint32_t)(i / L.M), a = (uint32_t)(i % L.M);
    const fr r = digest_same(roots + 32 * i, roots) ? rj[j] : row_rho(roots + 32 * i, j);
    fr mi;
    fr_zero(mi);
    if (!mbad[i]) {
        for (int w = 0; w < 4; w++) {
            const uint64_t v = m[4 * i + w];
            mi.v[2 * w] = (uint32_t)v;
            mi.v[2 * w + 1] = (uint32_t)(v >> 32);
        }
        mi = fr_to_mont(mi);
    }
    fr y = fr_mul(r, mi);
    for (int h = 0; h < L.log_r; h++) y = fr_add(y, g[(tree_off(L.R, h) + ((j >> h) ^ 1)) * L.M + a]);
    ys[i] = y;
}

// a proof shares its column's PST check when its root and the root of the column's row-0 proof
// are proof 0's, its row's D* is row 0's, and its y* is the row-0 proof's; the others are listed
__global__ void k_va_class(ProofLayout L, const uint8_t* roots, const g1a* Dstar, const fr* ys, int each,
                           uint8_t* shared, uint32_t* irr, uint32_t* nirr) {
    const uint64_t i = gtid();
    if (i >= (uint64_t)L.R * L.M) return;
    const uint32_t j = (uint32_t)(i / L.M), a = (uint32_t)(i % L.M);
    const bool sh = !each && digest_same(roots + 32 * i, roots) && digest_same(roots + 32 * (uint64_t)a, roots) &&
                    g1a_same(Dstar[j], Dstar[0]) && fr_same(ys[i], ys[a]);
    shared[i] = sh;
    if (!sh) irr[atomicAdd(nirr, 1u)] = (uint32_t)i;
}

// column jobs: E_a = D*_0 - y*_a g1, one 8-lane group each
__global__ void __launch_bounds__(128) k_va_colE(const g1a* Dstar, const fr* ys, uint32_t M, g1a* E) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t a0 = (uint64_t)blockIdx.x * 16 + grp;
    const bool valid = a0 < M;
    const uint64_t a = valid ? a0 : 0;
    const g1j yg = g1_mul8(sm[grp], lane, g1_generator(), ys[a]);
    if (valid && lane == 0) E[a] = g1_affine(g1_madd(g1j_neg(yg), Dstar[0]));
}

// jobs of the listed proofs irr[q0 .. q0 + nj): E = r_j C_j + sum_w D_w - y* g1, r_j from the
// proof's own root; one 8-lane group each
__global__ void __launch_bounds__(128) k_va_irrE(ProofLayout L, const uint32_t* irr, uint32_t q0, uint32_t nj,
                                                 const uint8_t* roots, const fr* ys, const uint8_t* rows_ser,
                                                 const uint8_t* D_ser, g1a* E, uint32_t* job_a) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t q0g = (uint64_t)blockIdx.x * 16 + grp;
    const bool valid = q0g < nj;
    const uint64_t q = valid ? q0g : 0;
    const uint64_t i = irr[q0 + q];
    const uint32_t j = (uint32_t)(i / L.M);
    g1a Cj;
    g1_decode(rows_ser + 96 * (size_t)j, Cj);         // a bad C_j or D_w fails the row's check
    g1j Ds = g1_mul8(sm[grp], lane, Cj, row_rho(roots + 32 * i, j));
    const g1j yg = g1_mul8(sm[grp], lane, g1_generator(), ys[i]);
    if (!valid || lane != 0) return;
    for (int h = 0; h < L.log_r; h++) {
        g1a D;
        g1_decode(D_ser + G1_SER * (tree_off(L.R, h) + ((j >> h) ^ 1)), D);
        Ds = g1_madd(Ds, D);
    }
    job_a[q] = (uint32_t)(i % L.M);
    E[q] = g1_affine(jac_add(Ds, g1j_neg(yg)));
}

__global__ void k_va_result(ProofLayout L, const uint32_t* blk_res, const uint32_t* row_bad, const uint8_t* mbad,
                            const uint8_t* shared, const uint32_t* col_res, const uint32_t* irr_res, uint8_t* ok,
                            unsigned long long* n_ok) {
    const uint64_t i = gtid();
    bool good = false;
    if (i < (uint64_t)L.R * L.M) {
        const uint32_t j = (uint32_t)(i / L.M), a = (uint32_t)(i % L.M);
        const uint32_t bad = blk_res[j / L.b] | row_bad[j] | mbad[i] | (shared[i] ? col_res[a] : irr_res[i]);
        good = bad == 0;
        ok[i] = good;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, good);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(n_ok, (unsigned long long)__popc(mask));
}

namespace {

template <class A>
struct AllBufs {
    fq12* Cd; uint32_t* cbad; uint8_t* roots; uint8_t* mbad; fr* ys; uint8_t* shared; fr* rj; g1a* Dstar;
    uint32_t* row_bad; uint32_t* irr; uint32_t* nirr; uint32_t* col_res; uint32_t* irr_res; uint8_t* ok;
    unsigned long long* n_ok;
    AllBufs(A& ar, const ProofLayout& L) {
        const uint64_t N = (uint64_t)L.R * L.M;
        Cd = (fq12*)ar.take(FQ12_BYTES);
        cbad = (uint32_t*)ar.take(4);
        roots = (uint8_t*)ar.take(32 * N);
        mbad = (uint8_t*)ar.take(N);
        ys = (fr*)ar.take(N * FR_BYTES);
        shared = (uint8_t*)ar.take(N);
        rj = (fr*)ar.take((size_t)L.R * FR_BYTES);
        Dstar = (g1a*)ar.take((size_t)L.R * G1A_BYTES);
        row_bad = (uint32_t*)ar.take((size_t)L.R * 4);
        irr = (uint32_t*)ar.take(N * 4);
        nirr = (uint32_t*)ar.take(8);
        col_res = (uint32_t*)ar.take((size_t)L.M * 4);
        irr_res = (uint32_t*)ar.take(N * 4);
        ok = (uint8_t*)ar.take(N);
        n_ok = (unsigned long long*)ar.take(8);
    }
};

// PST jobs per launch chain: all M columns at once, and the other proofs in chunks of this size
uint32_t verify_all_chunk(const ProofLayout& L) { return L.M > 8192 ? L.M : 8192; }

// the PST checks of nj jobs whose E (and column, if job_a) are in J; results at
// res[idx ? idx[q0 + q] : q]
template <class A>
void pst_jobs(const ProofLayout& L, JobBufs<A>& J, uint32_t nj, const uint32_t* job_a, const uint8_t* pst_ser,
              const g2a* g2tau, const uint32_t* idx, uint32_t q0, uint32_t* res, cudaStream_t s) {
    const int lc = L.log_c;
    const uint64_t np = (uint64_t)nj * (lc + 1);
    const PiSrc pi{pst_ser, 1, L.M, lc};
    cudaMemsetAsync(J.bad, 0, (size_t)nj * 4, s);
    FP_KERNEL("k_vp_pairs", s, k_vp_pairs<<<grid_for(np, 64), 64, 0, s>>>(pi, job_a, 0, J.E, nj, g2tau, J.bad, J.P,
                                                                        J.Q));
    FP_KERNEL("k_v_miller", s, k_v_miller<<<(unsigned)np, 128, 0, s>>>(J.P, J.Q, J.ml));
    FP_KERNEL("k_vp_prod", s, k_vp_prod<<<grid_for(nj, 64), 64, 0, s>>>(J.ml, lc + 1, nj, J.fe_in));
    final_exp_group(J.fe_in, nj, J.fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_vp_check", s, k_vp_check<<<grid_for(nj, 64), 64, 0, s>>>(J.fe_out, J.bad, nj, idx, q0, res));
}

}  // namespace

size_t verify_all_scratch_bytes(const ProofLayout& L) {
    SizeArena ar;
    AllBufs<SizeArena> Ab(ar, L);
    BlockBufs<SizeArena> Bb(ar, L.K, L.b, L.log_r);
    JobBufs<SizeArena> J(ar, verify_all_chunk(L), L.log_c);
    (void)Ab; (void)Bb; (void)J;
    return ar.n + 256;
}

uint64_t verify_all(const ProofLayout& L, const void* C_be, const void* m, const void* rows_ser, const void* blocks,
                    const void* row_tree, const void* top_tree, const void* D_ser, const void* g, const void* pst_ser,
                    const void* g1beta, const void* g2tau, int each, void* scratch, void* ok_out, cudaStream_t s) {
    const uint64_t N = (uint64_t)L.R * L.M;
    Arena ar{(uint8_t*)scratch};
    AllBufs<Arena> Ab(ar, L);
    BlockBufs<Arena> Bb(ar, L.K, L.b, L.log_r);
    const uint32_t chunk = verify_all_chunk(L);
    JobBufs<Arena> J(ar, chunk, L.log_c);
    const uint8_t* Cb = (const uint8_t*)C_be;
    const uint8_t* rs = (const uint8_t*)rows_ser;
    const uint8_t* Ds = (const uint8_t*)D_ser;
    const uint8_t* ps = (const uint8_t*)pst_ser;
    cudaMemsetAsync(Ab.nirr, 0, 8, s);
    cudaMemsetAsync(Ab.n_ok, 0, 8, s);
    // the checks of all K blocks
    const VSrc S{rs, (size_t)L.b * G1_SER, (const uint8_t*)blocks, L.bopen_len, 0, L.K, L.b, L.R, L.log_r};
    FP_KERNEL("k_v_cdec", s, k_v_cdec<<<1, 32, 0, s>>>(Cb, Ab.Cd, Ab.cbad));
    block_checks_front(S, Cb, (const g1a*)g1beta, Bb, s);
    FP_KERNEL("k_v_miller", s, k_v_miller<<<3 * L.K, 128, 0, s>>>(Bb.P, Bb.Q, Bb.ml));
    FP_KERNEL("k_vb_gt", s, k_vb_gt<<<2 * L.log_r * L.K, 128, 0, s>>>(S, Bb.st, Bb.ge));
    FP_KERNEL("k_vb_prod", s, k_vb_prod<<<grid_for(L.K, 64), 64, 0, s>>>(Bb.ml, Bb.ge, Ab.Cd, L.K, L.log_r, Bb.fe_in,
                                                                       Bb.cT));
    final_exp_group(Bb.fe_in, 2 * L.K, Bb.fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_vb_check", s, k_vb_check<<<grid_for(L.K, 64), 64, 0, s>>>(Bb.fe_out, Bb.cT, Ab.cbad, Bb.st, L.K,
                                                                         Bb.res));
    // element checks and the sharing classes
    const uint64_t* md = (const uint64_t*)m;
    FP_KERNEL("k_va_paths", s, k_va_paths<<<grid_for(N, 64), 64, 0, s>>>(L, md, (const uint8_t*)row_tree,
                                                                       (const uint8_t*)top_tree, rs, Ab.roots,
                                                                       Ab.mbad));
    FP_KERNEL("k_va_rows", s, k_va_rows<<<grid_for(L.R, 16), 128, 0, s>>>(L, Ab.roots, rs, Ds, Ab.rj, Ab.Dstar,
                                                                       Ab.row_bad));
    FP_KERNEL("k_va_y", s, k_va_y<<<grid_for(N), TPB, 0, s>>>(L, md, Ab.roots, Ab.rj, (const fr*)g, Ab.mbad, Ab.ys));
    FP_KERNEL("k_va_class", s, k_va_class<<<grid_for(N), TPB, 0, s>>>(L, Ab.roots, Ab.Dstar, Ab.ys, each, Ab.shared,
                                                                      Ab.irr, Ab.nirr));
    // one PST check per column
    FP_KERNEL("k_va_colE", s, k_va_colE<<<grid_for(L.M, 16), 128, 0, s>>>(Ab.Dstar, Ab.ys, L.M, J.E));
    pst_jobs(L, J, L.M, nullptr, ps, (const g2a*)g2tau, nullptr, 0, Ab.col_res, s);
    // and one for each proof outside the shared classes
    uint32_t nirr = 0;
    cudaMemcpyAsync(&nirr, Ab.nirr, 4, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (uint32_t q0 = 0; q0 < nirr; q0 += chunk) {
        const uint32_t nj = std::min(chunk, nirr - q0);
        FP_KERNEL("k_va_irrE", s, k_va_irrE<<<grid_for(nj, 16), 128, 0, s>>>(L, Ab.irr, q0, nj, Ab.roots, Ab.ys, rs,
                                                                          Ds, J.E, J.a));
        pst_jobs(L, J, nj, J.a, ps, (const g2a*)g2tau, Ab.irr, q0, Ab.irr_res, s);
    }
    FP_KERNEL("k_va_result", s, k_va_result<<<grid_for(N), TPB, 0, s>>>(L, Bb.res, Ab.row_bad, Ab.mbad, Ab.shared,
                                                                        Ab.col_res, Ab.irr_res, Ab.ok, Ab.n_ok));
    unsigned long long n_ok = 0;
    if (ok_out) cudaMemcpyAsync(ok_out, Ab.ok, N, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&n_ok, Ab.n_ok, 8, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return n_ok;
}

}  // namespace fpk
