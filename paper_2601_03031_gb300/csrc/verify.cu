// VC.Verify of one proof on the GPU (Sec. 4.2, Protocol 1 verification; FC.BVerify of Sec. 3 with
// the b_l shortcut of Sec. 4.3 and the fast verification of v_l; PST.Verify):
//   1. transcript (one thread): statement hash of block k, x_j from L_j, R_j, z, P(z), the Merkle
//      path from (i, m_i) and C_j to the root, r_j, y* = r_j m_i + sum y_w;
//   2. C_0's G1 part sum_a r_a C_a and the rounds' x_j L_j.1 + x_j^-1 R_j.1 (one thread per term,
//      pairwise sums), b_l = sum_a r_a prod_k x_k^-(bit l - k of a);
//   3. the GT fold C L_1^x1 R_1^(1/x1) ... (one 128-thread block per exponentiation);
//   4. pairings: e(A_l, v_l) against the folded C, e(g1^beta - z g1, W) e(-g1, v_l - P(z) g2) = 1,
//      e(D* - y* g1, g2) prod_t e(-pi_t, g2^tau_t - a_t g2) = 1, and b_l A_l against the folded
//      G1 part.
// Every serialised element is decoded with its checks (canonical coordinates, on the curve);
// a failed decode rejects the proof.
#include "k_common.cuh"
#include "warp12.cuh"

namespace fpk {

struct VState {
    uint32_t bad;
    uint8_t hstmt[32];
    fr x[32], xinv[32];            // Montgomery
    fr z, Pz, rj, ys, bl;          // Montgomery
    g1a Al, Cj;
    g2a vl, W;
    fq12 C;
    g1j blA, zg, ysg, rjCj;
    g2j Pzg;
};

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
FPG_DEV bool jac_eq(const g1j& p, const g1j& q) {
    const g1a a = g1_affine(p), b = g1_affine(q);
    return fq_eq(a.x, b.x) && fq_eq(a.y, b.y);
}
FPG_DEV g2a g2a_negate(const g2a& p) { return g2a_is_inf(p) ? p : g2a{p.x, fq2_neg(p.y)}; }

// offsets inside a proof of block size nk: block | pi_Ck | path | siblings | pst
struct VLayout {
    uint32_t nk;
    int lr, lc;
    __host__ __device__ size_t fc() const { return 96 * (size_t)nk; }
    __host__ __device__ size_t path() const { return fc() + (size_t)lr * ROUND_BYTES + G1_SER + 2 * G2_SER; }
    __host__ __device__ size_t sib() const { return path() + 32 * (size_t)(lr + lc); }
    __host__ __device__ size_t pst() const { return sib() + 128 * (size_t)lr; }
};

__global__ void k_v_transcript(const uint8_t* proof, const uint8_t* C_be, const uint8_t* mi_be, VLayout Ly, uint32_t b,
                               uint64_t i, uint32_t M, uint32_t k, uint32_t lo, VState* st) {
    if (gtid() != 0) return;
    uint32_t bad = 0;
    const uint8_t* blk = proof;
    const uint8_t* fc = proof + Ly.fc();
    const int lr = Ly.lr, lc = Ly.lc;
    if (!fq12_decode(C_be, st->C)) bad |= 1;
    // statement hash and the round challenges
    {
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, C_be, 576);
        uint8_t hdr[12];
        put_be32(hdr, k); put_be32(hdr + 4, b); put_be32(hdr + 8, Ly.nk);
        sha256_update(c, hdr, 12);
        sha256_update(c, blk, 96 * Ly.nk);
        sha256_final(c, st->hstmt);
    }
    uint8_t xprev[32];
    for (int j = 1; j <= lr; j++) {
        const uint8_t* rd = fc + (size_t)(j - 1) * ROUND_BYTES;
        const fr x = hash_to_fr_nonzero("FP-x", 4, xprev, j > 1 ? 32 : 0, rd, ROUND_BYTES, nullptr, 0);
        st->x[j - 1] = x;
        st->xinv[j - 1] = fr_inv(x);
        fr_to_be(xprev, x);
    }
    const uint8_t* tail = fc + (size_t)lr * ROUND_BYTES;
    if (!g1_decode(tail, st->Al) || !g2_decode(tail + G1_SER, st->vl) || !g2_decode(tail + G1_SER + G2_SER, st->W))
        bad |= 2;
    // z and P(z) = prod_j (1 + x_j^-1 z^(2^(l - j + 1)))
    const fr z = hash_to_fr("FP-z", 4, xprev, 32, tail + G1_SER, G2_SER, nullptr, 0);
    st->z = z;
    fr zp[34];
    zp[0] = z;
    for (int e = 1; e <= lr + 1; e++) zp[e] = fr_mul(zp[e - 1], zp[e - 1]);
    fr one, Pz;
    fr_one(one);
    Pz = one;
    for (int j = 1; j <= lr; j++) Pz = fr_mul(Pz, fr_add(one, fr_mul(st->xinv[j - 1], zp[lr - j + 1])));
    st->Pz = Pz;
    // Merkle path: leaf of (i, m_i) up the row tree, the row leaf with C_j, up the top tree
    const uint32_t j = (uint32_t)(i / M), a = (uint32_t)(i % M);
    const uint8_t* path = proof + Ly.path();
    uint8_t cur[32], buf[7 + 64 + 96];
    for (int q = 0; q < 7; q++) buf[q] = (uint8_t)"FP-leaf"[q];
    put_be64(buf + 7, i);
    for (int q = 0; q < 32; q++) buf[15 + q] = mi_be[q];
    sha256(cur, buf, 7 + 8 + 32);
    for (int l = 0; l < lc + lr; l++) {
        if (l == lc) {                                     // row leaf
            for (int q = 0; q < 6; q++) buf[q] = (uint8_t)"FP-row"[q];
            for (int q = 0; q < 32; q++) buf[6 + q] = cur[q];
            for (int q = 0; q < 96; q++) buf[38 + q] = blk[96 * (size_t)(j - lo) + q];
            sha256(cur, buf, 6 + 32 + 96);
        }
        const bool right = l < lc ? ((a >> l) & 1) : ((j >> (l - lc)) & 1);
        for (int q = 0; q < 7; q++) buf[q] = (uint8_t)"FP-node"[q];
        for (int q = 0; q < 32; q++) {
            buf[7 + q] = right ? path[32 * l + q] : cur[q];
            buf[39 + q] = right ? cur[q] : path[32 * l + q];
        }
        sha256(cur, buf, 7 + 64);
    }
    uint8_t rb[36];
    for (int q = 0; q < 32; q++) rb[q] = cur[q];
    put_be32(rb + 32, j);
    st->rj = hash_to_fr("FP-rho", 6, rb, 36, nullptr, 0, nullptr, 0);
    // y* = r_j m_i + sum_w y_w
    fr mi, ys;
    if (!fr_from_be32(mi_be, mi)) bad |= 4;
    ys = fr_mul(st->rj, mi);
    const uint8_t* sib = proof + Ly.sib();
    for (int h = 0; h < lr; h++) {
        fr y;
        if (!fr_from_be32(sib + 128 * h + 96, y)) bad |= 8;
        ys = fr_add(ys, y);
    }
    st->ys = ys;
    if (!g1_decode(blk + 96 * (size_t)(j - lo), st->Cj)) bad |= 16;
    st->bad = bad;
}

// terms of C_0's G1 part and the rounds' G1 parts (Jacobian), and the b_l summands
__global__ void k_v_terms(const uint8_t* proof, VLayout Ly, uint32_t lo, VState* st, g1j* T, fr* wt) {
    const uint64_t t = gtid();
    const uint32_t nk = Ly.nk;
    const int lr = Ly.lr;
    if (t >= nk + 2 * (uint64_t)lr) return;
    g1a P;
    uint32_t kw[8];
    if (t < nk) {
        const uint32_t a = lo + (uint32_t)t;
        if (!g1_decode(proof + 96 * t, P)) atomicOr(&st->bad, 32u);
        uint8_t buf[36];
        for (int q = 0; q < 32; q++) buf[q] = st->hstmt[q];
        put_be32(buf + 32, a);
        const fr r = hash_to_fr("FP-r", 4, buf, 36, nullptr, 0, nullptr, 0);
        fr w = r;
        for (int kk = 1; kk <= lr; kk++)
            if ((a >> (lr - kk)) & 1) w = fr_mul(w, st->xinv[kk - 1]);
        wt[t] = w;
        fr_canon_words(kw, r);
    } else {
        const int u = (int)(t - nk), jj = u >> 1, side = u & 1;
        const uint8_t* rd = proof + Ly.fc() + (size_t)jj * ROUND_BYTES;
        if (!g1_decode(rd + (side ? GT_SER + G1_SER + GT_SER : GT_SER), P)) atomicOr(&st->bad, 64u);
        fr_canon_words(kw, side ? st->xinv[jj] : st->x[jj]);
    }
    T[t] = g1_mul(P, kw);
}

__global__ void k_v_scalars(const fr* wt, uint32_t nk, VState* st) {
    if (gtid() != 0) return;
    fr s;
    fr_zero(s);
    for (uint32_t t = 0; t < nk; t++) s = fr_add(s, wt[t]);
    st->bl = s;
}

// 0: b_l A_l, 1: z g1, 2: y* g1, 3: r_j C_j, 4: P(z) g2
__global__ void k_v_muls(VState* st) {
    const uint64_t t = gtid();
    if (t >= 5) return;
    uint32_t kw[8];
    switch (t) {
        case 0: fr_canon_words(kw, st->bl); st->blA = g1_mul(st->Al, kw); break;
        case 1: fr_canon_words(kw, st->z); st->zg = g1_mul(g1_generator(), kw); break;
        case 2: fr_canon_words(kw, st->ys); st->ysg = g1_mul(g1_generator(), kw); break;
        case 3: fr_canon_words(kw, st->rj); st->rjCj = g1_mul(st->Cj, kw); break;
        default: fr_canon_words(kw, st->Pz); st->Pzg = g2_mul(g2_generator(), kw); break;
    }
}

// the pairs: 0 (A_l, v_l); 1 (g1^beta - z g1, W), 2 (-g1, v_l - P(z) g2); 3 (D* - y* g1, g2),
// 4 + idx (-pi_idx, g2^tau_t - a_t g2) with t = l_c - 1 - idx; also b_l A_l == the folded G1 part
__global__ void k_v_pairs(const uint8_t* proof, VLayout Ly, uint32_t a, const g1a* g1beta, const g2a* g2tau,
                          const g1j* c1, VState* st, g1a* P, g2a* Q) {
    if (gtid() != 0) return;
    const int lr = Ly.lr, lc = Ly.lc;
    uint32_t bad = 0;
    if (!jac_eq(c1[0], st->blA)) bad |= 128;
    const g1a g1 = g1_generator();
    const g2a g2 = g2_generator();
    P[0] = st->Al;
    Q[0] = st->vl;
    P[1] = g1_affine(g1_madd(g1j_neg(st->zg), g1beta[0]));
    Q[1] = st->W;
    P[2] = g1a_neg(g1);
    Q[2] = g2_affine(g2_madd(g2j{st->Pzg.X, fq2_neg(st->Pzg.Y), st->Pzg.Z}, st->vl));
    g1j Ds = st->rjCj;
    const uint8_t* sib = proof + Ly.sib();
    for (int h = 0; h < lr; h++) {
        g1a D;
        if (!g1_decode(sib + 128 * h, D)) bad |= 256;
        Ds = g1_madd(Ds, D);
    }
    P[3] = g1_affine(jac_add(Ds, g1j_neg(st->ysg)));
    Q[3] = g2;
    const uint8_t* pst = proof + Ly.pst();
    for (int idx = 0; idx < lc; idx++) {
        const int t = lc - 1 - idx;
        g1a pi;
        if (!g1_decode(pst + 96 * idx, pi)) bad |= 512;
        P[4 + idx] = g1a_neg(pi);
        g2a q = g2tau[t];
        if ((a >> t) & 1) q = g2_affine(g2_madd(g2_from_affine(q), g2a_negate(g2)));
        Q[4 + idx] = q;
    }
    atomicOr(&st->bad, bad);
}

__global__ void __launch_bounds__(128) k_v_miller(const g1a* P, const g2a* Q, fq12* out) {
    __shared__ WMill S;
    const int L = threadIdx.x;
    const uint64_t j = blockIdx.x;
    w_miller<4>(S, P[j], Q[j]);
    if (L < 12) reinterpret_cast<fq*>(&out[j])[2 * w_tower_pos(L >> 1) + (L & 1)] = S.f[L];
}

// L_j.T^(x_j) (block 2 (j-1)) and R_j.T^(1/x_j) (block 2 (j-1) + 1)
__global__ void __launch_bounds__(128) k_v_gt(const uint8_t* proof, VLayout Ly, VState* st, fq12* out) {
    __shared__ W12 W;
    const int L = threadIdx.x;
    const int jj = blockIdx.x >> 1, side = blockIdx.x & 1;
    const uint8_t* rd = proof + Ly.fc() + (size_t)jj * ROUND_BYTES + (side ? GT_SER + G1_SER : 0);
    if (L < 12) {
        const int pos = 2 * w_tower_pos(L >> 1) + (L & 1);
        fq v;
        if (!fq_from_be48(rd + 48 * pos, v)) {
            atomicOr(&st->bad, 1024u);
            fq_zero(v);
        }
        W.s[0][L] = v;
    }
    __syncthreads();
    uint32_t kw[8];
    fr_canon_words(kw, side ? st->xinv[jj] : st->x[jj]);
    w_exp<4>(W, W.s[1], W.s[0], kw, 256);
    if (L < 12) reinterpret_cast<fq*>(&out[blockIdx.x])[2 * w_tower_pos(L >> 1) + (L & 1)] = W.s[1][L];
}

// inputs of the three final exponentiations: e(A_l, v_l), the fast-verification product, the PST
// product; and the folded C
__global__ void k_v_prod(const fq12* ml, int np, const fq12* ge, int lr, VState* st, fq12* fe_in, fq12* cT) {
    if (gtid() != 0) return;
    fq12 c = st->C;
    for (int t = 0; t < 2 * lr; t++) c = fq12_mul(c, ge[t]);
    cT[0] = c;
    fe_in[0] = ml[0];
    fe_in[1] = fq12_mul(ml[1], ml[2]);
    fq12 p = ml[3];
    for (int t = 4; t < np; t++) p = fq12_mul(p, ml[t]);
    fe_in[2] = p;
}

__global__ void k_v_check(const fq12* fe_out, const fq12* cT, VState* st, uint32_t* result) {
    if (gtid() != 0) return;
    fq12 one;
    fq12_one(one);
    uint32_t bad = st->bad;
    if (!fq12_eq(fe_out[0], cT[0])) bad |= 2048;
    if (!fq12_eq(fe_out[1], one)) bad |= 4096;
    if (!fq12_eq(fe_out[2], one)) bad |= 8192;
    result[0] = bad;
}

void verify_one(const void* proof, const void* C_be, const void* mi_be, uint32_t nk, int lr, int lc, uint32_t b,
                uint64_t i, uint32_t M, uint32_t k, uint32_t lo, const void* g1beta, const void* g2tau, void* scratch,
                uint32_t* result, cudaStream_t s) {
    const VLayout Ly{nk, lr, lc};
    const uint64_t nterms = nk + 2 * (uint64_t)lr;
    uint64_t n1 = 1;
    while (n1 < nterms) n1 <<= 1;
    const int np = 4 + lc;
    uint8_t* p = (uint8_t*)scratch;
    auto take = [&](size_t bytes) {
        uint8_t* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    VState* st = (VState*)take(sizeof(VState));
    g1j* T = (g1j*)take(n1 * G1J_BYTES);
    g1j* T2 = (g1j*)take((n1 / 2 + 1) * G1J_BYTES);
    fr* wt = (fr*)take((size_t)nk * FR_BYTES);
    g1a* P = (g1a*)take((size_t)np * G1A_BYTES);
    g2a* Q = (g2a*)take((size_t)np * G2A_BYTES);
    fq12* ml = (fq12*)take((size_t)np * FQ12_BYTES);
    fq12* ge = (fq12*)take(2 * (size_t)lr * FQ12_BYTES);
    fq12* fe_in = (fq12*)take(3 * FQ12_BYTES);
    fq12* fe_out = (fq12*)take(3 * FQ12_BYTES);
    fq12* cT = (fq12*)take(FQ12_BYTES);
    cudaMemsetAsync(T, 0, n1 * G1J_BYTES, s);
    const uint8_t* pr = (const uint8_t*)proof;
    FP_KERNEL("k_v_transcript", s, k_v_transcript<<<1, 32, 0, s>>>(pr, (const uint8_t*)C_be, (const uint8_t*)mi_be, Ly,
                                                                   b, i, M, k, lo, st));
    FP_KERNEL("k_v_terms", s, k_v_terms<<<grid_for(nterms, 64), 64, 0, s>>>(pr, Ly, lo, st, T, wt));
    g1j* a = T;
    g1j* bb = T2;
    for (uint64_t n = n1; n > 1; n /= 2) {
        g1_pair_reduce(a, bb, n / 2, s);
        std::swap(a, bb);
    }
    FP_KERNEL("k_v_scalars", s, k_v_scalars<<<1, 32, 0, s>>>(wt, nk, st));
    FP_KERNEL("k_v_muls", s, k_v_muls<<<1, 32, 0, s>>>(st));
    FP_KERNEL("k_v_pairs", s, k_v_pairs<<<1, 32, 0, s>>>(pr, Ly, (uint32_t)(i % M), (const g1a*)g1beta,
                                                         (const g2a*)g2tau, a, st, P, Q));
    FP_KERNEL("k_v_miller", s, k_v_miller<<<np, 128, 0, s>>>(P, Q, ml));
    FP_KERNEL("k_v_gt", s, k_v_gt<<<2 * lr, 128, 0, s>>>(pr, Ly, st, ge));
    FP_KERNEL("k_v_prod", s, k_v_prod<<<1, 32, 0, s>>>(ml, np, ge, lr, st, fe_in, cT));
    final_exp_group(fe_in, 3, fe_out, nullptr, 1, 0, 0, s);
    FP_KERNEL("k_v_check", s, k_v_check<<<1, 32, 0, s>>>(fe_out, cT, st, result));
}

size_t verify_scratch_bytes(uint32_t nk, int lr, int lc) {
    uint64_t n1 = 1;
    while (n1 < nk + 2 * (uint64_t)lr) n1 <<= 1;
    const int np = 4 + lc;
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return r(sizeof(VState)) + r(n1 * G1J_BYTES) + r((n1 / 2 + 1) * G1J_BYTES) + r((size_t)nk * FR_BYTES) +
           r((size_t)np * G1A_BYTES) + r((size_t)np * G2A_BYTES) + r((size_t)np * FQ12_BYTES) +
           r(2 * (size_t)lr * FQ12_BYTES) + 2 * r(3 * FQ12_BYTES) + r(FQ12_BYTES) + 256;
}

}  // namespace fpk
