// Step 1 of OpenAll: FC.BOpen (Sec. 3, Eq. b and Eq. folding) for every block S_k at once, with
// b = sum_{a in S_k} r_a u_a held densely per block, and the faster-verification proof of v_l.
// Per-block arrays are laid out block-major: X[k * R + i].
#include <algorithm>

#include "group_ec.cuh"
#include "k_common.cuh"

namespace fpk {

__global__ void k_step1_init(const g1a* rows, const g2a* g2pow, uint32_t K, uint32_t R, g1a* A, g2a* v, fr* bvec) {
    uint64_t t = gtid();
    if (t >= (uint64_t)K * R) return;
    uint32_t i = (uint32_t)(t % R);
    A[t] = rows[i];
    v[t] = g2pow[2 * i];
    fr_zero(bvec[t]);
}

// SHA256(C || u32be(k) || u32be(b) || u32be(|S_k|) || C_a for a in S_k), for the K blocks
// k = k0 .. k0 + K - 1 (stored at local index k - k0)
// SHA256 of block k's statement C || u32be(k) || u32be(b) || u32be(|S_k|) || D_k, D_k the root of the
// tree over the block's row commitments C_a (leaves SHA256("FP-sleaf" || C_a), nodes
// SHA256("FP-snode" || left || right) pairing each level left to right, an odd last node carried up).
// One block per k: warps 0..7 hash the leaves and the levels (ping-pong between two halves of the
// scratch, nk digests each), warp 8 meanwhile absorbs C and the header into the final hash's state.
constexpr int STMT_TPB = 288;
__global__ void __launch_bounds__(STMT_TPB) k_stmt_hash(const uint8_t* C_ser, const uint8_t* rows_ser, uint32_t k0,
                                                        uint32_t R, uint32_t b, uint8_t* scratch, uint8_t* hstmt) {
    __shared__ sha256_ctx pre;
    __shared__ uint8_t* root;
    const uint32_t kl = blockIdx.x, k = k0 + kl, lo = k * b, hi = min(lo + b, R), nk = hi - lo;
    const uint32_t bb = min(b, R), tid = threadIdx.x, nt = STMT_TPB - 32;
    if (tid >= nt) {                      // warp 8: C and the header, beside the tree
        if (tid == nt) {
            sha256_init(pre);
            sha256_update(pre, C_ser, 576);
            uint8_t hdr[12];
            put_be32(hdr, k); put_be32(hdr + 4, b); put_be32(hdr + 8, nk);
            sha256_update(pre, hdr, 12);
        }
    } else {                              // warps 0..7: leaves, then the levels (barrier 1 of 256)
        uint8_t* src = scratch + (size_t)kl * 2 * bb * 32;
        uint8_t* dst = src + (size_t)bb * 32;
        for (uint32_t t = tid; t < nk; t += nt) {
            sha256_ctx c;
            sha256_init(c);
            sha256_update(c, (const uint8_t*)"FP-sleaf", 8);
            sha256_update(c, rows_ser + (size_t)(lo + t) * 96, 96);
            sha256_final(c, src + (size_t)t * 32);
        }
        for (uint32_t n = nk; n > 1; n = (n + 1) / 2) {
            asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
            for (uint32_t i = tid; i < (n + 1) / 2; i += nt) {
                if (2 * i + 1 < n) {
                    sha256_ctx c;
                    sha256_init(c);
                    sha256_update(c, (const uint8_t*)"FP-snode", 8);
                    sha256_update(c, src + (size_t)(2 * i) * 32, 64);
                    sha256_final(c, dst + (size_t)i * 32);
                } else {
                    for (int q = 0; q < 32; q++) dst[(size_t)i * 32 + q] = src[(size_t)(2 * i) * 32 + q];
                }
            }
            uint8_t* t = src;
            src = dst;
            dst = t;
        }
        if (tid == 0) root = src;
    }
    __syncthreads();
    if (tid == 0) {
        sha256_update(pre, root, 32);
        sha256_final(pre, hstmt + (size_t)kl * 32);
    }
}

// r_a = HFr("FP-r", SHA256(statement_k) || u32be(a)) placed at b[a] of block k (local index k - k0)
__global__ void k_block_r(const uint8_t* hstmt, uint32_t k0, uint32_t K, uint32_t R, uint32_t b, fr* bvec) {
    uint64_t t = gtid();
    if (t >= (uint64_t)K * b) return;
    const uint32_t kl = (uint32_t)(t / b), a = (k0 + kl) * b + (uint32_t)(t % b);
    if (a >= R) return;
    uint8_t buf[36];
    for (int q = 0; q < 32; q++) buf[q] = hstmt[(size_t)kl * 32 + q];
    put_be32(buf + 32, a);
    bvec[(size_t)kl * R + a] = hash_to_fr("FP-r", 4, buf, 36, nullptr, 0, nullptr, 0);
}

// Both folds of round j in one launch: blocks [0, nb_g2) fold v, the remaining blocks fold A and b.
__global__ void __launch_bounds__(64) k_fold(g1a* A, g2a* v, fr* bvec, const fr* x_mont, const fr* xinv_mont,
                                             uint32_t K, uint32_t R, uint32_t h, uint32_t nb_g2) {
    const bool g2 = blockIdx.x < nb_g2;
    uint64_t t = (uint64_t)(g2 ? blockIdx.x : blockIdx.x - nb_g2) * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)K * h) return;
    uint64_t k = t / h;
    uint32_t i = (uint32_t)(t % h);
    uint64_t lo = k * R + i, hi = k * R + h + i;
    uint32_t kw[8];
    if (g2) {
        fr_canon_words(kw, xinv_mont[k]);
        v[lo] = g2_affine(g2_madd(g2_mul(v[hi], kw), v[lo]));
    } else {
        fr_canon_words(kw, x_mont[k]);
        A[lo] = g1_affine(g1_madd(g1_mul(A[hi], kw), A[lo]));
        bvec[lo] = fr_add(bvec[lo], fr_mul(bvec[hi], xinv_mont[k]));
    }
}

// the G1 parts of round j's record (the GT parts are written by the final exponentiation); a quad of
// four threads per point shares the inversion (jac_to_affine_quad), whole quads leave together
__global__ void __launch_bounds__(64) k_round_g1_out(const g1j* sp, uint32_t K, int j, uint8_t* blocks,
                                                     size_t bopen_len) {
    const uint64_t t = gtid() >> 2;
    if (t >= (uint64_t)K * 2) return;
    g1a a;
    jac_to_affine_quad(a.x, a.y, sp[t]);
    if ((threadIdx.x & 3) == 0) {
        uint8_t* rec = blocks + (t >> 1) * bopen_len + (size_t)(j - 1) * ROUND_BYTES + (t & 1) * (GT_SER + G1_SER);
        g1a_to_be(rec + GT_SER, a);
    }
}

// Both folds of round j for few points: blocks [0, nb2) fold 4 points of v each (one warp per point,
// group_ec.cuh GEcW), the remaining blocks 16 points of A (8-lane groups) and the entries of b.
union FoldSmemW {
    GEcW g2[4];
    GEc<fq> g1[16];
};
__global__ void __launch_bounds__(128) k_fold_w(g1a* A, g2a* v, fr* bvec, const fr* x_mont, const fr* xinv_mont,
                                                uint32_t K, uint32_t R, uint32_t h, uint32_t nb2) {
    __shared__ FoldSmemW sm;
    uint32_t kw[8];
    if (blockIdx.x < nb2) {
        const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
        const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
        if (t >= (uint64_t)K * h) return;                     // warp-uniform
        const uint64_t k = t / h;
        const uint32_t i = (uint32_t)(t % h);
        const uint64_t lo = k * R + i, hi = k * R + h + i;
        fr_canon_words(kw, xinv_mont[k]);
        const GPt<fq2> r = gecw_add(sm.g2[w], L, gecw_g2_mul_proj(sm.g2[w], L, v[hi], kw),
                                    gec_from_affine_or_inf(v[lo].x, v[lo].y));
        g2a o;
        gec_to_affine(o.x, o.y, r);
        __syncwarp();
        if (L == 0) v[lo] = o;
        return;
    }
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t t0 = (uint64_t)(blockIdx.x - nb2) * 16 + grp;
    const bool valid = t0 < (uint64_t)K * h;
    const uint64_t t = valid ? t0 : 0;
    const uint64_t k = t / h;
    const uint32_t i = (uint32_t)(t % h);
    const uint64_t lo = k * R + i, hi = k * R + h + i;
    fr_canon_words(kw, x_mont[k]);
    const GPt<fq> r = gec_add(sm.g1[grp], lane, gec_g1_mul_proj_w2(sm.g1[grp], lane, A[hi], kw),
                              gec_from_affine_or_inf(A[lo].x, A[lo].y));
    g1a o;
    gec_to_affine(o.x, o.y, r);
    __syncwarp();
    if (valid && lane == 0) {
        A[lo] = o;
        bvec[lo] = fr_add(bvec[lo], fr_mul(bvec[hi], xinv_mont[k]));
    }
}

// Comb folds for few points.  The scalar multiplications x_j A[h + i] and x_j^-1 v[h + i] are the
// longest chain of a round after the challenge, but their bases are known one round earlier.  So
// k_comb_chain, run beside the round's Miller loops and final exponentiations, forms every
// 2^i A[h + i'] (i < 128) and 2^i v[h + i'] (i < 64), k_comb_tab the 16-entry table of each G1 window
// (B = 4^w A: entries a B + b (-phi(B)), a, b < 4) and of each G2 position (B = 2^i v: entries
// sum_{j in s} (-1)^j psi^j(B)) (group_ec.cuh, fixed-base combs), and k_fold_c, after the challenge,
// only adds one table entry per window or position: 64 independent additions per point, summed
// as 16 (G1) or 8 (G2) chains and a tree instead of a chain of 64 doublings and additions.
// Point t = (k, i < h) as in k_fold_w; the tables of point t start at t 64 16.
struct CombPtrs {
    GPt<fq>* chain1;     // [n][128]
    GPt<fq2>* chain2;    // [n][64]
    GPt<fq>* tab1;       // [n 64][16]
    GPt<fq2>* tab2;      // [n 64][16]
};
static CombPtrs comb_ptrs(void* base, uint32_t n) {
    CombPtrs c;
    uint8_t* p = (uint8_t*)base;
    c.chain1 = (GPt<fq>*)p;
    p += (size_t)n * 128 * sizeof(GPt<fq>);
    c.chain2 = (GPt<fq2>*)p;
    p += (size_t)n * 64 * sizeof(GPt<fq2>);
    c.tab1 = (GPt<fq>*)p;
    p += (size_t)n * 64 * 16 * sizeof(GPt<fq>);
    c.tab2 = (GPt<fq2>*)p;
    return c;
}
size_t fold_comb_bytes(uint32_t n) {
    return (size_t)n * 128 * sizeof(GPt<fq>) + (size_t)n * 64 * sizeof(GPt<fq2>) +
           (size_t)n * 64 * 16 * sizeof(GPt<fq>) + (size_t)n * 64 * 16 * sizeof(GPt<fq2>);
}

union CombSmem {
    GEcWs g2[4];
    GEcs<fq> g1[16];
};
// blocks [0, nb2): one warp per G2 point; the others: one 8-lane group per G1 point
__global__ void __launch_bounds__(128) k_comb_chain(const g1a* A, const g2a* v, uint32_t K, uint32_t R, uint32_t h,
                                                    uint32_t nb2, GPt<fq>* chain1, GPt<fq2>* chain2) {
    __shared__ CombSmem sm;
    const uint64_t n = (uint64_t)K * h;
    if (blockIdx.x < nb2) {
        const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
        const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
        if (t >= n) return;                                   // warp-uniform
        const uint64_t hi = (t / h) * R + h + (uint32_t)(t % h);
        GPt<fq2> acc = gec_from_affine_or_inf(v[hi].x, v[hi].y);
        GPt<fq2>* out = chain2 + t * 64;
        for (int i = 0; i < 64; i++) {
            if (i) acc = gecw_dbl(sm.g2[w], L, acc);
            if (L == 0) out[i] = acc;
        }
        return;
    }
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t t0 = (uint64_t)(blockIdx.x - nb2) * 16 + grp;
    const bool valid = t0 < n;
    const uint64_t t = valid ? t0 : 0;                        // idle groups repeat point 0, store nothing
    const uint64_t hi = (t / h) * R + h + (uint32_t)(t % h);
    GPt<fq> acc = gec_from_affine_or_inf(A[hi].x, A[hi].y);
    GPt<fq>* out = chain1 + t * 128;
    for (int i = 0; i < 128; i++) {
        if (i) acc = gec_dbl(sm.g1[grp], lane, acc);
        if (valid && lane == 0) out[i] = acc;
    }
}

// one thread per table: u < n 64 the G1 window table u = t 64 + w, then the G2 position tables
// (independent tables keep every lane busy, so one lane per table issues far fewer instructions per
// entry than the lane-parallel engines, which leaves more of the GPU to the round's pairings)
__global__ void __launch_bounds__(64) k_comb_tab(uint32_t n, const GPt<fq>* chain1, const GPt<fq2>* chain2,
                                                 GPt<fq>* tab1, GPt<fq2>* tab2) {
    const uint64_t m = (uint64_t)n * 64, u = gtid();
    if (u < m) {
        const uint64_t t = u / 64, w = u % 64;
        gpt_g1_comb_table(chain1[t * 128 + 2 * w], chain1[t * 128 + 2 * w + 1], tab1 + u * 16);
    } else if (u < 2 * m) {
        gpt_g2_comb_table(chain2[u - m], tab2 + (u - m) * 16);
    }
}

// blocks [0, n): one G2 point each, 8 warps (warp g adds the entries of positions g, g + 8, ...,
// g + 56, then a tree over the warps, then v[lo]); the others two G1 points each, 16 groups per
// point (group g adds windows g, g + 16, g + 32, g + 48, then a tree over the groups, then A[lo]).
// Every group of a warp runs every addition (the groups of a warp share one instruction stream);
// additions whose result is not needed are discarded.
struct FoldSmemC {
    union {
        GEcWs g2[8];
        GEcs<fq> g1[32];
    } e;
    union {
        GPt<fq2> g2[8];
        GPt<fq> g1[2][16];
    } part;
};
__global__ void __launch_bounds__(256) k_fold_c(g1a* A, g2a* v, fr* bvec, const fr* x_mont, const fr* xinv_mont,
                                                uint32_t K, uint32_t R, uint32_t h, const GPt<fq>* tab1,
                                                const GPt<fq2>* tab2) {
    __shared__ FoldSmemC sm;
    const uint64_t n = (uint64_t)K * h;
    uint32_t kw[8];
    if (blockIdx.x < n) {
        const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
        const uint64_t t = blockIdx.x, k = t / h;
        const uint64_t lo = k * R + (uint32_t)(t % h);
        fr_canon_words(kw, xinv_mont[k]);
        uint32_t d[4][2];
        gls_digits(d, kw);
        const GPt<fq2>* tb = tab2 + t * 64 * 16;
        GPt<fq2> acc = tb[w * 16 + gls_position(d, w)];
        for (int j = 1; j < 8; j++) {
            const int i = w + 8 * j;
            acc = gecw_add(sm.e.g2[w], L, acc, tb[i * 16 + gls_position(d, i)]);
        }
        for (int sh = 4; sh >= 1; sh >>= 1) {
            __syncthreads();
            if (L == 0) sm.part.g2[w] = acc;
            __syncthreads();
            if (w < sh) acc = gecw_add(sm.e.g2[w], L, acc, sm.part.g2[w + sh]);
        }
        if (w == 0) {
            acc = gecw_add(sm.e.g2[0], L, acc, gec_from_affine_or_inf(v[lo].x, v[lo].y));
            g2a o;
            gec_to_affine_quad(o.x, o.y, acc);                 // every quad of warp 0 (converged)
            __syncwarp();
            if (L == 0) v[lo] = o;
        }
        return;
    }
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7, half = grp >> 4, g = grp & 15;
    const uint64_t t0 = (blockIdx.x - n) * 2 + half;
    const bool valid = t0 < n;
    const uint64_t t = valid ? t0 : 0;                        // an idle half repeats point 0, stores nothing
    const uint64_t k = t / h;
    const uint32_t i = (uint32_t)(t % h);
    const uint64_t lo = k * R + i, hi = k * R + h + i;
    fr_canon_words(kw, x_mont[k]);
    uint32_t k1[5], k0[4];
    div_by_const<4, 5>(k1, k0, kw, GLV_D, GLV_BARRETT);
    const GPt<fq>* tb = tab1 + t * 64 * 16;
    GPt<fq> acc = tb[g * 16 + glv_window(k0, k1, g)];
    for (int j = 1; j < 4; j++) {
        const int w = g + 16 * j;
        acc = gec_add(sm.e.g1[grp], lane, acc, tb[w * 16 + glv_window(k0, k1, w)]);
    }
    for (int sh = 8; sh >= 1; sh >>= 1) {
        __syncthreads();
        if (lane == 0) sm.part.g1[half][g] = acc;
        __syncthreads();
        const GPt<fq> r = gec_add(sm.e.g1[grp], lane, acc, sm.part.g1[half][g < sh ? g + sh : g]);
        if (g < sh) acc = r;
    }
    acc = gec_add(sm.e.g1[grp], lane, acc, gec_from_affine_or_inf(A[lo].x, A[lo].y));
    g1a o;
    gec_to_affine_quad(o.x, o.y, acc);                        // the two quads of each group
    __syncthreads();                                          // every read of A[lo] before the store
    if (valid && g == 0 && lane == 0) {
        A[lo] = o;
        bvec[lo] = fr_add(bvec[lo], fr_mul(bvec[hi], xinv_mont[k]));
    }
}

// L_j.1 and R_j.1 terms at the support of b only, one 8-lane group per term, for the blocks
// k0 .. k0 + K - 1 (local index k - k0).  Block k's vector b is
// non-zero only at its statement indices S_k = [k b, k b + |S_k|) folded mod the current length 2h:
// term t < min(|S_k|, 2h) sits at p = (k b + t) mod 2h (all p < 2h when |S_k| > 2h); p < h is an
// L_j.1 term b[p] A[h + p], p >= h an R_j.1 term b[p] A[p - h].  Results go to the dense per-block
// layout out[k 2h + p] (Jacobian), whose other entries the caller has zeroed (Z = 0: identity).
__global__ void __launch_bounds__(128) k_sparse_g(const g1a* A, const fr* bvec, uint32_t k0, uint32_t K, uint32_t R,
                                                  uint32_t h, uint32_t b, uint32_t cmax, g1j* out) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t u0 = (uint64_t)blockIdx.x * 16 + grp;
    uint64_t k = u0 / cmax;
    uint32_t t = (uint32_t)(u0 % cmax);
    bool valid = k < K;
    uint32_t sk = valid ? min(b, R - (k0 + (uint32_t)k) * b) : 1;
    valid = valid && t < min(sk, 2 * h);
    if (!valid) { k = 0; t = 0; sk = min(b, R - k0 * b); }    // dummy work keeps the warp uniform
    const uint32_t p = sk <= 2 * h ? (uint32_t)(((uint64_t)(k0 + k) * b + t) % (2 * h)) : t;
    uint32_t kw[8];
    fr_canon_words(kw, bvec[k * R + p]);
    const GPt<fq> r = gec_g1_mul_proj_w2(sm[grp], lane, A[k * R + (p < h ? h + p : p - h)], kw);
    __syncwarp();
    if (valid && lane == 0) {
        g1j o;                                                // (X : Y : Z) -> Jacobian (X Z, Y Z^2, Z)
        o.X = fq_mul(r.X, r.Z);
        o.Y = fq_mul(r.Y, fq_sqr(r.Z));
        o.Z = r.Z;
        out[k * 2 * h + p] = o;
    }
}

// the same with the two SHA-256 halves of HFr on two lanes of a warp per block (they are
// independent); lane 0 finishes (a zero challenge falls back to the serial re-hash)
__global__ void __launch_bounds__(64) k_challenge2(const uint8_t* blocks, size_t bopen_len, uint32_t K, int j,
                                                   uint8_t* xprev, fr* x_mont, fr* xinv_mont, fr* xinv_all,
                                                   int log_r) {
    __shared__ uint8_t wide[2][64];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t k = (uint64_t)blockIdx.x * 2 + w;
    if (k >= K) return;                                       // warp-uniform
    const uint8_t* rec = blocks + k * bopen_len + (size_t)(j - 1) * ROUND_BYTES;
    uint8_t* xp = xprev + k * 32;
    if (L < 2) {
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, (const uint8_t*)"FP-x", 4);
        sha256_byte(c, (uint8_t)L);
        if (j > 1) sha256_update(c, xp, 32);
        sha256_update(c, rec, ROUND_BYTES);
        sha256_final(c, wide[w] + 32 * L);
    }
    __syncwarp();
    if (L < 4) {                                              // the inverse on the quad of lanes 0 .. 3
        fr x = fr_from_be64(wide[w]);
        if (fr_is_zero(x)) x = hash_to_fr_nonzero("FP-x", 4, xp, j > 1 ? 32 : 0, rec, ROUND_BYTES, nullptr, 0);
        const fr xi = fr_inv_quad(x);
        if (L == 0) {
            x_mont[k] = x;
            xinv_mont[k] = xi;
            xinv_all[k * log_r + (j - 1)] = xi;
            fr_to_be(xp, x);
        }
    }
}

// W = sum_i q_i g2^{beta^i}: one term per (k, i < 2R), padding terms are zero
__global__ void __launch_bounds__(64) k_w_terms(const g2a* g2pow, const fr* q_canon, uint32_t K, uint32_t R, g2j* out) {
    uint64_t t = gtid();
    if (t >= (uint64_t)K * 2 * R) return;
    uint32_t i = (uint32_t)(t % (2 * R));
    fr sc = q_canon[t];
    g2j res;
    if (i >= 2 * R - 1 || fr_is_zero(sc)) jac_set_inf(res);
    else res = g2_mul(g2pow[i], sc.v);
    out[t] = res;
}

// W terms with one warp per term (few terms: latency); results as Jacobian (X Z, Y Z^2, Z)
__global__ void __launch_bounds__(128) k_w_terms_w(const g2a* g2pow, const fr* q_canon, uint32_t K, uint32_t R,
                                                   g2j* out) {
    __shared__ GEcW sm[4];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
    if (t >= (uint64_t)K * 2 * R) return;                     // warp-uniform
    const uint32_t i = (uint32_t)(t % (2 * R));
    const fr sc = q_canon[t];
    if (i >= 2 * R - 1 || fr_is_zero(sc)) {
        if (L == 0) {
            g2j z;
            jac_set_inf(z);
            out[t] = z;
        }
        return;
    }
    const GPt<fq2> r = gecw_g2_mul_proj(sm[w], L, g2pow[i], sc.v);
    __syncwarp();
    if (L == 0) {
        g2j o;
        o.X = fq2_mul(r.X, r.Z);
        o.Y = fq2_mul(r.Y, fq2_sqr(r.Z));
        o.Z = r.Z;
        out[t] = o;
    }
}

// The fast-verification proof of v_l, one block per CTA: A_l and v_l go into the block's record,
// z = HFr("FP-z", x_l || v_l), and the quotient coefficients, stored canonical and zero-padded to 2R:
//   P(X) = prod_j (1 + x_j^-1 X^(2^(l - j + 1))): the coefficient of X^m (m even) is the product of
//   x_j^-1 over the bits l - j + 1 set in m, and 0 for odd m;
//   q = (P(X) - P(z)) / (X - z): q_(i-1) = sum_{m >= i} P_m z^(m - i), by chunks of C indices: each
//   thread runs its chunk's recurrence with a zero carry, one thread chains the chunk carries
//   (carry of the chunk below = local top + z^len carry), then each chunk adds z^(hi - i) carry.
constexpr int KZG_THREADS = 128, KZG_CHUNK_MAX = 128;   // chunk length C <= KZG_CHUNK_MAX, one chunk per thread
__global__ void __launch_bounds__(KZG_THREADS) k_kzg_p(const g1a* A, const g2a* v, const uint8_t* xprev,
                                                       const fr* xinv_all, uint32_t K, uint32_t R, int log_r,
                                                       uint8_t* blocks, size_t bopen_len, fr* pcoef, fr* q_canon,
                                                       uint32_t C) {
    __shared__ fr zpow[KZG_CHUNK_MAX + 1];
    __shared__ fr carry[KZG_THREADS];
    const uint32_t k = blockIdx.x;
    const int T = threadIdx.x;
    const uint32_t deg = 2 * R - 2;
    fr* P = pcoef + (size_t)k * (deg + 1);
    fr* q = q_canon + (size_t)k * (2 * R);
    if (T == 0) {
        uint8_t* tail = blocks + k * bopen_len + (size_t)log_r * ROUND_BYTES;
        g1a_to_be(tail, A[(size_t)k * R]);
        g2a_to_be(tail + G1_SER, v[(size_t)k * R]);
        const fr z = hash_to_fr("FP-z", 4, xprev + k * 32, 32, tail + G1_SER, G2_SER, nullptr, 0);
        fr_one(zpow[0]);
        for (uint32_t c = 1; c <= C; c++) zpow[c] = fr_mul(zpow[c - 1], z);
    }
    for (uint32_t m = T; m <= deg; m += KZG_THREADS) {
        fr c;
        fr_one(c);
        if (m & 1) {
            fr_zero(c);
        } else {
            for (int j = 1; j <= log_r; j++)
                if ((m >> (log_r - j + 1)) & 1) c = fr_mul(c, xinv_all[(size_t)k * log_r + (j - 1)]);
        }
        P[m] = c;
    }
    __syncthreads();
    // indices i = 1 .. deg produce q_(i-1); chunk c covers i in [1 + c C, min(1 + (c + 1) C, deg + 1))
    const uint32_t nchunks = (deg + C - 1) / C;
    for (uint32_t c = T; c < nchunks; c += KZG_THREADS) {
        const uint32_t lo = 1 + c * C, hi = min(lo + C, deg + 1);
        fr acc;
        fr_zero(acc);
        for (uint32_t i = hi - 1; i >= lo; i--) {
            acc = fr_add(P[i], fr_mul(zpow[1], acc));        // local q_(i-1) with zero carry from above
            q[i - 1] = acc;
        }
        carry[c] = acc;                                       // local q_(lo-1)
    }
    __syncthreads();
    if (T == 0) {
        // true q_(lo_c - 1) = local_c + z^(hi_c - lo_c) q_(hi_c - 1), q_deg = 0 above the top chunk;
        // carry[c] <- the true q_(hi_c - 1) that chunk c needs
        fr above;
        fr_zero(above);
        for (int c = (int)nchunks - 1; c >= 0; c--) {
            const uint32_t lo = 1 + c * C, hi = min(lo + C, deg + 1);
            const fr local = carry[c];
            carry[c] = above;
            above = fr_add(local, fr_mul(zpow[hi - lo], above));
        }
    }
    __syncthreads();
    for (uint32_t c = T; c < nchunks; c += KZG_THREADS) {
        const uint32_t lo = 1 + c * C, hi = min(lo + C, deg + 1);
        const fr cin = carry[c];
        for (uint32_t i = lo; i < hi; i++) q[i - 1] = fr_from_mont(fr_add(q[i - 1], fr_mul(zpow[hi - i], cin)));
    }
    if (T == 0) {
        fr_zero(q[deg]);
        fr_zero(q[deg + 1]);
    }
}

void step1_init(const void* rows, const void* g2pow, uint32_t K, uint32_t R, void* A, void* v, void* bvec,
                cudaStream_t s) {
    FP_KERNEL("k_step1_init", s, k_step1_init<<<grid_for((uint64_t)K * R), TPB, 0, s>>>((const g1a*)rows, (const g2a*)g2pow, K, R, (g1a*)A,
                                                          (g2a*)v, (fr*)bvec));
}
size_t stmt_hash_scratch_bytes(uint32_t K, uint32_t R, uint32_t b) { return (size_t)K * 2 * std::min(b, R) * 32; }
void step1_stmt_hash(const void* C_ser, const void* rows_ser, uint32_t k0, uint32_t K, uint32_t R, uint32_t b,
                     void* scratch, void* hstmt, cudaStream_t s) {
    FP_KERNEL("k_stmt_hash", s, k_stmt_hash<<<K, STMT_TPB, 0, s>>>((const uint8_t*)C_ser, (const uint8_t*)rows_ser, k0,
                                                                   R, b, (uint8_t*)scratch, (uint8_t*)hstmt));
}
void step1_block_r(const void* hstmt, uint32_t k0, uint32_t K, uint32_t R, uint32_t b, void* bvec, cudaStream_t s) {
    FP_KERNEL("k_block_r", s, k_block_r<<<grid_for((uint64_t)K * b, 64), 64, 0, s>>>((const uint8_t*)hstmt, k0, K, R, b,
                                                                                    (fr*)bvec));
}
void step1_sparse_terms(const void* A, const void* bvec, uint32_t k0, uint32_t K, uint32_t R, uint32_t h, uint32_t b,
                        void* out, cudaStream_t s) {
    const uint32_t cmax = std::min(b, 2 * h);
    cudaMemsetAsync(out, 0, (size_t)K * 2 * h * G1J_BYTES, s);
    FP_KERNEL("k_sparse_g", s, k_sparse_g<<<(unsigned)(((uint64_t)K * cmax + 15) / 16), 128, 0, s>>>(
                                   (const g1a*)A, (const fr*)bvec, k0, K, R, h, b, cmax, (g1j*)out));
}
void step1_gt_out(const void* ml, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s) {
    final_exp_group(ml, 2 * K, nullptr, (uint8_t*)blocks + (size_t)(j - 1) * ROUND_BYTES, 2, bopen_len,
                    GT_SER + G1_SER, s);
}
void step1_g1_out(const void* sp, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s) {
    FP_KERNEL("k_round_g1_out", s, k_round_g1_out<<<grid_for((uint64_t)K * 8, 64), 64, 0, s>>>((const g1j*)sp, K, j,
                                                                                          (uint8_t*)blocks,
                                                                                          bopen_len));
}
void step1_challenge(void* blocks, size_t bopen_len, uint32_t K, int j, void* xprev, void* x_mont, void* xinv_mont,
                     void* xinv_all, int log_r, cudaStream_t s) {
    FP_KERNEL("k_challenge2", s, k_challenge2<<<(K + 1) / 2, 64, 0, s>>>((const uint8_t*)blocks, bopen_len, K, j,
                                                                         (uint8_t*)xprev, (fr*)x_mont, (fr*)xinv_mont,
                                                                         (fr*)xinv_all, log_r));
}
void step1_kzg(const void* A, const void* v, const void* xprev, const void* xinv_all, uint32_t K, uint32_t R,
               int log_r, void* blocks, size_t bopen_len, void* pcoef, void* q_canon, cudaStream_t s) {
    // chunks of C >= 32 coefficients, at most one per thread: C <= KZG_CHUNK_MAX for 2R - 2 <= 2^14
    const uint32_t deg = 2 * R - 2;
    uint32_t C = (deg + KZG_THREADS - 1) / KZG_THREADS;
    if (C < 32) C = 32;
    FP_KERNEL("k_kzg_p", s, k_kzg_p<<<K, KZG_THREADS, 0, s>>>((const g1a*)A, (const g2a*)v, (const uint8_t*)xprev,
                                                             (const fr*)xinv_all, K, R, log_r, (uint8_t*)blocks,
                                                             bopen_len, (fr*)pcoef, (fr*)q_canon, C));
}
// Comb tables of fixed G2 bases (the W proofs' g2^{beta^i}, built once at setup): per base its 64
// position tables (gpt_g2_comb_table) at tab[(i 64 + pos) 16], from the chain 2^pos B_i (a warp per
// base, then a thread per table).
__global__ void __launch_bounds__(128) k_g2_chain(const g2a* pts, uint32_t n, GPt<fq2>* chain) {
    __shared__ GEcWs sm[4];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
    if (t >= n) return;                                       // warp-uniform
    GPt<fq2> acc = gec_from_affine_or_inf(pts[t].x, pts[t].y);
    for (int i = 0; i < 64; i++) {
        if (i) acc = gecw_dbl(sm[w], L, acc);
        if (L == 0) chain[t * 64 + i] = acc;
    }
}
__global__ void __launch_bounds__(64) k_g2_comb_tab(uint64_t m, const GPt<fq2>* chain, GPt<fq2>* tab) {
    const uint64_t u = gtid();
    if (u < m) gpt_g2_comb_table(chain[u], tab + u * 16);
}
size_t g2_comb_bytes(uint32_t n) { return (size_t)n * 64 * 16 * sizeof(GPt<fq2>); }
size_t g2_comb_chain_bytes(uint32_t n) { return (size_t)n * 64 * sizeof(GPt<fq2>); }
void g2_comb_tables(const void* pts_g2a, uint32_t n, void* chain_scratch, void* tab, cudaStream_t s) {
    if (!n) return;
    FP_KERNEL("k_g2_chain", s, k_g2_chain<<<(n + 3) / 4, 128, 0, s>>>((const g2a*)pts_g2a, n, (GPt<fq2>*)chain_scratch));
    FP_KERNEL("k_g2_comb_tab", s, k_g2_comb_tab<<<grid_for((uint64_t)n * 64, 64), 64, 0, s>>>(
                                      (uint64_t)n * 64, (const GPt<fq2>*)chain_scratch, (GPt<fq2>*)tab));
}

// W terms q_i g2^{beta^i} from the comb tables: one 128-thread block per term (k, i < 2R), 16 8-lane
// groups on G2 (group_ec.cuh with F = Fq2) each adding the entries of positions g, g + 16, g + 32,
// g + 48 of the GLS digits of q_i, then a tree over the groups; term 2R - 1 is the identity
__global__ void __launch_bounds__(128) k_w_comb(const GPt<fq2>* tab, const fr* q_canon, uint32_t R, g2j* out) {
    __shared__ GEcs<fq2> e[16];
    __shared__ GPt<fq2> part[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t t = blockIdx.x;
    const uint32_t i = (uint32_t)(t % (2 * R));
    const bool live = i < 2 * R - 1;
    uint32_t d[4][2];
    gls_digits(d, q_canon[t].v);
    const GPt<fq2>* tb = tab + (size_t)(live ? i : 0) * 64 * 16;
    const GPt<fq2> id = gec_identity<fq2>();
    GPt<fq2> acc = live ? tb[grp * 16 + gls_position(d, grp)] : id;
    for (int j = 1; j < 4; j++) {
        const int pos = grp + 16 * j;
        acc = gec_add(e[grp], lane, acc, live ? tb[pos * 16 + gls_position(d, pos)] : id);
    }
    for (int sh = 8; sh >= 1; sh >>= 1) {
        __syncthreads();
        if (lane == 0) part[grp] = acc;
        __syncthreads();
        const GPt<fq2> r = gec_add(e[grp], lane, acc, part[grp < sh ? grp + sh : grp]);
        if (grp < sh) acc = r;
    }
    if (grp == 0 && lane == 0) out[t] = proj_to_jac(acc);
}
void step1_w_comb(const void* tab, const void* q_canon, uint32_t K, uint32_t R, void* out, cudaStream_t s) {
    FP_KERNEL("k_w_comb", s, k_w_comb<<<(unsigned)((uint64_t)K * 2 * R), 128, 0, s>>>((const GPt<fq2>*)tab,
                                                                                    (const fr*)q_canon, R, (g2j*)out));
}

void step1_w_terms(const void* g2pow, const void* q_canon, uint32_t K, uint32_t R, void* out, cudaStream_t s) {
    const uint64_t n = (uint64_t)K * 2 * R;
    if (n <= engine_limits().wterm_warp_max) {      // few terms: a warp per term for latency
        FP_KERNEL("k_w_terms_w", s, k_w_terms_w<<<(unsigned)((n + 3) / 4), 128, 0, s>>>((const g2a*)g2pow,
                                                                                       (const fr*)q_canon, K, R,
                                                                                       (g2j*)out));
        return;
    }
    FP_KERNEL("k_w_terms", s, k_w_terms<<<grid_for(n, 64), 64, 0, s>>>((const g2a*)g2pow, (const fr*)q_canon, K, R,
                                                                      (g2j*)out));
}

}  // namespace fpk

namespace fpk {
uint64_t step1_miller_g(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, void* ml_out,
                        cudaStream_t s) {
    uint64_t n = (uint64_t)K * 2 * h;
    const EngineLimits lim = engine_limits();
    if (n > lim.miller_warp_max && n > lim.miller_block_max) {   // many pairs: threads, less work than warps
        const uint32_t group = step1_miller_group(n, h, lim);
        step1_miller(A, v, K, R, h, group, ml_out, s);
        return n / group;
    }
    round_miller_w(A, v, K, R, h, ml_out, s);      // few pairs: one warp or block each, for latency
    return n;
}
void step1_fold_pre(const void* A, const void* v, void* comb, uint32_t n_max, uint32_t K, uint32_t R, uint32_t h,
                    cudaStream_t s) {
    const uint32_t n = K * h;
    if (n > n_max) return;
    const CombPtrs c = comb_ptrs(comb, n_max);
    const uint32_t nb2 = (n + 3) / 4, nb1 = (n + 15) / 16;
    FP_KERNEL("k_comb_chain", s, k_comb_chain<<<nb2 + nb1, 128, 0, s>>>((const g1a*)A, (const g2a*)v, K, R, h, nb2,
                                                                       c.chain1, c.chain2));
    FP_KERNEL("k_comb_tab", s, k_comb_tab<<<grid_for((uint64_t)n * 128, 64), 64, 0, s>>>(n, c.chain1, c.chain2,
                                                                                       c.tab1, c.tab2));
}
void step1_fold(void* A, void* v, void* bvec, const void* x_mont, const void* xinv_mont, uint32_t K, uint32_t R,
                uint32_t h, const void* comb, uint32_t n_max, cudaStream_t s) {
    if (comb && (uint64_t)K * h <= n_max) {            // comb tables ready: table entries only
        const uint32_t n = K * h;
        const CombPtrs c = comb_ptrs(const_cast<void*>(comb), n_max);
        FP_KERNEL("k_fold_c", s, k_fold_c<<<n + (n + 1) / 2, 256, 0, s>>>((g1a*)A, (g2a*)v, (fr*)bvec,
                                                                         (const fr*)x_mont, (const fr*)xinv_mont, K,
                                                                         R, h, c.tab1, c.tab2));
        return;
    }
    if ((uint64_t)K * h <= engine_limits().fold_warp_max) {   // few points: a warp per G2 point, 8 lanes per G1
        const uint32_t nb2 = (uint32_t)(((uint64_t)K * h + 3) / 4), nb1 = (uint32_t)(((uint64_t)K * h + 15) / 16);
        FP_KERNEL("k_fold_w", s, k_fold_w<<<nb2 + nb1, 128, 0, s>>>((g1a*)A, (g2a*)v, (fr*)bvec, (const fr*)x_mont,
                                                                  (const fr*)xinv_mont, K, R, h, nb2));
        return;
    }
    uint32_t nb = grid_for((uint64_t)K * h, 64);
    FP_KERNEL("k_fold", s, k_fold<<<2 * nb, 64, 0, s>>>((g1a*)A, (g2a*)v, (fr*)bvec, (const fr*)x_mont,
                                                        (const fr*)xinv_mont, K, R, h, nb));
}
}  // namespace fpk
