// Evaluation proof of the committed vector's multilinear extension at a point r (Sec. 4.4,
// "Compatibility with a family of zkSNARKs", Eq. fANDfj).  Variable k pairs with bit k of
// i = j M + a: the column variables r_R = (r_0 .. r_{l_c - 1}), the row variables
// r_L = (r_{l_c} .. r_{log N - 1}).
//   T_j = prod_{s < l_R} (j_s r_{l_c + s} + (1 - j_s)(1 - r_{l_c + s}))       (T_{j, log mu}(r_L))
//   F[a] = sum_j T_j m[j M + a], y = F(r_R) = f_m(r)
//   C_F = sum_j T_j C_j (one MSM over the row commitments), the FC proof of C_F = <C, T> (FC.BOpen
//   with t = 1: r_0 = HFr("FP-r", SHA256("FP-eval" || C || u32be(log N) || r || C_F) || u32be(0)),
//   b = r_0 T, through the Step-1 round chain), and PST.Eval(F, r_R): for t = l_c - 1 .. 0,
//   q_t[c] = F[2^t + c] - F[c], pi_t = sum_c q_t[c] Lambda_t[c], F[c] <- F[c] + r_t q_t[c].
#include "group_ec.cuh"
#include "k_common.cuh"

namespace fpk {

// r_k from 32 canonical big-endian bytes each; err |= 1 for a value >= r
__global__ void k_eval_point(const uint8_t* r_be, int log_n, fr* r_mont, uint32_t* err) {
    const uint64_t k = gtid();
    if (k >= (uint64_t)log_n) return;
    fr c;
    const uint8_t* b = r_be + 32 * k;
    for (int w = 0; w < 8; w++) {
        const uint8_t* q = b + (7 - w) * 4;
        c.v[w] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
    }
    if (!mp::lt<8>(c.v, FR_P)) {
        atomicOr(err, 1u);
        fr_zero(c);
    }
    r_mont[k] = fr_to_mont(c);
}

// T_j for j < R, Montgomery and canonical (the MSM scalars)
__global__ void k_eval_weights(const fr* r_mont, int log_r, int log_c, fr* T_mont, fr* T_canon) {
    const uint64_t j = gtid();
    if (j >= (1ull << log_r)) return;
    fr one, acc;
    fr_one(one);
    acc = one;
    for (int s = 0; s < log_r; s++) {
        const fr rv = r_mont[log_c + s];
        acc = fr_mul(acc, ((j >> s) & 1) ? rv : fr_sub(one, rv));
    }
    T_mont[j] = acc;
    T_canon[j] = fr_from_mont(acc);
}

// F[a] = sum_j T_j m[j M + a] (Montgomery)
__global__ void k_eval_ftable(const fr* m_mont, const fr* T_mont, uint32_t R, uint32_t M, fr* F) {
    const uint64_t a = gtid();
    if (a >= M) return;
    fr acc;
    fr_zero(acc);
    for (uint32_t j = 0; j < R; j++) acc = fr_add(acc, fr_mul(T_mont[j], m_mont[(uint64_t)j * M + a]));
    F[a] = acc;
}

// r_0 from the statement (one thread), then bvec[j] = r_0 T_j
__global__ void k_eval_r0(const uint8_t* C_ser, const uint8_t* r_be, int log_n, const uint8_t* CF_ser, fr* r0) {
    if (gtid() != 0) return;
    sha256_ctx c;
    sha256_init(c);
    sha256_update(c, (const uint8_t*)"FP-eval", 7);
    sha256_update(c, C_ser, 576);
    uint8_t n4[4];
    put_be32(n4, (uint32_t)log_n);
    sha256_update(c, n4, 4);
    sha256_update(c, r_be, 32 * (uint32_t)log_n);
    sha256_update(c, CF_ser, 96);
    uint8_t buf[36];
    sha256_final(c, buf);
    put_be32(buf + 32, 0);
    r0[0] = hash_to_fr("FP-r", 4, buf, 36, nullptr, 0, nullptr, 0);
}
__global__ void k_eval_bvec(const fr* r0, const fr* T_mont, uint32_t R, fr* bvec) {
    const uint64_t j = gtid();
    if (j < R) bvec[j] = fr_mul(r0[0], T_mont[j]);
}

// PST.Eval's folds in one CTA: level t's quotient table at q + 2^t - 1 (the offset of Lambda_t),
// F folded in place; y = the final F[0], serialised
__global__ void __launch_bounds__(1024) k_eval_fold(fr* F, const fr* r_mont, int log_c, fr* q, uint8_t* y_out) {
    for (int t = log_c - 1; t >= 0; t--) {
        const uint32_t w = 1u << t;
        const fr rt = r_mont[t];
        for (uint32_t c = threadIdx.x; c < w; c += blockDim.x) {
            const fr d = fr_sub(F[w + c], F[c]);
            q[w - 1 + c] = d;
            F[c] = fr_add(F[c], fr_mul(rt, d));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) fr_to_be(y_out, F[0]);
}

// terms q_t[c] Lambda_t[c] (flat index e = 2^t - 1 + c for both tables), one 8-lane group each,
// written to out[t (M/2) + c] as Jacobian (the other slots of a level stay the identity)
__global__ void __launch_bounds__(128) k_eval_pst_terms(const fr* q, const g1a* lam, uint32_t M, g1j* out) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t e0 = (uint64_t)blockIdx.x * 16 + grp;
    const bool valid = e0 < M - 1;
    const uint64_t e = valid ? e0 : 0;
    const int t = 31 - __clz((uint32_t)(e + 1));
    const uint64_t c = e + 1 - (1ull << t);
    uint32_t kw[8];
    fr_canon_words(kw, q[e]);
    const GPt<fq> r = gec_g1_mul_proj_w2(sm[grp], lane, lam[e], kw);
    if (valid && lane == 0) {
        g1j o;
        o.X = fq_mul(r.X, r.Z);
        o.Y = fq_mul(r.Y, fq_sqr(r.Z));
        o.Z = r.Z;
        out[(uint64_t)t * (M / 2) + c] = o;
    }
}

void eval_point(const void* r_be, int log_n, void* r_mont, uint32_t* err, cudaStream_t s) {
    FP_KERNEL("k_eval_point", s, k_eval_point<<<1, 32, 0, s>>>((const uint8_t*)r_be, log_n, (fr*)r_mont, err));
}
void eval_weights(const void* r_mont, int log_r, int log_c, void* T_mont, void* T_canon, cudaStream_t s) {
    FP_KERNEL("k_eval_weights", s, k_eval_weights<<<grid_for(1ull << log_r, 64), 64, 0, s>>>(
                                       (const fr*)r_mont, log_r, log_c, (fr*)T_mont, (fr*)T_canon));
}
void eval_ftable(const void* m_mont, const void* T_mont, uint32_t R, uint32_t M, void* F, cudaStream_t s) {
    FP_KERNEL("k_eval_ftable", s, k_eval_ftable<<<grid_for(M, 64), 64, 0, s>>>((const fr*)m_mont, (const fr*)T_mont,
                                                                             R, M, (fr*)F));
}
void eval_bvec(const void* C_ser, const void* r_be, int log_n, const void* CF_ser, const void* T_mont, uint32_t R,
               void* r0, void* bvec, cudaStream_t s) {
    FP_KERNEL("k_eval_r0", s, k_eval_r0<<<1, 32, 0, s>>>((const uint8_t*)C_ser, (const uint8_t*)r_be, log_n,
                                                        (const uint8_t*)CF_ser, (fr*)r0));
    FP_KERNEL("k_eval_bvec", s, k_eval_bvec<<<grid_for(R, 64), 64, 0, s>>>((const fr*)r0, (const fr*)T_mont, R,
                                                                         (fr*)bvec));
}
void eval_pst_fold(void* F, const void* r_mont, int log_c, void* q, void* y_out, cudaStream_t s) {
    FP_KERNEL("k_eval_fold", s, k_eval_fold<<<1, 1024, 0, s>>>((fr*)F, (const fr*)r_mont, log_c, (fr*)q,
                                                              (uint8_t*)y_out));
}
void eval_pst_terms(const void* q, const void* lam, uint32_t M, void* out, cudaStream_t s) {
    if (M < 2) return;
    FP_KERNEL("k_eval_pst_terms", s, k_eval_pst_terms<<<grid_for(M - 1, 16), 128, 0, s>>>((const fr*)q,
                                                                                        (const g1a*)lam, M,
                                                                                        (g1j*)out));
}

}  // namespace fpk
