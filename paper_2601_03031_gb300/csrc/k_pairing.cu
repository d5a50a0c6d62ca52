// Batched Miller loops and final exponentiations.
#include "k_common.cuh"
#include "warp12.cuh"

namespace fpk {

// FC.Commit (Eq. genC): pair j is (C_j, v_j = g2^{beta^{2j}})
__global__ void __launch_bounds__(64) k_commit_miller(const g1a* rows, const g2a* g2pow, uint32_t R, fq12* out) {
    uint64_t j = gtid();
    if (j >= R) return;
    out[j] = miller_loop(rows[j], g2pow[2 * j]);
}

// Round j of FC.BOpen (Eq. folding) for every block at once, h = R / 2^j:
// pair t = (k, side, i): side 0 -> (A_R)[i] with (v_L)[i]  (L_j.T), side 1 -> (A_L)[i] with (v_R)[i]  (R_j.T)
__global__ void __launch_bounds__(64) k_step1_miller(const g1a* A, const g2a* v, uint32_t K, uint32_t R, uint32_t h,
                                                     fq12* out) {
    uint64_t t = gtid();
    if (t >= (uint64_t)K * 2 * h) return;
    uint64_t k = t / (2 * h);
    uint32_t r = (uint32_t)(t % (2 * h)), side = r / h, i = r % h;
    const g1a* Ak = A + k * R;
    const g2a* vk = v + k * R;
    out[t] = side == 0 ? miller_loop(Ak[h + i], vk[i]) : miller_loop(Ak[i], vk[h + i]);
}

// G consecutive pairs of the same (k, side) product in one multi-pair Miller loop; output t covers
// pairs (k, side, i) with i in [G t', G t' + G), t = (k 2 + side) (h / G) + t'
template <int G>
__global__ void __launch_bounds__(64) k_step1_miller_multi(const g1a* A, const g2a* v, uint32_t K, uint32_t R,
                                                           uint32_t h, fq12* out) {
    const uint64_t t = gtid();
    const uint32_t per = h / G;
    if (t >= (uint64_t)K * 2 * per) return;
    const uint64_t k = t / (2 * per);
    const uint32_t r = (uint32_t)(t % (2 * per)), side = r / per, i0 = (r % per) * G;
    const g1a* Ak = A + k * R;
    const g2a* vk = v + k * R;
    g1a P[G];
    g2a Q[G];
    for (int g = 0; g < G; g++) {
        P[g] = side == 0 ? Ak[h + i0 + g] : Ak[i0 + g];
        Q[g] = side == 0 ? vk[i0 + g] : vk[h + i0 + g];
    }
    out[t] = miller_loop_multi<G>(P, Q);
}

// one warp per final exponentiation (warp12.cuh): value t's result goes to out[t] and/or its
// serialisation to ser + (t / per) stride_a + (t % per) stride_b
__global__ void __launch_bounds__(128) k_final_exp_w(const fq12* in, uint32_t n, fq12* out, uint8_t* ser,
                                                     uint32_t per, size_t stride_a, size_t stride_b) {
    __shared__ W12 sm[4];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
    if (t >= n) return;                                   // warp-uniform
    W12& W = sm[w];
    w_from_tower<1>(W.s[0], in[t]);
    w_final_exp<1>(W);
    if (L < 12) {
        const int tp = w_tower_pos(L >> 1), e = L & 1;
        const fq v = W.s[2][L];
        if (out) reinterpret_cast<fq*>(&out[t])[2 * tp + e] = v;
        if (ser) fq_to_be(ser + (t / per) * stride_a + (t % per) * stride_b + 96 * tp + 48 * e, v);
    }
}

// one 128-thread block per final exponentiation (few of them: the 108 products of an Fq12
// product take one round instead of four)
__global__ void __launch_bounds__(128) k_final_exp_c(const fq12* in, uint32_t n, fq12* out, uint8_t* ser,
                                                     uint32_t per, size_t stride_a, size_t stride_b) {
    __shared__ W12 W;
    const int L = threadIdx.x;
    const uint64_t t = blockIdx.x;
    w_from_tower<4>(W.s[0], in[t]);
    w_final_exp<4>(W);
    if (L < 12) {
        const int tp = w_tower_pos(L >> 1), e = L & 1;
        const fq v = W.s[2][L];
        if (out) reinterpret_cast<fq*>(&out[t])[2 * tp + e] = v;
        if (ser) fq_to_be(ser + (t / per) * stride_a + (t % per) * stride_b + 96 * tp + 48 * e, v);
    }
}

// one thread per final exponentiation (many of them: the least work in total)
__global__ void k_final_exp_t(const fq12* in, uint32_t n, fq12* out, uint8_t* ser, uint32_t per, size_t stride_a,
                              size_t stride_b) {
    const uint64_t t = gtid();
    if (t >= n) return;
    const fq12 r = final_exp(in[t]);
    if (out) out[t] = r;
    if (ser) {
        const fq* c = reinterpret_cast<const fq*>(&r);
        for (int q = 0; q < 12; q++) fq_to_be(ser + (t / per) * stride_a + (t % per) * stride_b + 48 * q, c[q]);
    }
}

void final_exp_group(const void* in, uint32_t n, void* out, void* ser, uint32_t per, size_t stride_a,
                     size_t stride_b, cudaStream_t s) {
    if (!n) return;
    const EngineLimits lim = engine_limits();
    if (n > lim.fe_warp_max && n > lim.fe_block_max) {
        FP_KERNEL("k_final_exp_t", s, k_final_exp_t<<<grid_for(n, 64), 64, 0, s>>>((const fq12*)in, n, (fq12*)out,
                                                                                  (uint8_t*)ser, per, stride_a,
                                                                                  stride_b));
        return;
    }
    if (n <= lim.fe_block_max) {
        FP_KERNEL("k_final_exp_c", s, k_final_exp_c<<<n, 128, 0, s>>>((const fq12*)in, n, (fq12*)out, (uint8_t*)ser, per,
                                                                     stride_a, stride_b));
        return;
    }
    FP_KERNEL("k_final_exp_w", s, k_final_exp_w<<<(n + 3) / 4, 128, 0, s>>>((const fq12*)in, n, (fq12*)out,
                                                                           (uint8_t*)ser, per, stride_a, stride_b));
}

// pairwise Fq12 products out[i] = in[2i] in[2i+1]: one 128-thread block per product when there are
// few (latency), one thread per product otherwise
__global__ void k_fq12_pair(const fq12* in, fq12* out, uint64_t n) {
    uint64_t i = gtid();
    if (i < n) out[i] = fq12_mul(in[2 * i], in[2 * i + 1]);
}
__global__ void __launch_bounds__(128) k_fq12_pair_c(const fq12* in, fq12* out) {
    __shared__ W12 W;
    const int L = threadIdx.x;
    const uint64_t i = blockIdx.x;
    if (L < 12) {
        const int pos = 2 * w_tower_pos(L >> 1) + (L & 1);
        W.s[0][L] = reinterpret_cast<const fq*>(&in[2 * i])[pos];
        W.s[1][L] = reinterpret_cast<const fq*>(&in[2 * i + 1])[pos];
    }
    __syncthreads();
    w_mul<4>(W, W.s[2], W.s[0], W.s[1]);
    if (L < 12) reinterpret_cast<fq*>(&out[i])[2 * w_tower_pos(L >> 1) + (L & 1)] = W.s[2][L];
}
void fq12_pair_reduce(const void* in, void* out, uint64_t n, cudaStream_t s) {
    if (!n) return;
    if (n <= engine_limits().pair_block_max) {
        FP_KERNEL("k_fq12_pair_c", s, k_fq12_pair_c<<<(unsigned)n, 128, 0, s>>>((const fq12*)in, (fq12*)out));
        return;
    }
    FP_KERNEL("k_fq12_pair", s, k_fq12_pair<<<grid_for(n, 64), 64, 0, s>>>((const fq12*)in, (fq12*)out, n));
}

// Miller loops, one warp per pair (warp12.cuh).  Pair t of Step 1 round h: t = (k, side, i) with
// side 0: (A_k[h + i], v_k[i]) and side 1: (A_k[i], v_k[h + i]); Commit: (C_j, v_j = g2pow[2 j]).
__global__ void __launch_bounds__(128) k_round_miller_w(const g1a* A, const g2a* v, uint32_t K, uint32_t R,
                                                        uint32_t h, fq12* out) {
    __shared__ WMill sm[4];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t t = (uint64_t)blockIdx.x * 4 + w;
    if (t >= (uint64_t)K * 2 * h) return;                 // warp-uniform
    const uint64_t k = t / (2 * h);
    const uint32_t r = (uint32_t)(t % (2 * h)), side = r / h, i = r % h;
    const g1a* Ak = A + k * R;
    const g2a* vk = v + k * R;
    if (side == 0) w_miller<1>(sm[w], Ak[h + i], vk[i]);
    else w_miller<1>(sm[w], Ak[i], vk[h + i]);
    if (L < 12) reinterpret_cast<fq*>(&out[t])[2 * w_tower_pos(L >> 1) + (L & 1)] = sm[w].f[L];
}
__global__ void __launch_bounds__(128) k_commit_miller_w(const g1a* rows, const g2a* g2pow, uint32_t R, fq12* out) {
    __shared__ WMill sm[4];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t j = (uint64_t)blockIdx.x * 4 + w;
    if (j >= R) return;
    w_miller<1>(sm[w], rows[j], g2pow[2 * j]);
    if (L < 12) reinterpret_cast<fq*>(&out[j])[2 * w_tower_pos(L >> 1) + (L & 1)] = sm[w].f[L];
}
// the same with one 128-thread block per pair (fewer rounds per step)
__global__ void __launch_bounds__(128) k_round_miller_c(const g1a* A, const g2a* v, uint32_t K, uint32_t R,
                                                        uint32_t h, fq12* out) {
    __shared__ WMill S;
    const int L = threadIdx.x;
    const uint64_t t = blockIdx.x;
    const uint64_t k = t / (2 * h);
    const uint32_t r = (uint32_t)(t % (2 * h)), side = r / h, i = r % h;
    const g1a* Ak = A + k * R;
    const g2a* vk = v + k * R;
    if (side == 0) w_miller<4>(S, Ak[h + i], vk[i]);
    else w_miller<4>(S, Ak[i], vk[h + i]);
    if (L < 12) reinterpret_cast<fq*>(&out[t])[2 * w_tower_pos(L >> 1) + (L & 1)] = S.f[L];
}
__global__ void __launch_bounds__(128) k_commit_miller_c(const g1a* rows, const g2a* g2pow, fq12* out) {
    __shared__ WMill S;
    const int L = threadIdx.x;
    const uint64_t j = blockIdx.x;
    w_miller<4>(S, rows[j], g2pow[2 * j]);
    if (L < 12) reinterpret_cast<fq*>(&out[j])[2 * w_tower_pos(L >> 1) + (L & 1)] = S.f[L];
}
void round_miller_w(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, void* out, cudaStream_t s) {
    const uint64_t n = (uint64_t)K * 2 * h;
    if (n <= engine_limits().miller_block_max) {
        FP_KERNEL("k_round_miller_c", s, k_round_miller_c<<<(unsigned)n, 128, 0, s>>>((const g1a*)A, (const g2a*)v, K, R,
                                                                                     h, (fq12*)out));
        return;
    }
    FP_KERNEL("k_round_miller_w", s, k_round_miller_w<<<(unsigned)((n + 3) / 4), 128, 0, s>>>((const g1a*)A,
                                                                                             (const g2a*)v, K, R, h,
                                                                                             (fq12*)out));
}

void commit_miller(const void* rows, const void* g2pow, uint32_t R, void* out, cudaStream_t s) {
    const EngineLimits lim = engine_limits();
    if (R > lim.commit_warp_max && R > lim.commit_block_max) {   // many pairs: one thread each, less work
        FP_KERNEL("k_commit_miller", s, k_commit_miller<<<grid_for(R, 64), 64, 0, s>>>((const g1a*)rows,
                                                                                       (const g2a*)g2pow, R,
                                                                                       (fq12*)out));
        return;
    }
    if (R <= lim.commit_block_max) {
        FP_KERNEL("k_commit_miller_c", s, k_commit_miller_c<<<R, 128, 0, s>>>((const g1a*)rows, (const g2a*)g2pow,
                                                                             (fq12*)out));
        return;
    }
    FP_KERNEL("k_commit_miller_w", s, k_commit_miller_w<<<(R + 3) / 4, 128, 0, s>>>((const g1a*)rows,
                                                                                   (const g2a*)g2pow, R,
                                                                                   (fq12*)out));
}
// grouping pays once the grouped threads still fill the GPU several times over (2^16 threads)
uint32_t step1_miller_group(uint64_t n, uint32_t h, const EngineLimits& lim) {
    return (h >= 4 && n >= lim.miller_group_min) ? 4 : 1;
}
void step1_miller(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, uint32_t group, void* out,
                  cudaStream_t s) {
    if (group == 4) {                                   // 4 pairs per thread share the squarings
        const uint64_t n = (uint64_t)K * 2 * (h / 4);
        FP_KERNEL("k_step1_miller_multi", s,
                  k_step1_miller_multi<4><<<grid_for(n, 64), 64, 0, s>>>((const g1a*)A, (const g2a*)v, K, R, h,
                                                                        (fq12*)out));
        return;
    }
    uint64_t n = (uint64_t)K * 2 * h;
    FP_KERNEL("k_step1_miller", s, k_step1_miller<<<grid_for(n, 64), 64, 0, s>>>((const g1a*)A, (const g2a*)v, K, R, h, (fq12*)out));
}
}  // namespace fpk
