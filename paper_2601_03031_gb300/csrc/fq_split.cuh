// One Fq Montgomery product computed by the four warps of a 128-thread block together.
//
// A single lane's CIOS product (fp.cuh) is one warp's instruction stream of ~700 carry-chain
// multiply-adds; however many lanes take part, that stream runs on one of the SM's four
// sub-partitions, and it sets the latency of every round of the latency-bound engines.  Here lane
// t of each of the four warps (one warp per sub-partition) takes a quarter of product t, so a round
// of up to 32 products costs about a quarter of the multiply-adds per sub-partition plus two block
// barriers:
//   1. warp w: P_w = (x_{3w} + x_{3w+1} 2^32 + x_{3w+2} 2^64) y, three rows of the schoolbook
//      product (15 limbs), to shared memory;
//   2. every warp: T = x y = sum_w P_w 2^(96 w) (24 limbs); warp w folds its share of the low limbs,
//      S_w = sum_{k in K_w} T_k c_k with c_k = 2^(32 k - 320) mod p (K_w = {3w, 3w + 1, 3w + 2}
//      minus k >= 10), and warp 3 adds T >> 320; then
//      S = sum_w S_w = T 2^-320 (mod p) and S < 10 2^32 p + p^2 / 2^320 < 2^442 (14 limbs);
//   3. every warp: S + m p with m = -S p^-1 mod 2^64 is divisible by 2^64, and
//      X = (S + m p) / 2^64 = x y 2^-384 (mod p) with X < 2^378 + p < 2p; one conditional
//      subtraction gives the canonical value, equal to the one-lane product's.
// Every lane of every warp ends with product t (lanes whose operands are unused still compute a
// valid product).  All 128 threads of the block must call it with operands below p.
#pragma once
#include "fp.cuh"

struct FqSplitScratch {
    uint32_t a[4][15][32];   // phase-1 partials (warp, limb, lane): lane-minor, no bank conflicts
    uint32_t b[4][14][32];   // phase-2 partials
};

namespace fqs {
// acc[O .. O + 12] += a v (v: 12 limbs), the carry into acc[O + 13]
template <int O>
FPG_DEV void row_mac(uint32_t* acc, uint32_t a, const uint32_t* v) {
    acc[O] = ptx::mad_lo_cc(a, v[0], acc[O]);
#pragma unroll
    for (int j = 1; j < 12; j++) acc[O + j] = ptx::madc_lo_cc(a, v[j], acc[O + j]);
    acc[O + 12] = ptx::addc_cc(acc[O + 12], 0);
    acc[O + 13] = ptx::addc(acc[O + 13], 0);
    acc[O + 1] = ptx::mad_hi_cc(a, v[0], acc[O + 1]);
#pragma unroll
    for (int j = 1; j < 12; j++) acc[O + j + 1] = ptx::madc_hi_cc(a, v[j], acc[O + j + 1]);
    acc[O + 13] = ptx::addc(acc[O + 13], 0);
}

// the three limbs x_{3w}, x_{3w+1}, x_{3w+2} of warp w, chosen by selects so that every warp runs one
// instruction stream (four differing streams would each take their own room in the instruction cache)
FPG_DEV uint32_t limb_of_warp(const uint32_t* v, int w, int i) {
    return w == 0 ? v[i] : w == 1 ? v[3 + i] : w == 2 ? v[6 + i] : v[9 + i];
}

FPG_DEV void phase1(FqSplitScratch& sc, int w, int t, const fq& x, const fq& y) {
    uint32_t P[16];
#pragma unroll
    for (int j = 0; j < 16; j++) P[j] = 0;
    row_mac<0>(P, limb_of_warp(x.v, w, 0), y.v);
    row_mac<1>(P, limb_of_warp(x.v, w, 1), y.v);
    row_mac<2>(P, limb_of_warp(x.v, w, 2), y.v);
#pragma unroll
    for (int k = 0; k < 15; k++) sc.a[w][k][t] = P[k];
}

// warp w folds T_k for k = 3 w + i, i < 3 (k = 10, 11 have zero constants); warp 3 also adds T >> 320
FPG_DEV void phase2(FqSplitScratch& sc, int w, int t) {
    uint32_t T[24];
#pragma unroll
    for (int k = 0; k < 15; k++) T[k] = sc.a[0][k][t];
#pragma unroll
    for (int k = 15; k < 24; k++) T[k] = 0;
#pragma unroll
    for (int v = 1; v < 4; v++) {
        T[3 * v] = ptx::add_cc(T[3 * v], sc.a[v][0][t]);
#pragma unroll
        for (int k = 1; k < 15; k++) T[3 * v + k] = ptx::addc_cc(T[3 * v + k], sc.a[v][k][t]);
#pragma unroll
        for (int k = 3 * v + 15; k < 24; k++) T[k] = ptx::addc_cc(T[k], 0);
    }
    const uint32_t hi = w == 3 ? 0xffffffffu : 0u;
    uint32_t A[15];
#pragma unroll
    for (int j = 0; j < 14; j++) A[j] = T[10 + j] & hi;
    A[14] = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int k = 3 * w + i;
        uint32_t c[12];
#pragma unroll
        for (int j = 0; j < 12; j++) c[j] = FQ_FOLD[k][j];
        row_mac<0>(A, limb_of_warp(T, w, i), c);
    }
#pragma unroll
    for (int k = 0; k < 14; k++) sc.b[w][k][t] = A[k];
}

FPG_DEV fq phase3(const FqSplitScratch& sc, int t) {
    uint32_t U[16];
#pragma unroll
    for (int k = 0; k < 14; k++) U[k] = sc.b[0][k][t];
    U[14] = 0;
    U[15] = 0;
#pragma unroll
    for (int w = 1; w < 4; w++) {
        U[0] = ptx::add_cc(U[0], sc.b[w][0][t]);
#pragma unroll
        for (int k = 1; k < 14; k++) U[k] = ptx::addc_cc(U[k], sc.b[w][k][t]);
        U[14] = ptx::addc(U[14], 0);
    }
    const uint32_t m0 = U[0] * FQ_PINV64_LO;
    const uint32_t m1 = __umulhi(U[0], FQ_PINV64_LO) + U[0] * FQ_PINV64_HI + U[1] * FQ_PINV64_LO;
    uint32_t pl[12];
#pragma unroll
    for (int j = 0; j < 12; j++) pl[j] = FQ_P[j];
    row_mac<0>(U, m0, pl);
    row_mac<1>(U, m1, pl);
    fq X, D;
#pragma unroll
    for (int j = 0; j < 12; j++) X.v[j] = U[2 + j];
    D.v[0] = ptx::sub_cc(X.v[0], pl[0]);
#pragma unroll
    for (int j = 1; j < 12; j++) D.v[j] = ptx::subc_cc(X.v[j], pl[j]);
    const uint32_t borrow = ptx::subc(U[14], 0);      // all-ones when X < p
    return fq_select(borrow != 0, X, D);
}
}  // namespace fqs

// x y 2^-384 mod p for the operands of lane t = threadIdx.x % 32, the work split over the four warps
// (all 128 threads call; two block barriers)
FPG_NOINL fq fq_mul_split(fq x, fq y) {
    __shared__ FqSplitScratch sc;
    const int w = (threadIdx.x >> 5) & 3, t = threadIdx.x & 31;
    fqs::phase1(sc, w, t, x, y);
    __syncthreads();
    fqs::phase2(sc, w, t);
    __syncthreads();
    return fqs::phase3(sc, t);
}
