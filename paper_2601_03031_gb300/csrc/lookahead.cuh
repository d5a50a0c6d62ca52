// Look-ahead rounds of FC.BOpen (Sec. 3, Eq. folding): round j's outputs from round j-1's state and
// its challenge, so that the pairings of round j need not wait for round j-1's fold.
//
// Round j-1 has state A, v, b of length 2h per block (h = 2 h2) and challenge x; its fold gives
// A' = A_L + x A_R, v' = v_L + x^-1 v_R, b' = b_L + x^-1 b_R of length h = 2 h2.  By bilinearity,
// for i < h2,
//   e(A'[h2 + i], v'[i]) = e(A[h2 + i], v[i]) e(A[h + h2 + i], v[h + i])
//                          e(A[h2 + i], v[h + i])^(1/x) e(A[h + h2 + i], v[i])^x,
// so round j's L_j.T = U_L V_L^(1/x) W_L^x with U_L, V_L, W_L products of pairings over round j-1's
// state, and likewise R_j.T = U_R V_R^(1/x) W_R^x from e(A'[i], v'[h2 + i]).  The G1 parts expand
// the same way: L_j.1 = <A'_R, b'_L> = L1 + x Lx + (1/x) Lxi and R_j.1 = R1 + x Rx + (1/x) Rxi, with
// six sums over b's support in round j-1's state.  Everything but the final exponentiations by
// x^(+-1) (gt_exp.cuh) and the two G1 multiplications is known before x; the results are the same
// group elements as the direct round's, so the record bytes are identical.
//
// Kernels, in the order a round uses them:
//   k_la_miller_c   Miller loops of the 8 pair classes, one 128-thread block per pair
//                   (then pairwise products to 8 values per block and their final exponentiations)
//   k_la_sparse     the six G1 sums' terms (then pairwise sums and affine conversion)
//   k_la_gt_c       V^(1/x) and W^x, one 128-thread block each
//   k_la_gt_out     U V^(1/x) W^x, serialised into the round record
//   k_la_g1_out     S1 + x Sx + (1/x) Sxi, serialised into the round record
#pragma once
#include "group_ec.cuh"
#include "gt_exp.cuh"

namespace fpk {

// canonical little-endian words of a Montgomery Fr residue
FPG_DEV void la_canon(uint32_t* k, const fr& a) {
    const fr c = fr_from_mont(a);
#pragma unroll
    for (int j = 0; j < 8; j++) k[j] = c.v[j];
}

// Pair class cls (0..7) of the look-ahead Miller loops, for i < h2 in a state of half-length
// h = 2 h2: (index into A, index into v).  Classes 0, 1: U_L; 2: V_L; 3: W_L; 4, 5: U_R; 6: V_R;
// 7: W_R.
FPG_DEV void la_pair(int cls, uint32_t h2, uint32_t i, uint32_t& ia, uint32_t& iv) {
    const uint32_t h = 2 * h2;
    switch (cls) {
        case 0: ia = h2 + i; iv = i; break;
        case 1: ia = h + h2 + i; iv = h + i; break;
        case 2: ia = h2 + i; iv = h + i; break;
        case 3: ia = h + h2 + i; iv = i; break;
        case 4: ia = i; iv = h2 + i; break;
        case 5: ia = h + i; iv = h + h2 + i; break;
        case 6: ia = i; iv = h + h2 + i; break;
        default: ia = h + i; iv = h2 + i; break;
    }
}

// out[(k 8 + cls) h2 + i] = the Miller value of pair (cls, i) of block k (tower order); grid 8 K h2
__global__ void __launch_bounds__(128) k_la_miller_c(const g1a* A, const g2a* v, uint32_t R, uint32_t h2,
                                                     fq12* out) {
    __shared__ WMill S;
    const uint64_t t = blockIdx.x;
    const uint64_t k = t / (8 * (uint64_t)h2);
    const int cls = (int)((t / h2) % 8);
    const uint32_t i = (uint32_t)(t % h2);
    uint32_t ia, iv;
    la_pair(cls, h2, i, ia, iv);
    w_miller<4>(S, A[k * R + ia], v[k * R + iv]);
    const int L = threadIdx.x;
    if (L < 12) reinterpret_cast<fq*>(&out[t])[2 * w_tower_pos(L >> 1) + (L & 1)] = S.f[L];
}

// The six G1 sums' terms: two 8-lane groups per support term t < cmax of block k's b in a state of
// half-length h = 2 h2 (b's support: p = ((k0 + k) b + t) mod 2h for t < min(|S_k|, 2h), p = t when
// |S_k| > 2h), group g multiplying b[p] by one point.  With q = p / h2 and i = p mod h2:
//   q = 0: g0 A[h2 + i] -> L1,  g1 A[h + h2 + i] -> Lx      q = 1: g0 A[i] -> R1,  g1 A[h + i] -> Rx
//   q = 2: g0 A[h2 + i] -> Lxi, g1 A[h + h2 + i] -> L1      q = 3: g0 A[i] -> Rxi, g1 A[h + i] -> R1
// out[(k 6 + s) 2h + p] (Jacobian; s = 0 L1, 1 Lx, 2 Lxi, 3 R1, 4 Rx, 5 Rxi), whose other entries
// the caller has zeroed (the identity); grid (2 K cmax) / 16 blocks of 128 threads.
__global__ void __launch_bounds__(128) k_la_sparse(const g1a* A, const fr* bvec, uint32_t k0, uint32_t K, uint32_t R,
                                                   uint32_t h2, uint32_t b, uint32_t cmax, g1j* out) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7, g = grp & 1;
    const uint32_t h = 2 * h2;
    const uint64_t u0 = ((uint64_t)blockIdx.x * 16 + grp) >> 1;
    uint64_t k = u0 / cmax;
    uint32_t t = (uint32_t)(u0 % cmax);
    bool valid = k < K;
    uint32_t sk = valid ? min(b, R - (k0 + (uint32_t)k) * b) : 1;
    valid = valid && t < min(sk, 2 * h);
    if (!valid) { k = 0; t = 0; sk = min(b, R - k0 * b); }    // dummy work keeps the warp uniform
    const uint32_t p = sk <= 2 * h ? (uint32_t)(((uint64_t)(k0 + k) * b + t) % (2 * h)) : t;
    const uint32_t q = p / h2, i = p % h2;
    const uint32_t ia = (q & 1) ? (g ? h + i : i) : (g ? h + h2 + i : h2 + i);
    const int s = q == 0 ? (g ? 1 : 0) : q == 1 ? (g ? 4 : 3) : q == 2 ? (g ? 0 : 2) : (g ? 3 : 5);
    uint32_t kw[8];
    la_canon(kw, bvec[k * R + p]);
    const GPt<fq> r = gec_g1_mul_proj_w2(sm[grp], lane, A[k * R + ia], kw);
    __syncwarp();
    if (valid && lane == 0) {
        g1j o;                                                // (X : Y : Z) -> Jacobian (X Z, Y Z^2, Z)
        o.X = fq_mul(r.X, r.Z);
        o.Y = fq_mul(r.Y, fq_sqr(r.Z));
        o.Z = r.Z;
        out[(k * 6 + s) * 2 * h + p] = o;
    }
}

// pw[k 4 + e] = fe[k 8 + c_e]^(x_k^(+-1)): e = 0 V_L^(1/x) (c 2), 1 W_L^x (c 3), 2 V_R^(1/x) (c 6),
// 3 W_R^x (c 7); grid 4 K
__global__ void __launch_bounds__(128) k_la_gt_c(const fq12* fe, const fr* x_mont, const fr* xinv_mont, fq12* pw) {
    __shared__ WGt G;
    const uint64_t t = blockIdx.x, k = t / 4;
    const int e = (int)(t % 4);
    uint32_t c[8];
    la_canon(c, (e & 1) ? x_mont[k] : xinv_mont[k]);
    w_from_tower<4>(G.w.s[0], fe[k * 8 + 2 + 4 * (e >> 1) + (e & 1)]);
    w_gt_pow_bits<4>(G, G.w.s[1], G.w.s[0], c, 0, 64);
    const int L = threadIdx.x;
    if (L < 12) reinterpret_cast<fq*>(&pw[t])[2 * w_tower_pos(L >> 1) + (L & 1)] = G.w.s[1][L];
}

// side 0: L_j.T = fe[k 8] fe[k 8 + 1] pw[k 4] pw[k 4 + 1]; side 1: R_j.T from fe[k 8 + 4 ..] and
// pw[k 4 + 2 ..]; written big-endian at rec + k stride_k + side stride_side; grid 2 K
__global__ void __launch_bounds__(128) k_la_gt_out(const fq12* fe, const fq12* pw, uint8_t* rec, size_t stride_k,
                                                   size_t stride_side) {
    __shared__ W12 W;
    const uint64_t t = blockIdx.x, k = t / 2;
    const int side = (int)(t % 2);
    w_from_tower<4>(W.s[0], fe[k * 8 + 4 * side]);
    w_from_tower<4>(W.s[1], fe[k * 8 + 4 * side + 1]);
    w_mul<4>(W, W.s[2], W.s[0], W.s[1]);
    w_from_tower<4>(W.s[0], pw[k * 4 + 2 * side]);
    w_mul<4>(W, W.s[2], W.s[2], W.s[0]);
    w_from_tower<4>(W.s[1], pw[k * 4 + 2 * side + 1]);
    w_mul<4>(W, W.s[2], W.s[2], W.s[1]);
    const int L = threadIdx.x;
    if (L < 12) fq_to_be(rec + k * stride_k + side * stride_side + 96 * w_tower_pos(L >> 1) + 48 * (L & 1), W.s[2][L]);
}

// side 0: L_j.1 = L1 + x Lx + (1/x) Lxi; side 1: R_j.1 from R1, Rx, Rxi (acc: the six affine sums
// per block); two 8-lane groups per (k, side), one multiplication each, then the sum; written
// big-endian at rec + k stride_k + side stride_side; grid (4 K) / 16 blocks of 128 threads
__global__ void __launch_bounds__(128) k_la_g1_out(const g1a* acc, const fr* x_mont, const fr* xinv_mont, uint32_t K,
                                                   uint8_t* rec, size_t stride_k, size_t stride_side) {
    __shared__ GEc<fq> sm[16];
    __shared__ GPt<fq> part[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7, g = grp & 1;
    const uint64_t t0 = (uint64_t)blockIdx.x * 8 + (grp >> 1);
    const bool valid = t0 < 2 * (uint64_t)K;
    const uint64_t t = valid ? t0 : 0, k = t / 2;
    const int side = (int)(t % 2);
    uint32_t kw[8];
    la_canon(kw, g ? xinv_mont[k] : x_mont[k]);
    GPt<fq> r = gec_g1_mul_proj_w2(sm[grp], lane, acc[k * 6 + 3 * side + 1 + g], kw);
    __syncwarp();
    if (lane == 0) part[grp] = r;
    __syncwarp();
    r = gec_add(sm[grp], lane, r, part[grp ^ 1]);
    const g1a& s1 = acc[k * 6 + 3 * side];
    r = gec_add(sm[grp], lane, r, gec_from_affine_or_inf(s1.x, s1.y));
    g1a o;
    gec_to_affine(o.x, o.y, r);
    if (valid && g == 0 && lane == 0) g1a_to_be(rec + k * stride_k + side * stride_side, o);
}

}  // namespace fpk
