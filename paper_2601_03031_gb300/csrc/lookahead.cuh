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
// Kernels, in the order a round uses them; before the challenge:
//   k_la_miller_c   Miller loops of the 8 pair classes, one 128-thread block per pair
//                   (then pairwise products to 8 values per block and their final exponentiations)
//   k_la_sparse     the six G1 sums' terms (then pairwise sums and affine conversion)
//   k_la_gt_pre     the shifted GT bases of the 4-part exponentiations
//   k_la_g1_pre     the shifted G1 bases of the 4-part multiplications
// after it:
//   k_la_gt_c       the parts of V^(1/x) and W^x, one 128-thread block each
//   k_la_gt_out     U times the parts, serialised into the round record
//   k_la_g1_out     S1 + x Sx + (1/x) Sxi from the parts, serialised into the round record
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

// The exponentiations V^(1/x) and W^x of block k: e = 0 V_L (class 2), 1 W_L (class 3), 2 V_R (class 6),
// 3 W_R (class 7), exponent 1/x for even e and x for odd e; each in 4 parts of 16 bits of the
// base-|x| digits (gt_exp.cuh) on the bases g^(2^(16 p)).
FPG_DEV uint32_t la_gt_class(int e) { return 2 + 4 * (e >> 1) + (e & 1); }

// gpre[(k 4 + e) 3 + p - 1] = fe[k 8 + class e]^(2^(16 p)), p = 1..3 (48 cyclotomic squarings,
// before the challenge); grid 4 K
__global__ void __launch_bounds__(128) k_la_gt_pre(const fq12* fe, fq12* gpre) {
    __shared__ W12 W;
    const uint64_t t = blockIdx.x, k = t / 4;
    const int e = (int)(t % 4), L = threadIdx.x;
    w_from_tower<4>(W.s[0], fe[k * 8 + la_gt_class(e)]);
    for (int p = 1; p < 4; p++) {
        for (int i = 0; i < 16; i++) w_cyc_sqr<4>(W, W.s[0], W.s[0]);
        if (L < 12) reinterpret_cast<fq*>(&gpre[t * 3 + p - 1])[2 * w_tower_pos(L >> 1) + (L & 1)] = W.s[0][L];
    }
}

// pwp[(k 4 + e) 4 + part] = part `part` of exponentiation e of block k; grid 16 K
__global__ void __launch_bounds__(128) k_la_gt_c(const fq12* fe, const fq12* gpre, const fr* x_mont,
                                                 const fr* xinv_mont, fq12* pwp) {
    __shared__ WGt G;
    const uint64_t t = blockIdx.x, te = t / 4, k = te / 4;
    const int part = (int)(t % 4), e = (int)(te % 4);
    uint32_t c[8];
    la_canon(c, (e & 1) ? x_mont[k] : xinv_mont[k]);
    w_from_tower<4>(G.w.s[0], part ? gpre[te * 3 + part - 1] : fe[k * 8 + la_gt_class(e)]);
    w_gt_pow_bits<4>(G, G.w.s[1], G.w.s[0], c, 16 * part, 16);
    const int L = threadIdx.x;
    if (L < 12) reinterpret_cast<fq*>(&pwp[t])[2 * w_tower_pos(L >> 1) + (L & 1)] = G.w.s[1][L];
}

// side 0: L_j.T = U_L (classes 0, 1) times the 8 parts of exponentiations 0 and 1; side 1: R_j.T from
// classes 4, 5 and exponentiations 2, 3; written big-endian at rec + k stride_k + side stride_side;
// grid 2 K
__global__ void __launch_bounds__(128) k_la_gt_out(const fq12* fe, const fq12* pwp, uint8_t* rec, size_t stride_k,
                                                   size_t stride_side) {
    __shared__ W12 W;
    const uint64_t t = blockIdx.x, k = t / 2;
    const int side = (int)(t % 2);
    w_from_tower<4>(W.s[0], fe[k * 8 + 4 * side]);
    w_from_tower<4>(W.s[1], fe[k * 8 + 4 * side + 1]);
    w_mul<4>(W, W.s[2], W.s[0], W.s[1]);
    for (int q = 0; q < 8; q++) {
        w_from_tower<4>(W.s[0], pwp[(k * 4 + 2 * side) * 4 + q]);
        w_mul<4>(W, W.s[2], W.s[2], W.s[0]);
    }
    const int L = threadIdx.x;
    if (L < 12) fq_to_be(rec + k * stride_k + side * stride_side + 96 * w_tower_pos(L >> 1) + 48 * (L & 1), W.s[2][L]);
}

// The G1 multiplications x Sx and (1/x) Sxi of (k, side), item t = k 2 + side, m = 0 (Sx) or 1 (Sxi):
// each in 4 parts on the bases 2^(32 p) S (group_ec.cuh, gec_g1_mul_part<4>).
// acc2[(t 2 + m) 3 + p - 1] = 2^(32 p) acc[k 6 + 3 side + 1 + m], p = 1..3 (before the challenge);
// one 8-lane group per (t, m), grid (4 K) / 16 blocks
__global__ void __launch_bounds__(128) k_la_g1_pre(const g1a* acc, uint32_t K, g1a* acc2) {
    __shared__ GEc<fq> sm[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t u0 = (uint64_t)blockIdx.x * 16 + grp;
    const bool valid = u0 < 4 * (uint64_t)K;
    const uint64_t u = valid ? u0 : 0, t = u / 2, k = t / 2;
    const int side = (int)(t % 2), m = (int)(u % 2);
    const g1a& s0 = acc[k * 6 + 3 * side + 1 + m];
    GPt<fq> a = gec_from_affine_or_inf(s0.x, s0.y);
    for (int p = 1; p < 4; p++) {
        a = gec_g1_dbl_n(sm[grp], lane, a, 32);
        g1a o;
        gec_to_affine(o.x, o.y, a);
        if (valid && lane == 0) acc2[u * 3 + p - 1] = o;
    }
}

// side 0: L_j.1 = L1 + x Lx + (1/x) Lxi; side 1: R_j.1 from R1, Rx, Rxi.  Two items per block, eight
// 8-lane groups each (group g: m = g / 4, part g mod 4), the eight partial results summed pairwise
// across the block; written big-endian at rec + k stride_k + side stride_side; grid K
__global__ void __launch_bounds__(128) k_la_g1_out(const g1a* acc, const g1a* acc2, const fr* x_mont,
                                                   const fr* xinv_mont, uint32_t K, uint8_t* rec, size_t stride_k,
                                                   size_t stride_side) {
    __shared__ GEc<fq> sm[16];
    __shared__ GPt<fq> sums[2][16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7, g = grp & 7, m = g >> 2, part = g & 3;
    const uint64_t t0 = (uint64_t)blockIdx.x * 2 + (grp >> 3);
    const bool valid = t0 < 2 * (uint64_t)K;
    const uint64_t t = valid ? t0 : 0, k = t / 2;
    const int side = (int)(t % 2);
    uint32_t kw[8];
    la_canon(kw, m ? xinv_mont[k] : x_mont[k]);
    GPt<fq> r = gec_g1_mul_part<4>(sm[grp], lane, part ? acc2[(t * 2 + m) * 3 + part - 1] : acc[k * 6 + 3 * side + 1 + m],
                                   kw, part);
    for (int sh = 1, b = 0; sh < 8; sh <<= 1, b ^= 1) {        // every thread of the block takes part
        if (lane == 0) sums[b][grp] = r;
        __syncthreads();
        r = gec_add(sm[grp], lane, r, sums[b][grp ^ sh]);
    }
    const g1a& s1 = acc[k * 6 + 3 * side];
    r = gec_add(sm[grp], lane, r, gec_from_affine_or_inf(s1.x, s1.y));
    g1a o;
    gec_to_affine(o.x, o.y, r);
    if (valid && g == 0 && lane == 0) g1a_to_be(rec + k * stride_k + side * stride_side, o);
}

}  // namespace fpk
