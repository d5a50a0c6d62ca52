// Batched Pippenger multi-scalar multiplication on G1:
//     out[j] = sum_{i < n} k[j n + i] P[(j n + i) mod npts],   j < nbatch,
// for affine bases P (Montgomery form) and 256-bit scalars k (reduced mod r first, so for bases
// in G1 the result is the integer combination).
//
//   0. GLV split: k = k0 + k1 |x|^2 with k0 < |x|^2 and k1 < r / |x|^2, both below 2^128; since
//      phi(x, y) = (omega x, y) acts as [-x^2] on G1, k P = k0 P + k1 (-phi(P)).  The bases table
//      holds P_i and -phi(P_i), so every term becomes two half-length terms.
//   1. signed digits of each half over W windows of c or c - 1 bits covering 129 bits (msm.h):
//      d in (-2^(c_w-1), 2^(c_w-1)] with a carry into the next window.  Key (batch, window,
//      |d| - 1) selects a bucket; a negative digit negates the base.
//   2. counting sort of the (base, window) entries by key: histogram with atomics, exclusive scan,
//      scatter of base index | sign bit;
//   3. bucket sums with XYZZ mixed additions, load-balanced: fixed-size chunks of the sorted entry
//      list, one thread each, partial sums of runs that cross chunks added afterwards;
//   4. bucket reduction sum_b (b + 1) B_b: the buckets of a window are cut into S segments;
//      a thread per segment forms its running sums plus (start) x (segment sum), and the segment
//      results are added pairwise;
//   5. per batch, Horner over the windows (c_w doublings each) on an 8-lane group with the
//      complete projective formulas, then one inversion to affine.
// XYZZ coordinates: x = X / ZZ, y = Y / ZZZ (ZZ^3 = ZZZ^2), identity ZZ = 0; formulas madd-2008-s,
// add-2008-s and dbl-2008-s-1 of the Explicit-Formulas Database (curve coefficient a = 0).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "group_ec.cuh"
#include "k_common.cuh"

namespace fpk {

template <typename F> struct xyzz_t { F X, Y, ZZ, ZZZ; };
using xyzz = xyzz_t<fq>;

template <typename F> FPG_DEV void xyzz_inf(xyzz_t<F>& p) { f_set_zero(p.X); f_set_zero(p.Y); f_set_zero(p.ZZ); f_set_zero(p.ZZZ); }
template <typename F> FPG_DEV bool xyzz_is_inf(const xyzz_t<F>& p) { return f_is_zero(p.ZZ); }

template <typename F>
FPG_NOINL xyzz_t<F> xyzz_dbl(const xyzz_t<F>& p) {
    if (xyzz_is_inf(p)) return p;
    const F U = f_dbl(p.Y), V = f_sqr(U), W = f_mul(U, V), S = f_mul(p.X, V);
    const F X2 = f_sqr(p.X), M = f_add(f_dbl(X2), X2);
    xyzz_t<F> r;
    r.X = f_sub(f_sqr(M), f_dbl(S));
    r.Y = f_sub(f_mul(M, f_sub(S, r.X)), f_mul(W, p.Y));
    r.ZZ = f_mul(V, p.ZZ);
    r.ZZZ = f_mul(W, p.ZZZ);
    return r;
}
// 2 (x, y) for an affine point (y != 0 on these curves: no point of order 2)
template <typename F>
FPG_DEV xyzz_t<F> xyzz_dbl_affine(const F& x, const F& y) {
    const F U = f_dbl(y), V = f_sqr(U), W = f_mul(U, V), S = f_mul(x, V);
    const F X2 = f_sqr(x), M = f_add(f_dbl(X2), X2);
    xyzz_t<F> r;
    r.X = f_sub(f_sqr(M), f_dbl(S));
    r.Y = f_sub(f_mul(M, f_sub(S, r.X)), f_mul(W, y));
    r.ZZ = V;
    r.ZZZ = W;
    return r;
}
// p + (x, y), the second point affine and not the identity
template <typename F>
FPG_NOINL xyzz_t<F> xyzz_madd(const xyzz_t<F>& p, const F& x, const F& y) {
    xyzz_t<F> r;
    if (xyzz_is_inf(p)) { r.X = x; r.Y = y; f_set_one(r.ZZ); f_set_one(r.ZZZ); return r; }
    const F U2 = f_mul(x, p.ZZ), S2 = f_mul(y, p.ZZZ);
    const F P = f_sub(U2, p.X), R = f_sub(S2, p.Y);
    if (f_is_zero(P)) {
        if (f_is_zero(R)) return xyzz_dbl_affine(x, y);
        xyzz_inf(r);
        return r;
    }
    const F PP = f_sqr(P), PPP = f_mul(P, PP), Q = f_mul(p.X, PP);
    r.X = f_sub(f_sub(f_sqr(R), PPP), f_dbl(Q));
    r.Y = f_sub(f_mul(R, f_sub(Q, r.X)), f_mul(p.Y, PPP));
    r.ZZ = f_mul(p.ZZ, PP);
    r.ZZZ = f_mul(p.ZZZ, PPP);
    return r;
}
template <typename F>
FPG_NOINL xyzz_t<F> xyzz_add(const xyzz_t<F>& p, const xyzz_t<F>& q) {
    if (xyzz_is_inf(p)) return q;
    if (xyzz_is_inf(q)) return p;
    const F U1 = f_mul(p.X, q.ZZ), U2 = f_mul(q.X, p.ZZ);
    const F S1 = f_mul(p.Y, q.ZZZ), S2 = f_mul(q.Y, p.ZZZ);
    const F P = f_sub(U2, U1), R = f_sub(S2, S1);
    xyzz_t<F> r;
    if (f_is_zero(P)) {
        if (f_is_zero(R)) return xyzz_dbl(p);
        xyzz_inf(r);
        return r;
    }
    const F PP = f_sqr(P), PPP = f_mul(P, PP), Q = f_mul(U1, PP);
    r.X = f_sub(f_sub(f_sqr(R), PPP), f_dbl(Q));
    r.Y = f_sub(f_mul(R, f_sub(Q, r.X)), f_mul(S1, PPP));
    r.ZZ = f_mul(f_mul(p.ZZ, q.ZZ), PP);
    r.ZZZ = f_mul(f_mul(p.ZZZ, q.ZZZ), PPP);
    return r;
}
// m p for m >= 1 (double-and-add from the top set bit)
template <typename F>
FPG_DEV xyzz_t<F> xyzz_mul_small(const xyzz_t<F>& p, uint32_t m) {
    xyzz_t<F> acc = p;
    for (int i = 30 - __clz(m); i >= 0; i--) {
        acc = xyzz_dbl(acc);
        if ((m >> i) & 1) acc = xyzz_add(acc, p);
    }
    return acc;
}

// affine point type, identity test and serialisation per group
template <typename F> struct Aff;
template <> struct Aff<fq> { using T = g1a; static constexpr size_t SER = G1_SER; };
template <> struct Aff<fq2> { using T = g2a; static constexpr size_t SER = G2_SER; };
FPG_DEV bool aff_is_inf(const g1a& p) { return g1a_is_inf(p); }
FPG_DEV bool aff_is_inf(const g2a& p) { return g2a_is_inf(p); }
FPG_DEV void aff_to_be(uint8_t* o, const g1a& p) { g1a_to_be(o, p); }
FPG_DEV void aff_to_be(uint8_t* o, const g2a& p) { g2a_to_be(o, p); }

// ---------------------------------------------------------------------------- digits
FPG_DEV uint32_t win_bits(const uint32_t* a, int nw, int lo, int c) {
    const int word = lo >> 5, bit = lo & 31;
    const uint64_t two = (uint64_t)(word < nw ? a[word] : 0) | ((uint64_t)(word + 1 < nw ? a[word + 1] : 0) << 32);
    return (uint32_t)(two >> bit) & ((1u << c) - 1);
}

// k mod r for a 256-bit k (k < 2^256 < 3 r)
FPG_DEV void reduce_mod_r(uint32_t* k) {
    for (int it = 0; it < 2; it++) {
        if (mp::lt<8>(k, FR_P)) return;
        uint32_t t[8];
        mp::mod_sub<8>(t, k, FR_P, FR_P);           // k >= r: no borrow, t = k - r
#pragma unroll
        for (int i = 0; i < 8; i++) k[i] = t[i];
    }
}

// signed digits of one part a (nw words) over the shape's windows: emit(window, digit) for each
// non-zero digit
template <typename Emit>
FPG_DEV void part_digits(const uint32_t* a, int nw, const MsmShape& sh, Emit&& emit) {
    int32_t carry = 0;
    for (int w = 0; w < sh.W; w++) {
        const int cw = sh.bits(w);
        int32_t d = (int32_t)win_bits(a, nw, sh.lo(w), cw) + carry;
        carry = d > (1 << (cw - 1));
        if (carry) d -= 1 << cw;
        if (d) emit(w, d);
    }
}

// emit(part, window, digit) for every non-zero signed digit of the endomorphism parts of k mod r:
// G1 (GLV): k = k0 + k1 |x|^2, parts below 2^128 (bases P, -phi(P));
// G2 (GLS): k = d0 + d1 |x| + d2 |x|^2 + d3 |x|^3, parts below 2^64 (bases (-1)^h psi^h(Q))
template <typename Emit>
FPG_DEV void msm_digits_glv(const fr& s, const MsmShape& sh, Emit&& emit) {
    uint32_t k[8], k1[5], k0[4];
#pragma unroll
    for (int i = 0; i < 8; i++) k[i] = s.v[i];
    reduce_mod_r(k);
    div_by_const<4, 5>(k1, k0, k, GLV_D, GLV_BARRETT);
    part_digits(k0, 4, sh, [&](int w, int32_t d) { emit(0, w, d); });
    part_digits(k1, 5, sh, [&](int w, int32_t d) { emit(1, w, d); });
}
template <typename Emit>
FPG_DEV void msm_digits_gls(const fr& s, const MsmShape& sh, Emit&& emit) {
    uint32_t k[8], q[7], d[2], t8[8];
#pragma unroll
    for (int i = 0; i < 8; i++) k[i] = s.v[i];
    reduce_mod_r(k);
    for (int h = 0; h < 3; h++) {
        div_by_const<2, 7>(q, d, k, GLS_D, GLS_BARRETT);
        part_digits(d, 2, sh, [&](int w, int32_t dd) { emit(h, w, dd); });
        for (int i = 0; i < 8; i++) t8[i] = i < 7 ? q[i] : 0;
        for (int i = 0; i < 8; i++) k[i] = t8[i];
    }
    part_digits(k, 2, sh, [&](int w, int32_t dd) { emit(3, w, dd); });
}

template <typename F>
__global__ void k_msm_count(const fr* k, MsmShape sh, uint32_t* counts) {
    const uint64_t t = gtid();
    if (t >= sh.n * sh.nbatch) return;
    const uint64_t base = (t / sh.n) * sh.KW;
    auto emit = [&](int, int w, int32_t d) {
        atomicAdd(&counts[base + sh.off(w) + (uint32_t)(d < 0 ? -d : d) - 1], 1u);
    };
    if constexpr (std::is_same<F, fq>::value) msm_digits_glv(k[t], sh, emit);
    else msm_digits_gls(k[t], sh, emit);
}

template <typename F>
__global__ void k_msm_scatter(const fr* k, MsmShape sh, uint32_t* cursor, uint32_t* list, uint32_t* keys) {
    const uint64_t t = gtid();
    if (t >= sh.n * sh.nbatch) return;
    const uint64_t base = (t / sh.n) * sh.KW;
    const uint32_t pidx = (uint32_t)(t % sh.npts);
    auto emit = [&](int h, int w, int32_t d) {
        const uint32_t key = (uint32_t)(base + sh.off(w) + (uint32_t)(d < 0 ? -d : d) - 1);
        const uint32_t pos = atomicAdd(&cursor[key], 1u);
        list[pos] = (pidx + (uint32_t)h * (uint32_t)sh.npts) | (d < 0 ? 0x80000000u : 0u);
        keys[pos] = key;
    };
    if constexpr (std::is_same<F, fq>::value) msm_digits_glv(k[t], sh, emit);
    else msm_digits_gls(k[t], sh, emit);
}

// ---------------------------------------------------------------------------- scan
// exclusive scan, one level: each block of 1024 scans its slice and reports its total
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* sums) {
    __shared__ uint32_t s[1024];
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    const uint32_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t add = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) sums[blockIdx.x] = s[1023];
}
__global__ void __launch_bounds__(1024) k_scan_add(uint32_t* out, uint64_t n, const uint32_t* block_prefix) {
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += block_prefix[blockIdx.x];
}

static size_t scan_tmp_words(uint64_t n) {
    size_t w = 0;
    while (n > 1) {
        n = (n + 1023) / 1024;
        w += 2 * n;
    }
    return w + 2;
}
// exclusive scan of n values; tmp holds scan_tmp_words(n) words
static void exclusive_scan(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp, cudaStream_t s) {
    const uint64_t nb = (n + 1023) / 1024;
    FP_KERNEL("k_scan_block", s, k_scan_block<<<(unsigned)nb, 1024, 0, s>>>(in, out, n, tmp));
    if (nb > 1) {
        exclusive_scan(tmp, tmp + nb, nb, tmp + 2 * nb, s);
        FP_KERNEL("k_scan_add", s, k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(out, n, tmp + nb));
    }
}

// ---------------------------------------------------------------------------- buckets
// Load-balanced bucket sums: the sorted entry list (E entries, E = end of the last key's run) is cut
// into chunks of T consecutive entries, one thread each.  A thread sums each run of equal keys in its
// chunk; a run that neither started in the previous chunk nor continues into the next is the whole
// bucket and is stored there; the partial sum of a chunk's first run, when that run started
// earlier, goes to head[c], and the partial of its last run, when it continues, to tail[c] (a
// chunk inside one run stores it in head[c]).  k_msm_fixup then completes those buckets.
// Buckets without entries stay the identity (zeroed by the caller).
template <typename F>
__global__ void __launch_bounds__(128) k_msm_chunk(const typename Aff<F>::T* pts, const uint32_t* list,
                                                   const uint32_t* keys, const uint32_t* offsets,
                                                   const uint32_t* counts, uint64_t nk, uint32_t T,
                                                   xyzz_t<F>* buckets, xyzz_t<F>* head, xyzz_t<F>* tail) {
    const uint64_t c = gtid();
    const uint64_t E = nk ? (uint64_t)offsets[nk - 1] + counts[nk - 1] : 0;
    const uint64_t lo = c * T;
    if (lo >= E) return;
    const uint64_t hi = lo + T < E ? lo + T : E;
    xyzz_t<F> acc;
    xyzz_inf(acc);
    uint64_t run0 = lo;
    for (uint64_t i = lo; i < hi; i++) {
        const uint32_t e = list[i];
        const typename Aff<F>::T p = pts[e & 0x7fffffffu];
        if (!aff_is_inf(p)) acc = xyzz_madd(acc, p.x, (e >> 31) ? f_neg(p.y) : p.y);
        const uint32_t k = keys[i];
        if (i + 1 == hi || keys[i + 1] != k) {                   // end of a run inside this chunk
            const bool before = run0 == lo && lo > 0 && keys[lo - 1] == k;
            const bool after = i + 1 == hi && hi < E && keys[hi] == k;
            if (before) head[c] = acc;
            else if (after) tail[c] = acc;
            else buckets[k] = acc;
            xyzz_inf(acc);
            run0 = i + 1;
        }
    }
}

// buckets whose run starts in chunk c and continues: tail[c] plus the head partials of the chunks
// that start inside the same run
template <typename F>
__global__ void k_msm_fixup(const uint32_t* keys, const uint32_t* offsets, const uint32_t* counts, uint64_t nk,
                            uint32_t T, const xyzz_t<F>* head, const xyzz_t<F>* tail, xyzz_t<F>* buckets) {
    const uint64_t c = gtid();
    const uint64_t E = nk ? (uint64_t)offsets[nk - 1] + counts[nk - 1] : 0;
    const uint64_t lo = c * T;
    if (lo >= E) return;
    const uint64_t hi = lo + T < E ? lo + T : E;
    if (hi >= E) return;
    const uint32_t k = keys[hi - 1];
    if (keys[hi] != k) return;                                   // the last run ends in this chunk
    // the run continues past chunk c; chunk c computes it only if it starts in chunk c
    const uint32_t start = offsets[k];
    if (start < lo) return;
    xyzz_t<F> acc = tail[c];
    for (uint64_t d = c + 1; d * T < E && keys[d * T] == k; d++) acc = xyzz_add(acc, head[d]);
    buckets[k] = acc;
}

// segment s of window w of batch j: its L = B_w / S buckets b in [s L, (s + 1) L) give
// sum_b (b + 1) B_b
template <typename F>
__global__ void __launch_bounds__(128) k_msm_segment(MsmShape sh, const xyzz_t<F>* buckets, xyzz_t<F>* segs) {
    const uint64_t t = gtid();
    if (t >= sh.nsegs()) return;
    const uint64_t j = t / ((uint64_t)sh.W * sh.S);
    const int w = (int)((t / sh.S) % sh.W);
    const uint32_t s = (uint32_t)(t % sh.S), L = sh.buckets(w) / sh.S;
    const xyzz_t<F>* bk = buckets + j * sh.KW + sh.off(w) + (uint64_t)s * L;
    xyzz_t<F> run, acc;
    xyzz_inf(run);
    xyzz_inf(acc);
    for (int b = (int)L - 1; b >= 0; b--) {
        run = xyzz_add(run, bk[b]);
        acc = xyzz_add(acc, run);                   // sum_b (b - s L + 1) B_b
    }
    if (s && !xyzz_is_inf(run)) acc = xyzz_add(acc, xyzz_mul_small(run, s * L));
    segs[t] = acc;
}

template <typename F>
__global__ void k_msm_pair(const xyzz_t<F>* in, xyzz_t<F>* out, uint64_t n) {
    const uint64_t i = gtid();
    if (i < n) out[i] = xyzz_add(in[2 * i], in[2 * i + 1]);
}

// window sums to homogeneous projective (X ZZZ : Y ZZ : ZZ ZZZ), identity (0 : 1 : 0)
template <typename F>
__global__ void k_msm_to_proj(const xyzz_t<F>* in, GPt<F>* out, uint64_t n) {
    const uint64_t i = gtid();
    if (i >= n) return;
    const xyzz_t<F> p = in[i];
    GPt<F> r;
    if (xyzz_is_inf(p)) {
        r = gec_identity<F>();
    } else {
        r.X = f_mul(p.X, p.ZZZ);
        r.Y = f_mul(p.Y, p.ZZ);
        r.Z = f_mul(p.ZZ, p.ZZZ);
    }
    out[i] = r;
}

// per batch, on 8 lanes: sum_w 2^(lo_w) S_w by Horner from the top window, then affine; the
// serialised result of batch j goes to ser + j ser_stride
template <typename F>
__global__ void __launch_bounds__(64) k_msm_final(MsmShape sh, const GPt<F>* win, typename Aff<F>::T* out, uint8_t* ser,
                                                  size_t ser_stride) {
    __shared__ GEc<F> sm[8];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t j0 = (uint64_t)blockIdx.x * 8 + grp;
    const bool valid = j0 < sh.nbatch;
    const uint64_t j = valid ? j0 : 0;                // idle groups repeat batch 0's work
    GPt<F> acc = win[j * sh.W + sh.W - 1];
    for (int w = sh.W - 2; w >= 0; w--) {
        for (int q = 0; q < sh.bits(w); q++) acc = gec_dbl(sm[grp], lane, acc);
        acc = gec_add(sm[grp], lane, acc, win[j * sh.W + w]);
    }
    typename Aff<F>::T a;
    gec_to_affine(a.x, a.y, acc);
    if (valid && lane == 0) {
        if (out) out[j] = a;
        if (ser) aff_to_be(ser + j * ser_stride, a);
    }
}

// ---------------------------------------------------------------------------- bases
// first half of the bases table from serialised affine points; err |= 1 for a point that is not
// canonical, not on y^2 = x^3 + 4 or not in the order-r subgroup (all-zero bytes = identity)
__global__ void k_bases_load(const uint8_t* be, uint64_t n, g1a* tab, uint32_t* err) {
    const uint64_t i = gtid();
    if (i >= n) return;
    const uint8_t* p = be + i * G1_SER;
    fq c[2];
    bool zero = true;
    for (int h = 0; h < 2; h++) {
        for (int w = 0; w < 12; w++) {
            const uint8_t* q = p + h * 48 + (11 - w) * 4;
            c[h].v[w] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
            zero = zero && c[h].v[w] == 0;
        }
    }
    g1a a;
    fq_zero(a.x);
    fq_zero(a.y);
    if (!zero) {
        if (!mp::lt<12>(c[0].v, FQ_P) || !mp::lt<12>(c[1].v, FQ_P)) {
            atomicOr(err, 1u);
        } else {
            a.x = fq_to_mont(c[0]);
            a.y = fq_to_mont(c[1]);
            fq four;
            fq_one(four);
            four = fq_dbl(fq_dbl(four));
            if (!fq_eq(fq_sqr(a.y), fq_add(fq_mul(fq_sqr(a.x), a.x), four))) {
                atomicOr(err, 1u);
            } else {
                // subgroup: [r] P must be the identity (plain double-and-add, no endomorphism)
                g1j acc;
                jac_set_inf(acc);
                for (int i = 254; i >= 0; i--) {
                    acc = jac_dbl(acc);
                    if ((FR_P[i >> 5] >> (i & 31)) & 1) acc = jac_madd(acc, a.x, a.y);
                }
                if (!jac_is_inf(acc)) atomicOr(err, 1u);
            }
        }
    }
    tab[i] = a;
}

// second half of the table: -phi(P) = (omega x, -y)
__global__ void k_bases_endo(g1a* tab, uint64_t n) {
    const uint64_t i = gtid();
    if (i >= n) return;
    fq om;
    fq_from_const(om, GLV_OMEGA);
    const g1a p = tab[i];
    tab[n + i] = g1a_is_inf(p) ? p : g1a{fq_mul(p.x, om), fq_neg(p.y)};
}

void msm_bases_load(const void* be96, uint64_t n, void* tab, uint32_t* err, cudaStream_t s) {
    if (!n) return;
    FP_KERNEL("k_bases_load", s, k_bases_load<<<grid_for(n, 128), 128, 0, s>>>((const uint8_t*)be96, n, (g1a*)tab,
                                                                              err));
    FP_KERNEL("k_bases_endo", s, k_bases_endo<<<grid_for(n, 128), 128, 0, s>>>((g1a*)tab, n));
}
void msm_bases_endo(void* tab, uint64_t n, cudaStream_t s) {
    if (n) FP_KERNEL("k_bases_endo", s, k_bases_endo<<<grid_for(n, 128), 128, 0, s>>>((g1a*)tab, n));
}

// G2 bases table for the GLS parts: tab[h n + i] = (-1)^h psi^h(Q_i) for h < 4; entries i >= nvalid
// are the identity (padding)
__global__ void k_bases_g2(const g2a* pts, uint64_t nvalid, uint64_t n, g2a* tab) {
    const uint64_t i = gtid();
    if (i >= n) return;
    g2a b;
    fq2_zero(b.x);
    fq2_zero(b.y);
    if (i < nvalid) b = pts[i];
    const bool inf = g2a_is_inf(b);
    for (int h = 0; h < 4; h++) {
        if (h && !inf) b = g2_psi(b);
        g2a o = b;
        if ((h & 1) && !inf) o.y = fq2_neg(o.y);
        tab[h * n + i] = o;
    }
}
void msm_bases_g2(const void* pts, uint64_t nvalid, uint64_t n, void* tab, cudaStream_t s) {
    if (n) FP_KERNEL("k_bases_g2", s, k_bases_g2<<<grid_for(n, 128), 128, 0, s>>>((const g2a*)pts, nvalid, n,
                                                                                 (g2a*)tab));
}

// ---------------------------------------------------------------------------- shape and driver
MsmShape msm_shape(uint64_t n, uint32_t nbatch, uint64_t npts, int c, int parts, int part_bits) {
    MsmShape sh;
    sh.n = n;
    sh.nbatch = nbatch;
    sh.npts = npts;
    sh.H = parts;
    sh.W = (part_bits + c - 1) / c;
    sh.c = (part_bits + sh.W - 1) / sh.W;              // balanced widths: c or c - 1
    sh.n_hi = part_bits - sh.W * (sh.c - 1);
    sh.KW = sh.off(sh.W);
    // segments of at least 4 buckets in the narrowest window, at most about 2^15 segment threads
    // at most about lim.msm_segment_threads segment threads; entries per chunk of the bucket pass
    // so that there are about lim.msm_chunks chunks (enough to fill the GPU a few times over), >= 8
    const EngineLimits lim = engine_limits();
    const uint64_t seg_cap = lim.msm_segment_threads ? lim.msm_segment_threads : 1;
    uint32_t S = sh.buckets(sh.W - 1);
    while (S > 1 && sh.buckets(sh.W - 1) / S < 4) S >>= 1;
    while (S > 1 && (uint64_t)nbatch * sh.W * S > seg_cap) S >>= 1;
    sh.S = S;
    const uint64_t chunks = lim.msm_chunks ? lim.msm_chunks : 1;
    const uint64_t T = (sh.entries_max() + chunks - 1) / chunks;
    sh.T = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(T, 8), 1u << 30);
    return sh;
}

template <typename F>
static size_t scratch_bytes(const MsmShape& sh) {
    const uint64_t nk = sh.nkeys();
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const uint64_t nchunks = (sh.entries_max() + sh.T - 1) / sh.T;
    size_t b = 3 * r(nk * 4) + r(scan_tmp_words(nk) * 4);
    b += 2 * r(sh.entries_max() * 4);
    b += r(nk * sizeof(xyzz_t<F>));
    b += 2 * r(nchunks * sizeof(xyzz_t<F>));
    b += 2 * r(sh.nsegs() * sizeof(xyzz_t<F>));
    b += r((uint64_t)sh.nbatch * sh.W * sizeof(GPt<F>));
    return b;
}
size_t msm_scratch_bytes(const MsmShape& sh) { return scratch_bytes<fq>(sh); }
size_t msm_scratch_bytes_g2(const MsmShape& sh) { return scratch_bytes<fq2>(sh); }

// Window size from a cost model: per phase the larger of the throughput time (about 1.9e10 Fq
// products/s over the GPU) and the latency of one thread's dependent chain (about 2.7 us per
// product); mixed addition 10 field products, addition 14, group doubling/addition about
// 2 x 1.5 (fmul = Fq products per field product: 1 on G1, 3 on G2).
int msm_window_model(uint64_t n, uint32_t nbatch, int parts, int part_bits, double fmul) {
    const double tp = fmul / 1.9e10, lat = fmul * 2.7e-6;
    int best = 8;
    double bestt = 1e300;
    for (int c = 4; c <= 16; c++) {
        const MsmShape sh = msm_shape(n, nbatch, n, c, parts, part_bits);
        if (sh.c != c || sh.nkeys() > (1ull << 28) || sh.entries_max() > 0xffffffffull) continue;
        const double entries = (double)parts * n * nbatch * sh.W;
        const double per_bucket = entries / (double)sh.nkeys();
        const double t_bucket = std::max(entries * 10 * tp, per_bucket * 10 * lat);
        const double L = (double)(sh.buckets(0) / sh.S);
        const double t_seg = std::max((double)sh.nkeys() * 2 * 14 * tp, (2 * L + 1.5 * (c - 1)) * 14 * lat);
        const double t_pair = std::log2((double)sh.S) * 14 * lat;
        const double t_final = (double)part_bits * 2 * 1.5 * lat;
        const double t = t_bucket + t_seg + t_pair + t_final;
        if (t < bestt) {
            bestt = t;
            best = c;
        }
    }
    return best;
}

template <typename F>
static void msm_run(const void* bases, const void* k_canon, const MsmShape& sh, void* scratch, void* out_aff,
                    void* ser_out, size_t ser_stride, cudaStream_t s) {
    using X = xyzz_t<F>;
    constexpr bool g2 = std::is_same<F, fq2>::value;     // launch names: G2 launches end in _g2
    const uint64_t nk = sh.nkeys(), nseg = sh.nsegs(), nwin = (uint64_t)sh.nbatch * sh.W;
    uint8_t* p = (uint8_t*)scratch;
    auto take = [&](size_t bytes) {
        uint8_t* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    uint32_t* counts = (uint32_t*)take(nk * 4);
    uint32_t* offsets = (uint32_t*)take(nk * 4);
    uint32_t* cursor = (uint32_t*)take(nk * 4);
    uint32_t* scan_tmp = (uint32_t*)take(scan_tmp_words(nk) * 4);
    uint32_t* list = (uint32_t*)take(sh.entries_max() * 4);
    uint32_t* keys = (uint32_t*)take(sh.entries_max() * 4);
    const uint32_t T = sh.T;
    const uint64_t nchunks = (sh.entries_max() + T - 1) / T;
    X* buckets = (X*)take(nk * sizeof(X));
    X* head = (X*)take(nchunks * sizeof(X));
    X* tail = (X*)take(nchunks * sizeof(X));
    X* seg_a = (X*)take(nseg * sizeof(X));
    X* seg_b = (X*)take(nseg * sizeof(X));
    GPt<F>* proj = (GPt<F>*)take(nwin * sizeof(GPt<F>));
    const uint64_t terms = sh.n * sh.nbatch;
    cudaMemsetAsync(counts, 0, nk * 4, s);
    if (terms) {
        FP_KERNEL(g2 ? "k_msm_count_g2" : "k_msm_count", s,
                  k_msm_count<F><<<grid_for(terms, 128), 128, 0, s>>>((const fr*)k_canon, sh, counts));
    }
    exclusive_scan(counts, offsets, nk, scan_tmp, s);
    cudaMemcpyAsync(cursor, offsets, nk * 4, cudaMemcpyDeviceToDevice, s);
    if (terms) {
        FP_KERNEL(g2 ? "k_msm_scatter_g2" : "k_msm_scatter", s,
                  k_msm_scatter<F><<<grid_for(terms, 128), 128, 0, s>>>((const fr*)k_canon, sh, cursor, list, keys));
    }
    cudaMemsetAsync(buckets, 0, nk * sizeof(X), s);
    if (nchunks) {                                   // no terms: every bucket stays the identity
        FP_KERNEL(g2 ? "k_msm_chunk_g2" : "k_msm_chunk", s,
                  k_msm_chunk<F><<<grid_for(nchunks, 128), 128, 0, s>>>((const typename Aff<F>::T*)bases, list, keys,
                                                                       offsets, counts, nk, T, buckets, head, tail));
        FP_KERNEL(g2 ? "k_msm_fixup_g2" : "k_msm_fixup", s,
                  k_msm_fixup<F><<<grid_for(nchunks, 128), 128, 0, s>>>(keys, offsets, counts, nk, T, head, tail,
                                                                       buckets));
    }
    FP_KERNEL(g2 ? "k_msm_segment_g2" : "k_msm_segment", s, k_msm_segment<F><<<grid_for(nseg, 128), 128, 0, s>>>(sh, buckets, seg_a));
    X* a = seg_a;
    X* b = seg_b;
    for (uint64_t m = nseg; m > nwin; m /= 2) {
        FP_KERNEL(g2 ? "k_msm_pair_g2" : "k_msm_pair", s, k_msm_pair<F><<<grid_for(m / 2, 128), 128, 0, s>>>(a, b, m / 2));
        std::swap(a, b);
    }
    FP_KERNEL(g2 ? "k_msm_to_proj_g2" : "k_msm_to_proj", s, k_msm_to_proj<F><<<grid_for(nwin, 128), 128, 0, s>>>(a, proj, nwin));
    FP_KERNEL(g2 ? "k_msm_final_g2" : "k_msm_final", s,
              k_msm_final<F><<<grid_for(sh.nbatch, 8), 64, 0, s>>>(sh, proj, (typename Aff<F>::T*)out_aff,
                                                                  (uint8_t*)ser_out, ser_stride));
}

void msm_g1(const void* bases, const void* k_canon, const MsmShape& sh, void* scratch, void* out_g1a, void* ser_out,
            cudaStream_t s) {
    msm_run<fq>(bases, k_canon, sh, scratch, out_g1a, ser_out, G1_SER, s);
}
void msm_g2(const void* bases, const void* k_canon, const MsmShape& sh, void* scratch, void* out_g2a, void* ser_out,
            size_t ser_stride, cudaStream_t s) {
    msm_run<fq2>(bases, k_canon, sh, scratch, out_g2a, ser_out, ser_stride, s);
}

}  // namespace fpk
