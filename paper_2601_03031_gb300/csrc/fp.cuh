// Prime-field arithmetic for the BLS12-381 base field Fq (12 x 32-bit limbs) and scalar field
// Fr (8 x 32-bit limbs), Montgomery form with R = 2^(32 N), little-endian limbs.
//
// Every multiply is a CIOS Montgomery product written as explicit PTX carry chains
// (mad.lo/hi.cc, madc.lo/hi.cc, addc): per outer step one low-half chain and one high-half
// chain for a*b_i, then the same two chains for m*p with m = t_0 * (-p^-1 mod 2^32).  The
// integer multiply-add pipe executes all of it; there is no floating point anywhere.
#pragma once
#include <cstdint>

#include "constants.cuh"

#ifndef FPG_PRIMITIVES_EXTERNAL
#define FPG_DEV __device__ __forceinline__
#define FPG_NOINL static __device__ __noinline__

namespace ptx {
FPG_DEV uint32_t add_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t addc_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t addc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t sub_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t subc_cc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t subc(uint32_t a, uint32_t b) { uint32_t r; asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b)); return r; }
FPG_DEV uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("mad.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
FPG_DEV uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("madc.lo.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
FPG_DEV uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("mad.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
FPG_DEV uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; asm volatile("madc.hi.cc.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c)); return r; }
}  // namespace ptx
#endif

struct fq { uint32_t v[12]; };
struct fr { uint32_t v[8]; };

namespace mp {

// r = a * b * 2^(-32 N) mod P, for a, b < P and 4P < 2^(32 N).
template <int N>
FPG_DEV void mont_mul(uint32_t* r, const uint32_t* a, const uint32_t* b, const uint32_t* P, uint32_t pinv) {
    uint32_t t[N + 2];
#pragma unroll
    for (int j = 0; j < N + 2; j++) t[j] = 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const uint32_t bi = b[i];
        t[0] = ptx::mad_lo_cc(a[0], bi, t[0]);
#pragma unroll
        for (int j = 1; j < N; j++) t[j] = ptx::madc_lo_cc(a[j], bi, t[j]);
        t[N] = ptx::addc_cc(t[N], 0);
        t[N + 1] = ptx::addc(t[N + 1], 0);
        t[1] = ptx::mad_hi_cc(a[0], bi, t[1]);
#pragma unroll
        for (int j = 1; j < N; j++) t[j + 1] = ptx::madc_hi_cc(a[j], bi, t[j + 1]);
        t[N + 1] = ptx::addc(t[N + 1], 0);
        const uint32_t m = t[0] * pinv;
        t[0] = ptx::mad_lo_cc(m, P[0], t[0]);
#pragma unroll
        for (int j = 1; j < N; j++) t[j] = ptx::madc_lo_cc(m, P[j], t[j]);
        t[N] = ptx::addc_cc(t[N], 0);
        t[N + 1] = ptx::addc(t[N + 1], 0);
        t[1] = ptx::mad_hi_cc(m, P[0], t[1]);
#pragma unroll
        for (int j = 1; j < N; j++) t[j + 1] = ptx::madc_hi_cc(m, P[j], t[j + 1]);
        t[N + 1] = ptx::addc(t[N + 1], 0);
#pragma unroll
        for (int j = 0; j <= N; j++) t[j] = t[j + 1];
        t[N + 1] = 0;
    }
    uint32_t s[N];
    s[0] = ptx::sub_cc(t[0], P[0]);
#pragma unroll
    for (int j = 1; j < N; j++) s[j] = ptx::subc_cc(t[j], P[j]);
    const uint32_t borrow = ptx::subc(t[N], 0);     // all-ones when t < P
#pragma unroll
    for (int j = 0; j < N; j++) r[j] = borrow ? t[j] : s[j];
}

// r = a + b mod P (a + b < 2^(32 N) because P < 2^(32 N - 1))
template <int N>
FPG_DEV void mod_add(uint32_t* r, const uint32_t* a, const uint32_t* b, const uint32_t* P) {
    uint32_t t[N], s[N];
    t[0] = ptx::add_cc(a[0], b[0]);
#pragma unroll
    for (int j = 1; j < N; j++) t[j] = ptx::addc_cc(a[j], b[j]);
    s[0] = ptx::sub_cc(t[0], P[0]);
#pragma unroll
    for (int j = 1; j < N; j++) s[j] = ptx::subc_cc(t[j], P[j]);
    const uint32_t borrow = ptx::subc(0, 0);
#pragma unroll
    for (int j = 0; j < N; j++) r[j] = borrow ? t[j] : s[j];
}

template <int N>
FPG_DEV void mod_sub(uint32_t* r, const uint32_t* a, const uint32_t* b, const uint32_t* P) {
    uint32_t t[N], s[N];
    t[0] = ptx::sub_cc(a[0], b[0]);
#pragma unroll
    for (int j = 1; j < N; j++) t[j] = ptx::subc_cc(a[j], b[j]);
    const uint32_t borrow = ptx::subc(0, 0);
    s[0] = ptx::add_cc(t[0], P[0]);
#pragma unroll
    for (int j = 1; j < N; j++) s[j] = ptx::addc_cc(t[j], P[j]);
#pragma unroll
    for (int j = 0; j < N; j++) r[j] = borrow ? s[j] : t[j];
}

template <int N>
FPG_DEV bool is_zero(const uint32_t* a) {
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < N; j++) acc |= a[j];
    return acc == 0;
}

template <int N>
FPG_DEV bool eq(const uint32_t* a, const uint32_t* b) {
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < N; j++) acc |= a[j] ^ b[j];
    return acc == 0;
}

// canonical a < P ?
template <int N>
FPG_DEV bool lt(const uint32_t* a, const uint32_t* P) {
    uint32_t s = ptx::sub_cc(a[0], P[0]);
#pragma unroll
    for (int j = 1; j < N; j++) s = ptx::subc_cc(a[j], P[j]);
    (void)s;
    return ptx::subc(0, 0) != 0;
}

// Plain modular inverse of x (0 < x < P, P odd) by batched division steps (the divstep iteration of
// Bernstein and Yang, "Fast constant-time gcd computation and modular inversion", 2019, run in its
// variable-time form: the values inverted here are public).  State: integers f (odd) and g with
// f = d x and g = e x (mod P), from f = P, g = x, d = 0, e = 1.  One division step, by delta and the
// parity of g: if delta > 0 and g is odd, (f, g) <- (g, (g - f) / 2) and delta <- 1 - delta; else if g
// is odd, g <- (g + f) / 2; else g <- g / 2; delta <- delta + 1 in the last two cases.  Thirty steps
// depend only on the low 32 bits of f and g, so they run on one word each and yield a matrix
// [[u, v], [q, r]] (|u| + |v|, |q| + |r| <= 2^30) with 2^30 (f', g') = (u f + v g, q f + r g); the
// full-width f, g and the residues d, e (times 2^-30 mod P, by adding the multiple of P that clears
// the low 30 bits) are then updated once per batch.  When g = 0, f = +-1 = gcd and x^-1 = +-d.
// Returns 0 for x = 0.  pinv = -P^-1 mod 2^32.
template <int N>
FPG_DEV void ds_lincomb(uint32_t* out, int32_t a, const uint32_t* x, int32_t b, const uint32_t* y) {
    // out (N + 2 words, two's complement) = a x + b y for signed N + 1 word x, y
    int64_t carry = 0;
#pragma unroll
    for (int i = 0; i <= N; i++) {
        const int64_t xi = i < N ? (int64_t)x[i] : (int64_t)(int32_t)x[i];
        const int64_t yi = i < N ? (int64_t)y[i] : (int64_t)(int32_t)y[i];
        const int64_t t = (int64_t)a * xi + (int64_t)b * yi + carry;
        out[i] = (uint32_t)t;
        carry = t >> 32;
    }
    out[N + 1] = (uint32_t)carry;
}
// arithmetic right shift by 30 of an N + 2 word two's complement value into N + 1 words
template <int N>
FPG_DEV void ds_shr30(uint32_t* out, const uint32_t* t) {
#pragma unroll
    for (int i = 0; i <= N; i++) out[i] = (t[i] >> 30) | (t[i + 1] << 2);
}
template <int N>
FPG_DEV bool ds_is_neg(const uint32_t* a) { return (int32_t)a[N] < 0; }

// thirty division steps on the low words fl, gl of f and g (delta updated), without branches.  With
// s = all-ones for a swap (delta > 0 and g odd) and o = all-ones for g odd, one step is
//   g <- g + ((f & o) ^ s) - s    (g - f on a swap, g + f for g odd, g otherwise)
//   f <- f + (g & s)              (on a swap the old g), then g <- g / 2,
// the same on the matrix (q <- q + ((u & o) ^ s) - s, u <- 2 (u + (q & s)), likewise v, w) and
// nd = -delta <- (nd ^ s) - s - 1 (1 - delta on a swap, 1 + delta otherwise).  The dependent chain
// from one step's g to the next is four operations.  Returns the batch's matrix:
// 2^30 (f', g') = (u f + v g, q f + w g).
FPG_DEV void ds_batch30(uint32_t fl, uint32_t gl, int32_t& delta, int32_t& u, int32_t& v, int32_t& q,
                        int32_t& w) {
    uint32_t f = fl, g = gl, nd = 0u - (uint32_t)delta;
    uint32_t uu = 1, vv = 0, qq = 0, ww = 1;
#pragma unroll 6
    for (int i = 0; i < 30; i++) {
        const uint32_t o = 0u - (g & 1u);
        const uint32_t sw = o & (uint32_t)((int32_t)nd >> 31);
        g = g + ((f & o) ^ sw) - sw;
        f += g & sw;
        g >>= 1;
        qq = qq + ((uu & o) ^ sw) - sw;
        ww = ww + ((vv & o) ^ sw) - sw;
        uu = (uu + (qq & sw)) << 1;
        vv = (vv + (ww & sw)) << 1;
        nd = (nd ^ sw) - sw - 1u;
    }
    delta = (int32_t)(0u - nd);
    u = (int32_t)uu;
    v = (int32_t)vv;
    q = (int32_t)qq;
    w = (int32_t)ww;
}

// r = +-d (minus when fneg) normalised into [0, P), for d in (-P, P) (N + 1 word two's complement)
template <int N>
FPG_DEV void ds_finish(uint32_t* r, uint32_t* d, bool fneg, const uint32_t* P) {
    if (fneg) {                                              // d <- -d
        uint32_t z[N + 1];
        uint32_t bw = 0;
#pragma unroll
        for (int j = 0; j <= N; j++) {
            const uint64_t s = (uint64_t)0 - d[j] - bw;
            z[j] = (uint32_t)s;
            bw = (uint32_t)(s >> 63);
        }
#pragma unroll
        for (int j = 0; j <= N; j++) d[j] = z[j];
    }
    // d in (-P, P): add P when negative (the loops are bounds, one pass suffices)
    for (int it = 0; it < 4 && ds_is_neg<N>(d); it++) {
        uint64_t c = 0;
#pragma unroll
        for (int j = 0; j <= N; j++) {
            const uint64_t s = (uint64_t)d[j] + (j < N ? P[j] : 0) + c;
            d[j] = (uint32_t)s;
            c = s >> 32;
        }
    }
    for (int it = 0; it < 4; it++) {
        uint32_t z[N + 1];
        uint64_t bw = 0;
#pragma unroll
        for (int j = 0; j <= N; j++) {
            const uint64_t s = (uint64_t)d[j] - (j < N ? P[j] : 0) - bw;
            z[j] = (uint32_t)s;
            bw = (s >> 63) & 1;
        }
        if (bw) break;                                       // d < P
#pragma unroll
        for (int j = 0; j <= N; j++) d[j] = z[j];
    }
#pragma unroll
    for (int j = 0; j < N; j++) r[j] = d[j];
}

template <int N>
FPG_DEV void inv_ds(uint32_t* r, const uint32_t* x, const uint32_t* P, uint32_t pinv) {
    uint32_t f[N + 1], g[N + 1], d[N + 1], e[N + 1];
#pragma unroll
    for (int j = 0; j < N; j++) { f[j] = P[j]; g[j] = x[j]; d[j] = 0; e[j] = 0; }
    f[N] = g[N] = d[N] = e[N] = 0;
    e[0] = 1;
    if (is_zero<N>(x)) {
#pragma unroll
        for (int j = 0; j < N; j++) r[j] = 0;
        return;
    }
    int32_t delta = 1;
    const uint32_t mask30 = (1u << 30) - 1;
    // d, e <- (a d + b e) 2^-30 mod P, kept in (-P, P) as N + 1 word two's complement
    auto mod_update = [&](uint32_t* out, int32_t a, int32_t b) {
        uint32_t t[N + 2];
        ds_lincomb<N>(t, a, d, b, e);
        const uint32_t k = (t[0] * pinv) & mask30;        // t + k P = 0 mod 2^30
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < N + 2; i++) {
            const uint64_t s = (uint64_t)t[i] + (i < N ? (uint64_t)k * P[i] : 0) + c;
            t[i] = (uint32_t)s;
            c = s >> 32;
        }
        ds_shr30<N>(out, t);
        // out in (-P, 2P) for d, e in (-P, P): subtract P once if out >= P, back into (-P, P)
        if (!ds_is_neg<N>(out)) {
            uint32_t z[N + 1];
            uint64_t bw = 0;
#pragma unroll
            for (int j = 0; j <= N; j++) {
                const uint64_t s = (uint64_t)out[j] - (j < N ? P[j] : 0) - bw;
                z[j] = (uint32_t)s;
                bw = (s >> 63) & 1;
            }
            if (!bw) {
#pragma unroll
                for (int j = 0; j <= N; j++) out[j] = z[j];
            }
        }
    };
    // at most 2 x 32 N divsteps for P < 2^(32 N); the guard only bounds the loop on bad input
    for (int batch = 0; batch < 4 * 32 * N / 30 + 4; batch++) {
        if (is_zero<N + 1>(g)) break;
        int32_t u, v, q, w;
        ds_batch30(f[0], g[0], delta, u, v, q, w);
        uint32_t t[N + 2], nf[N + 1], ng[N + 1], nd[N + 1], ne[N + 1];
        ds_lincomb<N>(t, u, f, v, g);
        ds_shr30<N>(nf, t);
        ds_lincomb<N>(t, q, f, w, g);
        ds_shr30<N>(ng, t);
        mod_update(nd, u, v);
        mod_update(ne, q, w);
#pragma unroll
        for (int j = 0; j <= N; j++) { f[j] = nf[j]; g[j] = ng[j]; d[j] = nd[j]; e[j] = ne[j]; }
    }
    ds_finish<N>(r, d, ds_is_neg<N>(f), P);
}

// The same inverse computed by the four lanes of a quad (lanes 4m .. 4m + 3 of one warp, all four
// calling converged).  Lane q keeps one state value (q = 0: f, 1: g, 2: d, 3: e) and lanes q and
// q ^ 1 hold a pair, so a batch is the thirty division steps (every lane runs them on the broadcast
// low words of f and g), an exchange of the pair's values and one update per lane instead of four
// updates on one lane.  x is taken from the quad's first lane, so the four lanes agree on every
// branch; every lane returns the inverse.
template <int N>
FPG_DEV void inv_ds_quad(uint32_t* r, const uint32_t* x_in, const uint32_t* P, uint32_t pinv) {
    const int lane = (int)(threadIdx.x & 31), base = lane & 28, qd = lane & 3;
    const unsigned qmask = 0xfu << base;
    uint32_t x[N];
#pragma unroll
    for (int j = 0; j < N; j++) x[j] = __shfl_sync(qmask, x_in[j], base);
    if (is_zero<N>(x)) {
#pragma unroll
        for (int j = 0; j < N; j++) r[j] = 0;
        return;
    }
    uint32_t s[N + 1];                                       // this lane's value: f = P, g = x, d = 0, e = 1
#pragma unroll
    for (int j = 0; j < N; j++) s[j] = qd == 0 ? P[j] : qd == 1 ? x[j] : (qd == 3 && j == 0) ? 1u : 0u;
    s[N] = 0;
    const bool second = (qd & 1) != 0;                       // g or e: the second value of its pair
    const uint32_t modm = qd >= 2 ? 0xffffffffu : 0u;        // d and e are residues mod P
    const uint32_t mask30 = (1u << 30) - 1;
    int32_t delta = 1;
    for (int batch = 0; batch < 4 * 32 * N / 30 + 4; batch++) {
        const uint32_t fl = __shfl_sync(qmask, s[0], base);
        const uint32_t gl = __shfl_sync(qmask, s[0], base + 1);
        const int gz = __shfl_sync(qmask, (int)is_zero<N + 1>(s), base + 1);
        if (gz) break;
        int32_t u, v, q, w;
        ds_batch30(fl, gl, delta, u, v, q, w);
        uint32_t X[N + 1], Y[N + 1];                         // the pair (f, g) or (d, e)
#pragma unroll
        for (int j = 0; j <= N; j++) {
            const uint32_t o = __shfl_xor_sync(qmask, s[j], 1);
            X[j] = second ? o : s[j];
            Y[j] = second ? s[j] : o;
        }
        // f' = (u f + v g) / 2^30, g' = (q f + w g) / 2^30; d', e' the same times 2^-30 mod P: the
        // multiple k P that clears the low 30 bits is added on the residue lanes only
        uint32_t t[N + 2];
        ds_lincomb<N>(t, second ? q : u, X, second ? w : v, Y);
        const uint32_t k = (t[0] * pinv) & mask30 & modm;
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < N + 2; i++) {
            const uint64_t a = (uint64_t)t[i] + (i < N ? (uint64_t)k * P[i] : 0) + c;
            t[i] = (uint32_t)a;
            c = a >> 32;
        }
        ds_shr30<N>(s, t);
        // residues: from (-P, 2P) back into (-P, P) by subtracting P when s >= P
        uint32_t z[N + 1];
        uint64_t bw = 0;
#pragma unroll
        for (int j = 0; j <= N; j++) {
            const uint64_t a = (uint64_t)s[j] - (j < N ? P[j] : 0) - bw;
            z[j] = (uint32_t)a;
            bw = (a >> 63) & 1;
        }
        const uint32_t take = modm & ~(0u - (uint32_t)ds_is_neg<N>(s)) & ((uint32_t)bw - 1u);
#pragma unroll
        for (int j = 0; j <= N; j++) s[j] = (z[j] & take) | (s[j] & ~take);
    }
    // f = +-1 (lane 0) and d (lane 2): x^-1 = +-d
    const bool fneg = __shfl_sync(qmask, (int)ds_is_neg<N>(s), base) != 0;
    uint32_t d[N + 1];
#pragma unroll
    for (int j = 0; j <= N; j++) d[j] = __shfl_sync(qmask, s[j], base + 2);
    ds_finish<N>(r, d, fneg, P);
}

}  // namespace mp

// ---------------------------------------------------------------------------------------
// Fq
// ---------------------------------------------------------------------------------------
FPG_DEV void fq_zero(fq& a) {
#pragma unroll
    for (int j = 0; j < 12; j++) a.v[j] = 0;
}
FPG_DEV void fq_one(fq& a) {
#pragma unroll
    for (int j = 0; j < 12; j++) a.v[j] = FQ_ONE[j];
}
FPG_DEV void fq_from_const(fq& a, const uint32_t* c) {
#pragma unroll
    for (int j = 0; j < 12; j++) a.v[j] = c[j];
}
// The Montgomery products are out of line: one copy of the ~700-instruction body per translation
// unit instead of one per call site.  Inlined, a group operation's dozen products overflow the
// instruction cache and every product runs about three times slower; the call costs a few moves
// (arguments and result travel in registers).
static __device__ __noinline__ fq fq_mul_ool(fq a, fq b) {
    fq r;
    mp::mont_mul<12>(r.v, a.v, b.v, FQ_P, FQ_PINV);
    return r;
}
FPG_DEV fq fq_mul(const fq& a, const fq& b) { return fq_mul_ool(a, b); }
FPG_DEV fq fq_sqr(const fq& a) { return fq_mul(a, a); }
FPG_DEV fq fq_add(const fq& a, const fq& b) { fq r; mp::mod_add<12>(r.v, a.v, b.v, FQ_P); return r; }
FPG_DEV fq fq_sub(const fq& a, const fq& b) { fq r; mp::mod_sub<12>(r.v, a.v, b.v, FQ_P); return r; }
FPG_DEV fq fq_dbl(const fq& a) { return fq_add(a, a); }
// c ? a : b by per-limb masks.  The lane-parallel engines form every operand this way: lanes of one
// warp that chose between whole field elements by a branch would take divergent paths, which the
// warp runs one after another.
FPG_DEV fq fq_select(bool c, const fq& a, const fq& b) {
    const uint32_t m = 0u - (uint32_t)c;
    fq r;
#pragma unroll
    for (int j = 0; j < 12; j++) r.v[j] = (a.v[j] & m) | (b.v[j] & ~m);
    return r;
}
FPG_DEV fq fq_neg(const fq& a) { fq z; fq_zero(z); return fq_sub(z, a); }
FPG_DEV bool fq_is_zero(const fq& a) { return mp::is_zero<12>(a.v); }
FPG_DEV bool fq_eq(const fq& a, const fq& b) { return mp::eq<12>(a.v, b.v); }
FPG_DEV fq fq_to_mont(const fq& a) { fq r2; fq_from_const(r2, FQ_R2); return fq_mul(a, r2); }
FPG_DEV fq fq_from_mont(const fq& a) {
    fq one; fq_zero(one); one.v[0] = 1;
    return fq_mul(a, one);
}
// Inverse of a Montgomery residue aR: the plain inverse (aR)^-1 by batched division steps, then one
// Montgomery product with R^3 gives a^-1 R.  0 maps to 0.
FPG_NOINL fq fq_inv(const fq& a) {
    fq t, r3;
    mp::inv_ds<12>(t.v, a.v, FQ_P, FQ_PINV);
    fq_from_const(r3, FQ_R3);
    return fq_mul(t, r3);
}
// the same on the four lanes of a quad (mp::inv_ds_quad: all four call converged; the value of the
// quad's first lane is inverted, every lane returns it)
FPG_NOINL fq fq_inv_quad(const fq& a) {
    fq t, r3;
    mp::inv_ds_quad<12>(t.v, a.v, FQ_P, FQ_PINV);
    fq_from_const(r3, FQ_R3);
    return fq_mul(t, r3);
}

// ---------------------------------------------------------------------------------------
// Fr
// ---------------------------------------------------------------------------------------
FPG_DEV void fr_zero(fr& a) {
#pragma unroll
    for (int j = 0; j < 8; j++) a.v[j] = 0;
}
FPG_DEV void fr_one(fr& a) {
#pragma unroll
    for (int j = 0; j < 8; j++) a.v[j] = FR_ONE[j];
}
static __device__ __noinline__ fr fr_mul_ool(fr a, fr b) {
    fr r;
    mp::mont_mul<8>(r.v, a.v, b.v, FR_P, FR_PINV);
    return r;
}
FPG_DEV fr fr_mul(const fr& a, const fr& b) { return fr_mul_ool(a, b); }
FPG_DEV fr fr_add(const fr& a, const fr& b) { fr r; mp::mod_add<8>(r.v, a.v, b.v, FR_P); return r; }
FPG_DEV fr fr_sub(const fr& a, const fr& b) { fr r; mp::mod_sub<8>(r.v, a.v, b.v, FR_P); return r; }
FPG_DEV bool fr_is_zero(const fr& a) { return mp::is_zero<8>(a.v); }
FPG_DEV fr fr_to_mont(const fr& a) {
    fr r2;
#pragma unroll
    for (int j = 0; j < 8; j++) r2.v[j] = FR_R2[j];
    return fr_mul(a, r2);
}
FPG_DEV fr fr_from_mont(const fr& a) {
    fr one; fr_zero(one); one.v[0] = 1;
    return fr_mul(a, one);
}
FPG_DEV bool fr_canonical_lt_r(const fr& a) { return mp::lt<8>(a.v, FR_P); }
FPG_NOINL fr fr_inv(const fr& a) {
    fr t, r3;
    mp::inv_ds<8>(t.v, a.v, FR_P, FR_PINV);
#pragma unroll
    for (int j = 0; j < 8; j++) r3.v[j] = FR_R3[j];
    return fr_mul(t, r3);
}
// the same on the four lanes of a quad (as fq_inv_quad)
FPG_NOINL fr fr_inv_quad(const fr& a) {
    fr t, r3;
    mp::inv_ds_quad<8>(t.v, a.v, FR_P, FR_PINV);
#pragma unroll
    for (int j = 0; j < 8; j++) r3.v[j] = FR_R3[j];
    return fr_mul(t, r3);
}
// Montgomery form of the 512-bit big-endian integer in `be` reduced mod r:
// mont(hi 2^256 + lo) = mont_mul(hi, R^3) + mont_mul(lo, R^2) with R = 2^256.
FPG_DEV fr fr_from_be64(const uint8_t* be) {
    fr hi, lo, r2, r3;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint8_t* h = be + 28 - 4 * j;
        const uint8_t* l = be + 60 - 4 * j;
        hi.v[j] = ((uint32_t)h[0] << 24) | ((uint32_t)h[1] << 16) | ((uint32_t)h[2] << 8) | h[3];
        lo.v[j] = ((uint32_t)l[0] << 24) | ((uint32_t)l[1] << 16) | ((uint32_t)l[2] << 8) | l[3];
        r2.v[j] = FR_R2[j];
        r3.v[j] = FR_R3[j];
    }
    return fr_add(fr_mul(hi, r3), fr_mul(lo, r2));
}
// canonical big-endian bytes of an Fr residue
FPG_DEV void fr_to_be(uint8_t* out, const fr& a) {
    fr c = fr_from_mont(a);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        uint32_t w = c.v[7 - j];
        out[4 * j] = (uint8_t)(w >> 24); out[4 * j + 1] = (uint8_t)(w >> 16);
        out[4 * j + 2] = (uint8_t)(w >> 8); out[4 * j + 3] = (uint8_t)w;
    }
}
FPG_DEV void fq_to_be(uint8_t* out, const fq& a) {
    fq c = fq_from_mont(a);
#pragma unroll
    for (int j = 0; j < 12; j++) {
        uint32_t w = c.v[11 - j];
        out[4 * j] = (uint8_t)(w >> 24); out[4 * j + 1] = (uint8_t)(w >> 16);
        out[4 * j + 2] = (uint8_t)(w >> 8); out[4 * j + 3] = (uint8_t)w;
    }
}
