"""Writes constants.cuh, the compile-time constants of the CUDA path, from first principles
with Python integers (run: python gen_constants.py).  Nothing here is shared with any other
part of the repository.

  * BLS12-381 from its seed x = -0xd201000000010000: r = x^4 - x^2 + 1, p = (x-1)^2 r/3 + x.
  * Montgomery constants for R = 2^384 (Fq, 12 x 32-bit limbs) and R = 2^256 (Fr, 8 limbs).
  * Standard generators of G1 and G2 (checked on their curves and of order r below).
  * Frobenius coefficients xi^(k(p-1)/6), xi^(k(p^2-1)/6) for Fq12 = Fq2[w]/(w^6 - xi), xi = 1+u.
  * SHA-256 round constants and initial hash value from FIPS 180-4 Sec. 4.2.2 / 5.3.3: the
    first 32 bits of the fractional parts of the cube (square) roots of the first 64 (8) primes.
"""
import os

X = -0xD201000000010000
R = X**4 - X**2 + 1
P = (X - 1) ** 2 * R // 3 + X
H1 = (X - 1) ** 2 // 3
assert P.bit_length() == 381 and R.bit_length() == 255 and (X - 1) ** 2 % 3 == 0

G1 = (0x17F1D3A73197D7942695638C4FA9AC0FC3688C4F9774B905A14E3A3F171BAC586C55E83FF97A1AEFFB3AF00ADB22C6BB,
      0x08B3F481E3AAA0F1A09E30ED741D8AE4FCF5E095D5D00AF600DB18CB2C04B3EDD03CC744A2888AE40CAA232946C5E7E1)
G2 = ((0x024AA2B2F08F0A91260805272DC51051C6E47AD4FA403B02B4510B647AE3D1770BAC0326A805BBEFD48056C8C121BDB8,
       0x13E02B6052719F607DACD3A088274F65596BD0D09920B61AB5DA61BBDC7F5049334CF11213945D57E5AC7D055D042B7E),
      (0x0CE5D527727D6E118CC9CDC6DA2E351AADFD9BAA8CBDD3A76D429A695160D12C923AC9CC3BACA289E193548608B82801,
       0x0606C4A02EA734CC32ACD2B02BC28B99CB3E287E85A763AF267492AB572E99AB3F370D275CEC1DA1AAA9075FF05F79BE))


def f2mul(a, b):
    return ((a[0] * b[0] - a[1] * b[1]) % P, (a[0] * b[1] + a[1] * b[0]) % P)


def f2pow(a, e):
    r = (1, 0)
    while e:
        if e & 1:
            r = f2mul(r, a)
        a = f2mul(a, a)
        e >>= 1
    return r


# curve checks (y^2 = x^3 + 4 and the twist y^2 = x^3 + 4(1+u))
assert (G1[1] ** 2 - G1[0] ** 3 - 4) % P == 0
lhs = f2mul(G2[1], G2[1])
rhs = f2mul(f2mul(G2[0], G2[0]), G2[0])
assert ((lhs[0] - rhs[0] - 4) % P, (lhs[1] - rhs[1] - 4) % P) == (0, 0)


def g1_mul(k, pt):  # affine double-and-add, only for the order check
    def add(A, B):
        if A is None: return B
        if B is None: return A
        if A[0] == B[0]:
            if (A[1] + B[1]) % P == 0: return None
            lam = 3 * A[0] * A[0] * pow(2 * A[1], -1, P) % P
        else:
            lam = (B[1] - A[1]) * pow(B[0] - A[0], -1, P) % P
        x3 = (lam * lam - A[0] - B[0]) % P
        return (x3, (lam * (A[0] - x3) - A[1]) % P)
    acc = None
    for bit in bin(k)[2:]:
        acc = add(acc, acc)
        if bit == "1":
            acc = add(acc, pt)
    return acc


assert g1_mul(R, G1) is None

XI = (1, 1)


def f2inv(a):
    n = pow((a[0] * a[0] + a[1] * a[1]) % P, -1, P)
    return (a[0] * n % P, (-a[1]) * n % P)


# GLV on G1: phi(x, y) = (omega x, y) acts as [lambda] with lambda = -x^2 mod r for the cube root of
# unity omega picked below; k = k0 + k1 |x|^2 gives k P = k0 P + k1 (-phi(P)).
_g = 2
while pow(_g, (P - 1) // 3, P) == 1:
    _g += 1
_w = pow(_g, (P - 1) // 3, P)
OMEGA = None
for _om in (_w, _w * _w % P):
    if g1_mul((-X * X) % R, G1) == ((_om * G1[0]) % P, G1[1]):
        OMEGA = _om
assert OMEGA is not None
XABS = -X
D_GLV = XABS * XABS
BAR_GLV = (1 << 256) // D_GLV           # Barrett constant for floor(k / |x|^2), k < 2^256
BAR_X = (1 << 256) // XABS              # Barrett constant for floor(k / |x|)
# GLS on G2: psi(x, y) = (conj(x) cx, conj(y) cy), cx = xi^-((p-1)/3), cy = xi^-((p-1)/2), acts as [x];
# with base-|x| digits d_i of k, k Q = d0 Q - d1 psi(Q) + d2 psi^2(Q) - d3 psi^3(Q).
PSI_CX = f2inv(f2pow(XI, (P - 1) // 3))
PSI_CY = f2inv(f2pow(XI, (P - 1) // 2))


def psi(pt):
    (x0, x1), (y0, y1) = pt
    return (f2mul((x0, (-x1) % P), PSI_CX), f2mul((y0, (-y1) % P), PSI_CY))


def g2_affine_mul(k, pt):          # affine double-and-add on the twist, only for the check below
    def add(A, B):
        if A is None: return B
        if B is None: return A
        if A[0] == B[0]:
            if ((A[1][0] + B[1][0]) % P, (A[1][1] + B[1][1]) % P) == (0, 0): return None
            num = f2mul((3, 0), f2mul(A[0], A[0]))
            lam = f2mul(num, f2inv(((2 * A[1][0]) % P, (2 * A[1][1]) % P)))
        else:
            lam = f2mul(((B[1][0] - A[1][0]) % P, (B[1][1] - A[1][1]) % P),
                        f2inv(((B[0][0] - A[0][0]) % P, (B[0][1] - A[0][1]) % P)))
        l2 = f2mul(lam, lam)
        x3 = ((l2[0] - A[0][0] - B[0][0]) % P, (l2[1] - A[0][1] - B[0][1]) % P)
        t = f2mul(lam, ((A[0][0] - x3[0]) % P, (A[0][1] - x3[1]) % P))
        return (x3, ((t[0] - A[1][0]) % P, (t[1] - A[1][1]) % P))
    acc = None
    for bit in bin(k)[2:]:
        acc = add(acc, acc)
        if bit == "1":
            acc = add(acc, pt)
    return acc


assert psi(G2) == g2_affine_mul(X % R, G2)
FROB1 = [f2pow(XI, k * (P - 1) // 6) for k in range(6)]
FROB2 = [f2pow(XI, k * (P * P - 1) // 6) for k in range(6)]
assert all(c[1] == 0 for c in FROB2)


def limbs(v, n):
    return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)]


def arr(name, v, n):
    return f"__constant__ uint32_t {name}[{n}] = {{" + ", ".join(f"0x{w:08x}u" for w in limbs(v, n)) + "};\n"


def mont(v, n):
    return v * (1 << (32 * n)) % (P if n == 12 else R)


def primes(k):
    ps, c = [], 2
    while len(ps) < k:
        if all(c % q for q in ps):
            ps.append(c)
        c += 1
    return ps


def iroot(v, k):
    lo, hi = 0, 1
    while hi**k <= v:
        hi *= 2
    while lo < hi - 1:
        mid = (lo + hi) // 2
        if mid**k <= v:
            lo = mid
        else:
            hi = mid
    return lo


SHA_K = [iroot(p << (3 * 32), 3) & 0xFFFFFFFF for p in primes(64)]       # frac(cbrt(p)) * 2^32
SHA_H = [iroot(p << (2 * 32), 2) & 0xFFFFFFFF for p in primes(8)]        # frac(sqrt(p)) * 2^32
assert SHA_K[0] == 0x428A2F98 and SHA_H[0] == 0x6A09E667

out = ["// Generated by gen_constants.py -- do not edit.  See that script for the derivations.\n",
       "#pragma once\n#include <cstdint>\n\n"]
out.append(arr("FQ_P", P, 12))
out.append(f"#define FQ_PINV 0x{(-pow(P, -1, 2**32)) % 2**32:08x}u\n")
out.append(arr("FQ_ONE", mont(1, 12), 12))
out.append(arr("FQ_R2", (1 << 768) % P, 12))
out.append(arr("FQ_PM2", P - 2, 12))
out.append(arr("FQ_R3", (1 << 1152) % P, 12))
out.append(arr("FR_P", R, 8))
out.append(f"#define FR_PINV 0x{(-pow(R, -1, 2**32)) % 2**32:08x}u\n")
out.append(arr("FR_ONE", mont(1, 8), 8))
out.append(arr("FR_R2", (1 << 512) % R, 8))
out.append(arr("FR_R3", (1 << 768) % R, 8))
out.append(arr("FR_PM2", R - 2, 8))
out.append(arr("G1_GEN_X", mont(G1[0], 12), 12))
out.append(arr("G1_GEN_Y", mont(G1[1], 12), 12))
out.append(arr("G2_GEN_X0", mont(G2[0][0], 12), 12))
out.append(arr("G2_GEN_X1", mont(G2[0][1], 12), 12))
out.append(arr("G2_GEN_Y0", mont(G2[1][0], 12), 12))
out.append(arr("G2_GEN_Y1", mont(G2[1][1], 12), 12))
out.append(arr("FQ_FOUR", mont(4, 12), 12))
for k in range(6):
    out.append(arr(f"FROB1_{k}_C0", mont(FROB1[k][0], 12), 12))
    out.append(arr(f"FROB1_{k}_C1", mont(FROB1[k][1], 12), 12))
    out.append(arr(f"FROB2_{k}", mont(FROB2[k][0], 12), 12))
out.append(f"#define BLS_X_ABS 0x{-X:016x}ull\n")
out.append(arr("GLV_OMEGA", mont(OMEGA, 12), 12))
out.append(arr("GLV_D", D_GLV, 4))
out.append(arr("GLV_BARRETT", BAR_GLV, 5))
out.append(arr("GLS_D", XABS, 2))
out.append(arr("GLS_BARRETT", BAR_X, 7))
out.append(arr("PSI_CX0", mont(PSI_CX[0], 12), 12))
out.append(arr("PSI_CX1", mont(PSI_CX[1], 12), 12))
out.append(arr("PSI_CY0", mont(PSI_CY[0], 12), 12))
out.append(arr("PSI_CY1", mont(PSI_CY[1], 12), 12))
out.append(arr("BLS_H1", H1, 4))


def wnaf(k, w):
    """Width-w non-adjacent form of k > 0, least significant digit first: odd digits |d| < 2^(w-1),
    every nonzero digit followed by at least w - 1 zeros."""
    digits = []
    while k:
        if k & 1:
            d = k % (1 << w)
            if d >= 1 << (w - 1):
                d -= 1 << w
            k -= d
        else:
            d = 0
        digits.append(d)
        k >>= 1
    return digits


H1_WNAF = wnaf(H1, 4)
assert sum(d << i for i, d in enumerate(H1_WNAF)) == H1
out.append(f"#define BLS_H1_WNAF_LEN {len(H1_WNAF)}\n")
out.append("__constant__ signed char BLS_H1_WNAF[" + str(len(H1_WNAF)) + "] = {" +
           ", ".join(str(d) for d in H1_WNAF) + "};\n")
# the block-split Fq product (fq_split.cuh): c_k = 2^(32 k - 320) mod p for the limbs k < 10 of a
# double-width product folded into its high part, and -p^-1 mod 2^64 for the closing two-limb
# Montgomery step
# (rows 10 and 11 are zero: the warps all run three fold rows, the surplus ones with a zero factor)
out.append("__constant__ uint32_t FQ_FOLD[12][12] = {" + ", ".join(
    "{" + ", ".join(f"0x{w:08x}u" for w in limbs(pow(2, 32 * k - 320, P) if k < 10 else 0, 12)) + "}"
    for k in range(12)) + "};\n")
out.append(f"#define FQ_PINV64_LO 0x{(-pow(P, -1, 2**64)) % 2**32:08x}u\n")
out.append(f"#define FQ_PINV64_HI 0x{((-pow(P, -1, 2**64)) % 2**64) >> 32:08x}u\n")
out.append("__constant__ uint32_t SHA256_K[64] = {" + ", ".join(f"0x{k:08x}u" for k in SHA_K) + "};\n")
out.append("__constant__ uint32_t SHA256_H0[8] = {" + ", ".join(f"0x{k:08x}u" for k in SHA_H) + "};\n")
open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "constants.cuh"), "w").write("".join(out))
