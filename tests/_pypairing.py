"""An independent, very slow pure-Python optimal-ate pairing for BLS12-381, used only to pin
the oracle's pairing.  It shares nothing with the oracle's representation or formulas:

  * Fq12 is Fq[w]/(w^12 - 2 w^6 + 2): with u = w^6 - 1 one has u^2 = -1, so this is the
    same field as Fq2[w]/(w^6 - (1 + u)), written over Fq with twelve coefficients.
  * Q in E'(Fq2) is mapped onto E(Fq12): y^2 = x^3 + 4 by (x', y') -> (x' w^-2, y' w^-3).
  * Miller's algorithm runs in affine coordinates ON E(Fq12) with general chord/tangent
    slopes, including the vertical lines, so f_{n,Q} is the exact Miller function with
    divisor n(Q) - ([n]Q) - (n-1)(O).
  * For the negative loop parameter x, f_{x,Q} = 1 / (f_{|x|,Q} v_{[|x|]Q}) by the definition
    of Miller functions, and e(P, Q) = f_{x,Q}(P)^((p^12 - 1)/r).
"""
from __future__ import annotations

from tests._pyref import P, R, X

# ---------------------------------------------------------------- Fq[w]/(w^12 - 2w^6 + 2)
DEG = 12


def _reduce(c):
    c = list(c)
    for k in range(len(c) - 1, DEG - 1, -1):       # w^k = 2 w^(k-6) - 2 w^(k-12)
        v = c[k]
        if v:
            c[k - 6] = (c[k - 6] + 2 * v) % P
            c[k - 12] = (c[k - 12] - 2 * v) % P
        c[k] = 0
    return [v % P for v in c[:DEG]] + [0] * max(0, DEG - len(c))


def mul(a, b):
    c = [0] * (2 * DEG - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                c[i + j] += x * y
    return _reduce(c)


def add(a, b):
    return [(x + y) % P for x, y in zip(a, b)]


def sub(a, b):
    return [(x - y) % P for x, y in zip(a, b)]


def scal(a, s):
    return [x * s % P for x in a]


def const(v):
    return [v % P] + [0] * (DEG - 1)


def _poly_divmod(n, d):
    n = list(n)
    while n and n[-1] == 0:
        n.pop()
    dd = list(d)
    while dd and dd[-1] == 0:
        dd.pop()
    inv = pow(dd[-1], -1, P)
    q = [0] * max(1, len(n) - len(dd) + 1)
    while len(n) >= len(dd) and n:
        s = n[-1] * inv % P
        k = len(n) - len(dd)
        q[k] = s
        for i, v in enumerate(dd):
            n[k + i] = (n[k + i] - s * v) % P
        while n and n[-1] == 0:
            n.pop()
    return q, n


def inv(a):
    """Extended Euclid in Fq[w] against the modulus polynomial."""
    modp = [2, 0, 0, 0, 0, 0, P - 2, 0, 0, 0, 0, 0, 1]
    r0, r1 = modp, list(a)
    s0, s1 = [0], [1]
    while any(r1):
        q, rem = _poly_divmod(r0, r1)
        # s2 = s0 - q s1
        prod = [0] * (len(q) + len(s1))
        for i, x in enumerate(q):
            for j, y in enumerate(s1):
                prod[i + j] = (prod[i + j] + x * y) % P
        s2 = [((s0[i] if i < len(s0) else 0) - (prod[i] if i < len(prod) else 0)) % P
              for i in range(max(len(s0), len(prod)))]
        r0, r1, s0, s1 = r1, rem, s1, s2
    g = r0
    while g and g[-1] == 0:
        g.pop()
    assert len(g) == 1, "not invertible"
    ginv = pow(g[0], -1, P)
    res = [v * ginv % P for v in s0]
    return _reduce(res + [0] * max(0, 2 * DEG - 1 - len(res)))


def power(a, e):
    acc = const(1)
    base = a
    while e:
        if e & 1:
            acc = mul(acc, base)
        base = mul(base, base)
        e >>= 1
    return acc


W = [0, 1] + [0] * (DEG - 2)
W_INV = inv(W)


def fq2_embed(c0, c1):
    """c0 + c1 u with u = w^6 - 1."""
    v = [0] * DEG
    v[0] = (c0 - c1) % P
    v[6] = c1 % P
    return v


# ---------------------------------------------------------------- curve over Fq12
def ec_double(T):
    x, y = T
    lam = mul(scal(mul(x, x), 3), inv(scal(y, 2)))
    x3 = sub(sub(mul(lam, lam), x), x)
    y3 = sub(mul(lam, sub(x, x3)), y)
    return (x3, y3), lam


def ec_add(T, Q):
    x1, y1 = T
    x2, y2 = Q
    lam = mul(sub(y2, y1), inv(sub(x2, x1)))
    x3 = sub(sub(mul(lam, lam), x1), x2)
    y3 = sub(mul(lam, sub(x1, x3)), y1)
    return (x3, y3), lam


def line(T, lam, Pt):
    """l(P) = yP - yT - lam (xP - xT)."""
    return sub(sub(Pt[1], T[1]), mul(lam, sub(Pt[0], T[0])))


def vertical(T, Pt):
    return sub(Pt[0], T[0])


def miller_abs(Q, Pt, n):
    """f_{n,Q}(P) by the affine double-and-add Miller algorithm, vertical lines included."""
    f_num, f_den = const(1), const(1)
    T = Q
    for i in range(n.bit_length() - 2, -1, -1):
        T2, lam = ec_double(T)
        f_num = mul(mul(f_num, f_num), line(T, lam, Pt))
        f_den = mul(mul(f_den, f_den), vertical(T2, Pt))
        T = T2
        if (n >> i) & 1:
            T3, lam = ec_add(T, Q)
            f_num = mul(f_num, line(T, lam, Pt))
            f_den = mul(f_den, vertical(T3, Pt))
            T = T3
    return f_num, f_den, T


def pairing_tower(P_aff, Q_aff):
    """e(P, Q) for affine P in E(Fq) (ints), Q in E'(Fq2) ((c0, c1) pairs); returns 12 Fq."""
    Pt = (const(P_aff[0]), const(P_aff[1]))
    w2inv = mul(W_INV, W_INV)
    w3inv = mul(w2inv, W_INV)
    Qx = mul(fq2_embed(*Q_aff[0]), w2inv)
    Qy = mul(fq2_embed(*Q_aff[1]), w3inv)
    # sanity: the untwisted point lies on y^2 = x^3 + 4
    assert sub(mul(Qy, Qy), add(mul(mul(Qx, Qx), Qx), const(4))) == [0] * DEG
    n = -X
    num, den, T = miller_abs((Qx, Qy), Pt, n)
    # f_{x,Q} = 1 / (f_{|x|,Q} v_{[|x|]Q}) for x = -|x|
    f = mul(den, inv(mul(num, vertical(T, Pt))))
    return power(f, (P**12 - 1) // R)


def to_tower_bytes(a) -> bytes:
    """Coefficients over Fq of w^0..w^11 -> tower-order GT bytes (c0.c0, c0.c1, c0.c2, c1.c0, ...),
    using w^(k+6) = w^k (1 + u): flat Fq2 coefficient of w^k is (a_k + a_{k+6}) + a_{k+6} u."""
    flat = [((a[k] + a[k + 6]) % P, a[k + 6] % P) for k in range(6)]
    order = [0, 2, 4, 1, 3, 5]
    return b"".join(flat[k][0].to_bytes(48, "big") + flat[k][1].to_bytes(48, "big") for k in order)


def pairing_bytes(P96: bytes, Q192: bytes) -> bytes:
    Px, Py = int.from_bytes(P96[:48], "big"), int.from_bytes(P96[48:], "big")
    q = [int.from_bytes(Q192[48 * i: 48 * i + 48], "big") for i in range(4)]
    return to_tower_bytes(pairing_tower((Px, Py), ((q[0], q[1]), (q[2], q[3]))))
