"""Pure-Python BLS12-381 group arithmetic (affine, Python integers) used only to PIN the oracle.

Nothing here shares code or representation with the oracle: G1 is E(Fq): y^2 = x^3 + 4 and G2 is
the twist E'(Fq2): y^2 = x^3 + 4(1 + u) with Fq2 = Fq[u]/(u^2 + 1), both with the textbook affine
chord-and-tangent law and plain double-and-add scalar multiplication; the identity is None.  GT
elements are powers of e(g1, g2), which the independent pure-Python pairing in _pypairing computes.
"""
from __future__ import annotations

import functools

from tests import _pypairing as pyp
from tests._pyref import P, R, mle_eval

# ---------------------------------------------------------------- Fq2 = Fq[u]/(u^2 + 1)


def f2_add(a, b):
    return ((a[0] + b[0]) % P, (a[1] + b[1]) % P)


def f2_sub(a, b):
    return ((a[0] - b[0]) % P, (a[1] - b[1]) % P)


def f2_mul(a, b):
    return ((a[0] * b[0] - a[1] * b[1]) % P, (a[0] * b[1] + a[1] * b[0]) % P)


def f2_inv(a):
    n = pow((a[0] * a[0] + a[1] * a[1]) % P, -1, P)
    return (a[0] * n % P, -a[1] * n % P)


# ---------------------------------------------------------------- the two curves, one law
class _Field:
    def __init__(self, add, sub, mul, inv, small):
        self.add, self.sub, self.mul, self.inv, self.small = add, sub, mul, inv, small


_FQ = _Field(lambda a, b: (a + b) % P, lambda a, b: (a - b) % P, lambda a, b: a * b % P,
             lambda a: pow(a, -1, P), lambda k: k % P)
_FQ2 = _Field(f2_add, f2_sub, f2_mul, f2_inv, lambda k: (k % P, 0))


def _ec_add(F, p, q):
    if p is None:
        return q
    if q is None:
        return p
    (x1, y1), (x2, y2) = p, q
    if x1 == x2:
        if F.add(y1, y2) == F.small(0):
            return None
        lam = F.mul(F.mul(F.small(3), F.mul(x1, x1)), F.inv(F.mul(F.small(2), y1)))
    else:
        lam = F.mul(F.sub(y2, y1), F.inv(F.sub(x2, x1)))
    x3 = F.sub(F.sub(F.mul(lam, lam), x1), x2)
    return (x3, F.sub(F.mul(lam, F.sub(x1, x3)), y1))


def _ec_mul(F, p, k):
    acc = None
    for bit in bin(k % R)[2:]:
        acc = _ec_add(F, acc, acc)
        if bit == "1":
            acc = _ec_add(F, acc, p)
    return acc


def g1_from_bytes(b: bytes):
    x, y = int.from_bytes(b[:48], "big"), int.from_bytes(b[48:96], "big")
    return None if x == 0 and y == 0 else (x, y)


def g1_bytes(p) -> bytes:
    return bytes(96) if p is None else p[0].to_bytes(48, "big") + p[1].to_bytes(48, "big")


def g2_from_bytes(b: bytes):
    c = [int.from_bytes(b[48 * i:48 * i + 48], "big") for i in range(4)]
    return None if not any(c) else ((c[0], c[1]), (c[2], c[3]))


def g2_bytes(p) -> bytes:
    if p is None:
        return bytes(192)
    (x0, x1), (y0, y1) = p
    return b"".join(v.to_bytes(48, "big") for v in (x0, x1, y0, y1))


def g1_add(p, q):
    return _ec_add(_FQ, p, q)


def g1_mul(p, k):
    return _ec_mul(_FQ, p, k)


def g2_add(p, q):
    return _ec_add(_FQ2, p, q)


def g2_mul(p, k):
    return _ec_mul(_FQ2, p, k)


def on_g1(p) -> bool:
    return p is None or (p[1] * p[1] - p[0] ** 3 - 4) % P == 0


def on_g2(p) -> bool:
    if p is None:
        return True
    x, y = p
    return f2_sub(f2_mul(y, y), f2_add(f2_mul(x, f2_mul(x, x)), (4, 4))) == (0, 0)


class Groups:
    """Exponent-to-bytes maps s -> g1^s, g2^s, e(g1, g2)^s for the generators g1, g2 (given as
    serialised points); results are cached by exponent."""

    def __init__(self, g1_gen: bytes, g2_gen: bytes):
        self.g1 = g1_from_bytes(g1_gen)
        self.g2 = g2_from_bytes(g2_gen)
        assert on_g1(self.g1) and on_g2(self.g2)
        assert g1_mul(self.g1, R) is None and g2_mul(self.g2, R) is None
        self._gt = None

    @functools.lru_cache(maxsize=None)
    def G1(self, s: int) -> bytes:
        return g1_bytes(g1_mul(self.g1, s % R))

    @functools.lru_cache(maxsize=None)
    def G2(self, s: int) -> bytes:
        return g2_bytes(g2_mul(self.g2, s % R))

    @functools.lru_cache(maxsize=None)
    def GT(self, s: int) -> bytes:
        if self._gt is None:
            Px, Py = self.g1
            self._gt = pyp.pairing_tower((Px, Py), self.g2)
        return pyp.to_tower_bytes(pyp.power(self._gt, s % R))


def commit_closed_form(grp: Groups, beta: int, tau: list[int], nrows: int, M: int, m: list[int]):
    """VC.Commit from the trapdoor: C_j = g1^{f_j(tau)} and C = e(g1, g2)^{sum_j f_j(tau) beta^{2j}},
    f_j the multilinear extension of row j (Eqs. genCi and genC).  Returns (C, rows) as bytes."""
    f = [mle_eval(m[j * M:(j + 1) * M], tau) for j in range(nrows)]
    rows = b"".join(grp.G1(v) for v in f)
    return grp.GT(sum(f[j] * pow(beta, 2 * j, R) for j in range(nrows))), rows
