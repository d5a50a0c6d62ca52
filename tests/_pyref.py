"""Independent pure-Python reference pieces used to PIN the oracle (never to produce stored
expected values for the GPU path).  Everything here is computed with Python integers from
the mathematical definitions, not from the oracle's code."""
from __future__ import annotations

import hashlib

X = -0xD201000000010000
R = X**4 - X**2 + 1
P = (X - 1) ** 2 * R // 3 + X


def eq_weight(t: int, c: int, tau) -> int:
    """prod_{s<t} (c_s tau_s + (1 - c_s)(1 - tau_s)) mod r (Eq. multi-extension's basis)."""
    acc = 1
    for s in range(t):
        acc = acc * (tau[s] if (c >> s) & 1 else (1 - tau[s])) % R
    return acc


def mle_eval(table, tau) -> int:
    """f(tau) for the multilinear extension of `table` with variable x_s <-> bit s."""
    t = len(table).bit_length() - 1
    return sum(v * eq_weight(t, c, tau) for c, v in enumerate(table)) % R


def hfr(tag: str, data: bytes) -> int:
    t = tag.encode()
    wide = hashlib.sha256(t + b"\x00" + data).digest() + hashlib.sha256(t + b"\x01" + data).digest()
    return int.from_bytes(wide, "big") % R


def proof_size(b: int, log_n: int, g1: int, g2: int, gt: int, fr: int, digest: int = 32) -> int:
    """|pi_i| = b G1 + (2l GT + (2l+1) G1 + 2 G2) + l (G1 + Fr) + l G1 + log N digests, l = log mu
    (Sec. 3 "Efficiency: proof size" and Sec. 4.3 "Proof size")."""
    ell = log_n // 2
    return b * g1 + (2 * ell * gt + (2 * ell + 1) * g1 + 2 * g2) + ell * (g1 + fr) + ell * g1 + log_n * digest
