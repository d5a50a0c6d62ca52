"""The look-ahead round kernels (lookahead.cuh) compiled for the host and checked against a direct
round computed with the oracle's group operations (no GPU).  Cases: two blocks covering all four
quadrants of b's support; a stride beyond the live state with two pairs per class; a block larger
than the live state (b dense over it, as in a late round or the evaluation proof).

From a state A, v, b of round j-1 (length 2h per block) and its challenge x, the kernels produce
round j's record L_j.T, L_j.1, R_j.T, R_j.1 without folding first; the reference folds
(A' = A_L + x A_R, v' = v_L + x^-1 v_R, b' = b_L + x^-1 b_R) and evaluates the round directly:
L_j.T = prod e(A'[h2 + i], v'[i]), R_j.T = prod e(A'[i], v'[h2 + i]), L_j.1 = sum b'[i] A'[h2 + i],
R_j.1 = sum b'[h2 + i] A'[i] (Sec. 3, Eq. folding).  The states are random (with an identity point),
b lives on the protocol's support positions, and the stride may exceed the live length.
"""
import ctypes
import os
import random
import shutil
import subprocess

import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_03031_gb300", "csrc")
R_FR = O.const_r()


@pytest.fixture(scope="module")
def la(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    lib = str(tmp_path_factory.mktemp("emu") / "liblookahead.so")
    subprocess.check_call([gxx, "-std=c++20", "-O1", "-shared", "-fPIC", f"-I{CSRC}", "-o", lib,
                           os.path.join(HERE, "emu", "lookahead.cpp")])
    L = ctypes.CDLL(lib)
    L.emu_la_round.restype = None
    return L


def support(k0, k, bsz, R, h):
    """Positions of block k's b in a state of length 2h (the protocol's support rule)."""
    sk = min(bsz, R - (k0 + k) * bsz)
    return [((k0 + k) * bsz + t) % (2 * h) if sk <= 2 * h else t for t in range(min(sk, 2 * h))]


def direct_round(A, v, b, x, h2):
    """Round j's record from round j-1's state by folding first (oracle group operations)."""
    h = 2 * h2
    xi = pow(x, -1, R_FR)
    Af = [O.g1_add(A[i], O.g1_mul(A[h + i], x)) for i in range(h)]
    vf = [O.g2_add(v[i], O.g2_mul(v[h + i], xi)) for i in range(h)]
    bf = [(b[i] + xi * b[h + i]) % R_FR for i in range(h)]
    one = O.fq12_pow(O.pairing(O.g1_gen(), O.g2_gen()), 0)
    LT, RT, L1, R1 = one, one, bytes(96), bytes(96)
    for i in range(h2):
        LT = O.fq12_mul(LT, O.pairing(Af[h2 + i], vf[i]))
        RT = O.fq12_mul(RT, O.pairing(Af[i], vf[h2 + i]))
        L1 = O.g1_add(L1, O.g1_mul(Af[h2 + i], bf[i]))
        R1 = O.g1_add(R1, O.g1_mul(Af[i], bf[h2 + i]))
    return LT + L1 + RT + R1


@pytest.mark.parametrize("K,R,h2,k0,bsz", [(2, 4, 1, 0, 3), (1, 16, 2, 1, 5), (1, 16, 1, 0, 16)])
def test_lookahead_round_equals_direct_round(la, K, R, h2, k0, bsz):
    rnd = random.Random(K * 1000 + R * 10 + h2)
    h = 2 * h2
    A = [O.g1_mul(O.g1_gen(), rnd.randrange(1, R_FR)) for _ in range(K * R)]
    A[1] = bytes(96)                                              # an identity row
    v = [O.g2_mul(O.g2_gen(), rnd.randrange(1, R_FR)) for _ in range(K * R)]
    b = [0] * (K * R)
    for k in range(K):
        for p in support(k0, k, bsz, R, h):
            b[k * R + p] = rnd.randrange(1, R_FR)
    x = [rnd.randrange(1, R_FR) for _ in range(K)]
    rec = ctypes.create_string_buffer(K * 2 * (576 + 96))
    la.emu_la_round(K, R, h2, k0, bsz, b"".join(A), b"".join(v),
                    b"".join(t.to_bytes(32, "big") for t in b), b"".join(t.to_bytes(32, "big") for t in x), rec)
    for k in range(K):
        exp = direct_round(A[k * R:(k + 1) * R], v[k * R:(k + 1) * R], b[k * R:(k + 1) * R], x[k], h2)
        assert rec.raw[k * 1344:(k + 1) * 1344] == exp, k
