"""Pins of the oracle's Fiat-Shamir transcript and Merkle byte layouts.

Every byte of every proof pi_i (and the commitment, the Merkle root and r_j) is re-derived here in
pure Python from the protocol's definitions and the encoding readings, with hashlib for SHA-256,
tests._pyref.hfr for HFr, and group elements formed as powers of the generators from their known
discrete logarithms (tests._pyec: an independent affine group law; GT powers of e(g1, g2) from the
independent pure-Python pairing).  Nothing is taken from the oracle but the public setup's
generators, its trapdoor (beta, tau) and the proofs being checked.

The readings re-derived (the paper leaves the random oracles and the Merkle instantiation open:
Sec. 2 "random oracles", Sec. 3 FC.BOpen with Eq. b, Sec. 4.2 "Making our protocol
non-interactive"):
  * r_a = HFr("FP-r", SHA256(C || u32be(k) || u32be(b) || u32be(|S_k|) || D_k) || u32be(a)), D_k the
    root of the tree over the block's C_a: leaves SHA256("FP-sleaf" || C_a), nodes
    SHA256("FP-snode" || left || right) pairing each level left to right, an odd last node carried
    up unchanged;
  * x_j = HFr("FP-x", x_{j-1} || L_j.T || L_j.1 || R_j.T || R_j.1), x_0 empty;
  * z = HFr("FP-z", x_l || v_l), W = g2^{(P(beta) - P(z)) / (beta - z)},
    P(X) = prod_j (1 + x_j^{-1} X^{2^{l_R - j + 1}});
  * leaves SHA256("FP-leaf" || u64be(i) || m_i), nodes SHA256("FP-node" || left || right), row
    leaves SHA256("FP-row" || s_j || C_j), r_j = HFr("FP-rho", root || u32be(j));
  * proof = block (C_a) || pi_{C_k} || path (row tree leaf-up, then the tree over the rows) ||
    sibling pairs (D_w, g_w[a]) leaf-up || (pi_{l_c - 1} .. pi_0).
Each mutation test changes one reading and checks that the re-derivation then disagrees with the
oracle, so a plausible slip in any of them (little-endian integers, swapped node children, a
zero-filled x_0, a different sibling order) cannot pass.
"""
from __future__ import annotations

import dataclasses
import functools
import hashlib

import pytest

import oracle as O
from paper_2601_03031_gb300 import inputs as I
from tests import _pyec
from tests._pyref import R as RR, hfr, mle_eval


@dataclasses.dataclass(frozen=True)
class Reading:
    int_order: str = "big"          # byte order of k, b, |S_k|, a, i, j in the hashed strings
    node_swap: bool = False         # hash (right, left) instead of (left, right)
    x0_zero: bool = False           # x_0 as 32 zero bytes instead of the empty string
    stmt_no_counts: bool = False    # leave u32(b) || u32(|S_k|) out of the statement
    stmt_rows_flat: bool = False    # the C_a themselves in the statement instead of their tree root
    stmt_odd_dup: bool = False      # an odd last node of the statement tree paired with itself
    z_without_x: bool = False       # z from v_l alone
    path_root_first: bool = False   # path digests listed root-down instead of leaf-up
    rho_tag: str = "FP-rho"


def sha(*parts: bytes) -> bytes:
    return hashlib.sha256(b"".join(parts)).digest()


def u32(v: int, rd: Reading) -> bytes:
    return v.to_bytes(4, rd.int_order)


def u64(v: int, rd: Reading) -> bytes:
    return v.to_bytes(8, rd.int_order)


def stmt_rows(rows: list, rd: Reading) -> bytes:
    """D_k: the tree over the block's row commitments (or, read flat, the commitments themselves)."""
    if rd.stmt_rows_flat:
        return b"".join(rows)
    level = [sha(b"FP-sleaf", r) for r in rows]
    while len(level) > 1:
        pairs = [(level[i], level[i + 1]) for i in range(0, len(level) - 1, 2)]
        up = [sha(b"FP-snode", *((r, l) if rd.node_swap else (l, r))) for l, r in pairs]
        if len(level) % 2:
            up.append(sha(b"FP-snode", level[-1], level[-1]) if rd.stmt_odd_dup else level[-1])
        level = up
    return level[0]


def hfr_nonzero(tag: str, data: bytes) -> int:
    """A challenge that must be inverted is re-hashed with a 0x01 byte appended while it is 0."""
    x = hfr(tag, data)
    while x == 0:
        data += b"\x01"
        x = hfr(tag, data)
    return x


def merkle(leaves: list[bytes], rd: Reading) -> list[list[bytes]]:
    """All levels of the binary tree over `leaves` (level 0 the leaves, last level the root)."""
    levels = [leaves]
    while len(levels[-1]) > 1:
        prev = levels[-1]
        nxt = []
        for s in range(len(prev) // 2):
            l, r = prev[2 * s], prev[2 * s + 1]
            nxt.append(sha(b"FP-node", r, l) if rd.node_swap else sha(b"FP-node", l, r))
        levels.append(nxt)
    return levels


class Derivation:
    """Everything OpenAll outputs, re-derived from m, the trapdoor and the readings."""

    def __init__(self, grp: _pyec.Groups, beta: int, tau: list[int], R: int, M: int, m: list[int], b: int,
                 rd: Reading = Reading()):
        self.grp, self.beta, self.tau, self.R, self.M, self.m, self.b, self.rd = grp, beta, tau, R, M, m, b, rd
        self.lr, self.lc = R.bit_length() - 1, M.bit_length() - 1
        self.K = (R + b - 1) // b
        # VC.Commit: C_j = g1^{f_j(tau)}, C = e(g1, g2)^{sum_j f_j(tau) beta^{2j}}
        self.f = [mle_eval(m[j * M:(j + 1) * M], tau) for j in range(R)]
        self.rows = [grp.G1(v) for v in self.f]
        self.C = grp.GT(sum(self.f[j] * pow(beta, 2 * j, RR) for j in range(R)))
        self._step2()
        self.blocks = [self._bopen(k) for k in range(self.K)]

    # ------------------------------------------------------------------ FC.BOpen of block k
    def _bopen(self, k: int) -> bytes:
        rd, R, b, grp = self.rd, self.R, self.b, self.grp
        lo, hi = k * b, min((k + 1) * b, R)
        stmt = self.C + u32(k, rd)
        if not rd.stmt_no_counts:
            stmt += u32(b, rd) + u32(hi - lo, rd)
        stmt += stmt_rows(self.rows[lo:hi], rd)
        hs = sha(stmt)
        bv = [0] * R
        for a in range(lo, hi):
            bv[a] = hfr("FP-r", hs + u32(a, rd))
        # state in exponent form: A[i] = g1^alpha[i], v[i] = g2^nu[i]
        alpha = list(self.f)
        nu = [pow(self.beta, 2 * i, RR) for i in range(R)]
        xprev = bytes(32) if rd.x0_zero else b""
        xinv = []
        out = b""
        for j in range(1, self.lr + 1):
            h = R >> j
            LT = sum(alpha[h + i] * nu[i] for i in range(h)) % RR           # A_R * v_L
            RT = sum(alpha[i] * nu[h + i] for i in range(h)) % RR           # A_L * v_R
            L1 = sum(bv[i] * alpha[h + i] for i in range(h)) % RR          # <A_R, b_L>
            R1 = sum(bv[h + i] * alpha[i] for i in range(h)) % RR          # <A_L, b_R>
            rec = grp.GT(LT) + grp.G1(L1) + grp.GT(RT) + grp.G1(R1)
            out += rec
            x = hfr_nonzero("FP-x", xprev + rec)
            xi = pow(x, -1, RR)
            xinv.append(xi)
            xprev = x.to_bytes(32, "big")
            for i in range(h):
                alpha[i] = (alpha[i] + x * alpha[h + i]) % RR
                nu[i] = (nu[i] + xi * nu[h + i]) % RR
                bv[i] = (bv[i] + xi * bv[h + i]) % RR
        v_l = grp.G2(nu[0])
        out += grp.G1(alpha[0]) + v_l
        z = hfr("FP-z", (b"" if rd.z_without_x else xprev) + v_l)

        def Pf(X):
            acc = 1
            for j in range(1, self.lr + 1):
                acc = acc * (1 + xinv[j - 1] * pow(X, 1 << (self.lr - j + 1), RR)) % RR
            return acc
        assert Pf(self.beta) == nu[0]                       # v_l = g2^{P(beta)}
        w = (Pf(self.beta) - Pf(z)) * pow(self.beta - z, -1, RR) % RR
        return out + grp.G2(w)

    # ------------------------------------------------------------------ Step 2
    def _step2(self):
        rd, R, M = self.rd, self.R, self.M
        self.row_trees = []
        for j in range(R):
            leaves = [sha(b"FP-leaf", u64(j * M + a, rd), self.m[j * M + a].to_bytes(32, "big")) for a in range(M)]
            self.row_trees.append(merkle(leaves, rd))
        row_leaves = [sha(b"FP-row", self.row_trees[j][-1][0], self.rows[j]) for j in range(R)]
        self.top = merkle(row_leaves, rd)
        self.root = self.top[-1][0]
        self.rj = [hfr(rd.rho_tag, self.root + u32(j, rd)) for j in range(R)]
        # fold tree: node s at level h covers rows [s 2^h, (s+1) 2^h)
        self.g = [[[self.rj[j] * self.m[j * M + a] % RR for a in range(M)] for j in range(R)]]
        for h in range(1, self.lr + 1):
            prev = self.g[-1]
            self.g.append([[(prev[2 * s][a] + prev[2 * s + 1][a]) % RR for a in range(M)] for s in range(R >> h)])
        self.gstar = self.g[-1][0]

    def D(self, h: int, s: int) -> bytes:
        return self.grp.G1(mle_eval(self.g[h][s], self.tau))     # D_w = g1^{g_w(tau)}

    def pst(self, a: int) -> bytes:
        out = b""
        for t in range(self.lc - 1, -1, -1):
            p, w = a >> (t + 1), 1 << t
            Q = [(self.gstar[(2 * p + 1) * w + c] - self.gstar[2 * p * w + c]) % RR for c in range(w)]
            out += self.grp.G1(mle_eval(Q, self.tau[:t]) if t else Q[0])
        return out

    def proof(self, i: int) -> bytes:
        rd, M, R = self.rd, self.M, self.R
        j, a = divmod(i, M)
        k = j // self.b
        lo, hi = k * self.b, min((k + 1) * self.b, R)
        out = b"".join(self.rows[lo:hi]) + self.blocks[k]
        path = [self.row_trees[j][l][(a >> l) ^ 1] for l in range(self.lc)]
        tpath = [self.top[l][(j >> l) ^ 1] for l in range(self.lr)]
        if rd.path_root_first:
            path, tpath = path[::-1], tpath[::-1]
        out += b"".join(path) + b"".join(tpath)
        for h in range(self.lr):
            s = (j >> h) ^ 1
            out += self.D(h, s) + self.g[h][s][a].to_bytes(32, "big")
        return out + self.pst(a)


@functools.lru_cache(maxsize=None)
def groups():
    return _pyec.Groups(O.g1_gen(), O.g2_gen())


@functools.lru_cache(maxsize=None)
def case(log_n: int, b: int, seed: int = 7):
    pp = O.PP(log_n, seed)
    mv = I.vector(seed + 50, log_n)
    ml = mv.tobytes()
    C, rows = O.commit(pp, ml)
    pr = O.Prover(pp, ml, C, rows, b)
    pr.blocks(threads=1)
    pr.step2()
    beta, tau = pp.trapdoor()
    return pp, I.to_ints(mv), C, rows, pr, beta, tau


def derive(log_n: int, b: int, rd: Reading = Reading()) -> Derivation:
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    return Derivation(groups(), beta, tau, pp.R, pp.M, m, b, rd)


CASES = [(4, 1), (4, 3), (5, 2)]       # ragged last block at (4, 3); R < M at log N = 5


@pytest.mark.parametrize("log_n,b", CASES)
def test_commitment_and_root(log_n, b):
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    d = derive(log_n, b)
    assert b"".join(d.rows) == rows
    assert d.C == C
    root, rjb, gsb, dsb = pr.step2_parts()
    assert root == d.root
    assert rjb == b"".join(v.to_bytes(32, "big") for v in d.rj)
    assert gsb == b"".join(v.to_bytes(32, "big") for v in d.gstar)
    assert dsb == d.D(d.lr, 0)


@pytest.mark.parametrize("log_n,b", CASES)
def test_every_block_record(log_n, b):
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    d = derive(log_n, b)
    for k in range(d.K):
        assert pr.block_bytes(k) == d.blocks[k], f"block {k}"


@pytest.mark.parametrize("log_n,b", CASES)
def test_every_proof_byte_for_byte(log_n, b):
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    d = derive(log_n, b)
    for i in range(pp.N):
        assert pr.proof(i) == d.proof(i), f"proof {i}"


MUTATIONS = [
    Reading(int_order="little"),
    Reading(node_swap=True),
    Reading(x0_zero=True),
    Reading(stmt_no_counts=True),
    Reading(stmt_rows_flat=True),
    Reading(stmt_odd_dup=True),
    Reading(z_without_x=True),
    Reading(path_root_first=True),
    Reading(rho_tag="FP-r"),
]


@pytest.mark.parametrize("rd", MUTATIONS, ids=lambda r: ",".join(
    f"{f.name}={getattr(r, f.name)}" for f in dataclasses.fields(r) if getattr(r, f.name) != f.default))
def test_a_changed_reading_is_detected(rd):
    """One reading changed: the re-derived proofs must no longer all equal the oracle's."""
    log_n, b = 4, 3
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    d = derive(log_n, b, rd)
    assert any(pr.proof(i) != d.proof(i) for i in range(pp.N))


@pytest.mark.parametrize("log_n,b", CASES)
def test_state_export_layout(log_n, b):
    """The oracle's whole-state export (the layout the GPU library's state export shares) holds the
    re-derived block records, Merkle trees level by level, r_j, every fold-tree node and the PST
    quotient commitments, in the documented order."""
    from tests import _state
    pp, m, C, rows, pr, beta, tau = case(log_n, b)
    d = derive(log_n, b)
    st = _state.split(pr.state(), pp.R, pp.M, d.K, d.lr)
    assert st["blocks"] == b"".join(d.blocks)
    assert st["row_trees"] == b"".join(b"".join(b"".join(lv) for lv in t) for t in d.row_trees)
    assert st["top_tree"] == b"".join(b"".join(lv) for lv in d.top)
    assert st["r_j"] == b"".join(v.to_bytes(32, "big") for v in d.rj)
    nodes = [(h, s) for h in range(d.lr + 1) for s in range(pp.R >> h)]
    assert st["D_w"] == b"".join(d.D(h, s) for h, s in nodes)
    assert st["g_w"] == b"".join(v.to_bytes(32, "big") for h, s in nodes for v in d.g[h][s])
    pst = b""
    for t in range(d.lc):
        w = 1 << t
        for p in range(pp.M >> (t + 1)):
            Q = [(d.gstar[(2 * p + 1) * w + c] - d.gstar[2 * p * w + c]) % RR for c in range(w)]
            pst += d.grp.G1(mle_eval(Q, d.tau[:t]) if t else Q[0])
    assert st["pst"] == pst
