"""Comparison of the whole shared OpenAll state (the GPU library's state export against the oracle's),
part by part, so that a mismatch names the part and the first differing entry."""
from __future__ import annotations


def split(state: bytes, R: int, M: int, K: int, log_r: int) -> dict:
    blen = 1344 * log_r + 480
    sizes = [("blocks", K * blen), ("row_trees", R * (2 * M - 1) * 32), ("top_tree", (2 * R - 1) * 32),
             ("r_j", R * 32), ("D_w", (2 * R - 1) * 96), ("g_w", (2 * R - 1) * M * 32), ("pst", (M - 1) * 96)]
    out, off = {}, 0
    for name, n in sizes:
        out[name] = state[off:off + n]
        off += n
    assert off == len(state), (off, len(state))
    out["blen"] = blen
    return out


def _first_diff(a: bytes, b: bytes, unit: int) -> int:
    for q in range(0, min(len(a), len(b)), unit):
        if a[q:q + unit] != b[q:q + unit]:
            return q // unit
    return -1


def assert_equal(got: bytes, exp: bytes, R: int, M: int, K: int, log_r: int, blocks=None) -> None:
    """Every part equal; block records only for `blocks` (all when None), the ones the oracle ran."""
    g, e = split(got, R, M, K, log_r), split(exp, R, M, K, log_r)
    blen = g["blen"]
    for k in (range(K) if blocks is None else blocks):
        assert g["blocks"][k * blen:(k + 1) * blen] == e["blocks"][k * blen:(k + 1) * blen], f"block record {k}"
    units = {"row_trees": 32, "top_tree": 32, "r_j": 32, "D_w": 96, "g_w": 32, "pst": 96}
    for name, u in units.items():
        assert g[name] == e[name], f"{name}: first differing entry {_first_diff(g[name], e[name], u)}"
