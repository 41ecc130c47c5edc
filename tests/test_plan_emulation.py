"""CPU emulation of the level kernels' index maps on the library's own plans.

For every tile of every level the test gathers the A-operand rows exactly as
the kernels address them (gather table G, insertion position q, offsets
rr % b^q + b^(q+1) (rr / b^q) + a b^q), multiplies by X in FP64, and scatters
the result with the kernels' output map.  It asserts that every read and
write stays inside its buffer, that every output entry is written exactly
once, and that the final C equals the oracle's [A; X, ..., X] packed by the
oracle.  No GPU is involved.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def emulate(st, m, n, p, b, prec, A_bcss, X, nlev=None):
    """Runs levels 0 .. nlev-1 (default all m) and returns the last level's output."""
    nbar, pbar = -(-n // b), -(-p // b)
    Xpad = np.zeros((pbar * b, nbar * b))
    Xpad[:p, :n] = X
    parent = A_bcss
    for d in range(m if nlev is None else nlev):
        tiles, G, info = st.sttsm_plan_level(m, n, p, b, prec, d)
        k, R, bm = info["k"], info["R"], info["bm"]
        P_par, P_out, rows_pp, BM = info["P_parent"], info["P_out"], info["rows_per_parent"], info["BM"]
        assert R == b ** (m - 1) and bm == b ** m
        out_size = info["nodes_out"] * P_out * bm
        if d == m - 1:
            assert out_size == st.bcss_num_elems(m, p, b)
        out = np.zeros(out_size)
        count = np.zeros(out_size, dtype=np.int64)
        OFF = G[P_out * nbar:].reshape(k + 1, R)
        G = G[: P_out * nbar].reshape(P_out, nbar)
        assert np.all((G >> 3) < P_par) and np.all((G & 7) <= k)
        rrs = np.arange(R)
        for q in range(k + 1):
            assert np.array_equal(OFF[q], rrs % b ** q + b ** (q + 1) * (rrs // b ** q))
        kk = np.arange(nbar * b)
        ib, a = kk // b, kk % b
        for inst, par, cb, row0, col0, ncols, _, _ in tiles:
            assert inst == 0 and 0 <= par < info["nodes_parent"] and 0 < ncols
            g = row0 + np.arange(BM)
            g = g[g < rows_pp]
            assert g.size > 0
            pr, rr = g // R, g % R
            gq = G[pr[:, None], ib[None, :]]
            q, rank = gq & 7, gq >> 3
            bq = b ** q
            off = OFF[q, rr[:, None]] + a[None, :] * bq
            assert off.min() >= 0 and off.max() < bm
            idx = (par * P_par + rank) * bm + off
            assert idx.min() >= 0 and idx.max() < parent.size
            cols = col0 + np.arange(ncols)
            assert cols.max() < Xpad.shape[0]
            T = parent[idx] @ Xpad[cols, :].T
            jb, c = cols // b, cols % b
            bk = b ** k
            rowoff = OFF[k, rr]
            oidx = ((cb + jb)[None, :] * P_out + pr[:, None]) * bm + rowoff[:, None] + bk * c[None, :]
            assert oidx.min() >= 0 and oidx.max() < out_size
            out[oidx] = T
            np.add.at(count, oidx.reshape(-1), 1)
        assert np.all(count == 1), "every output entry is written exactly once"
        parent = out
    return parent


CASES = [(3, 24, 24, 8), (1, 10, 7, 4), (2, 9, 11, 3), (3, 17, 5, 6), (4, 13, 9, 4), (5, 7, 6, 2), (4, 20, 12, 5),
         (3, 40, 40, 4), (2, 300, 260, 64), (6, 6, 5, 2), (3, 40, 33, 1), (2, 64, 64, 1), (4, 21, 21, 7),
         (3, 5, 3, 8), (2, 3, 10, 4), (8, 3, 2, 1), (7, 4, 3, 2), (6, 5, 4, 1),
         # degenerate: one entry, n = 1 < b, p = 1, m = 1 with n = p = 1
         (3, 1, 1, 1), (3, 1, 6, 4), (4, 5, 1, 2), (2, 1, 1, 8), (1, 1, 1, 1)]


@pytest.mark.parametrize("m,n,p,b", CASES)
@pytest.mark.parametrize("precname", ["fp64", "bf16x6"])
def test_plan_emulation_matches_oracle(st, m, n, p, b, precname):
    prec = st.STTSM_FP64 if precname == "fp64" else st.STTSM_BF16X6
    A = synth.sym_uniform_dense(m, n, 7)
    X = synth.x_gaussian(8, p, n)
    A_bcss = oracle.bcss_pack(A, m, n, b)
    C_emu = emulate(st, m, n, p, b, prec, A_bcss, X)
    C_ref = oracle.bcss_pack(oracle.sttsm_chain(A, X, m), m, p, b)
    assert np.linalg.norm(C_emu - C_ref) <= 1e-12 * np.linalg.norm(C_ref)


def test_tile_columns_stay_within_x_rows(st):
    """Columns of every tile index rows of the padded X (pbar * b rows); a parent's
    columns are cut into equal widths (multiples of 16, <= 256) that cover them once."""
    m, n, p, b = 3, 768, 768, 64
    for d in range(m):
        tiles, _, info = st.sttsm_plan_level(m, n, p, b, st.STTSM_BF16X6, d)
        assert np.all(tiles[:, 4] + tiles[:, 5] <= 12 * 64)
        assert np.all(tiles[:, 5] <= 256) and np.all(tiles[:, 5] % 16 == 0) and np.all(tiles[:, 4] % 16 == 0)
        # per (parent, row0): widths differ by at most 16 apart from the last one
        key = tiles[:, 1].astype(np.int64) * (1 << 32) + tiles[:, 3]
        for k in np.unique(key)[:200]:
            w = tiles[key == k, 5]
            assert w.sum() == ((tiles[key == k, 4] + w).max()) and (len(w) == 1 or w[:-1].min() >= w.max() - 16)
