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
        for inst, par, cb, row0, col0, ncols, order16x8, _ in tiles:
            assert inst == 0 and 0 <= par < info["nodes_parent"] and 0 < ncols
            t = np.arange(BM)
            # TMA-fed tiles of 16 fastest x 8 next rows (pad0 = 1), else consecutive rows
            g = row0 + (t % 16 + b * (t // 16) if order16x8 else t)
            if order16x8:
                assert BM == 128 and (row0 % R) % b % 16 == 0 and g.max() // R == row0 // R
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


CASES = [(3, 96, 96, 48), (3, 150, 100, 48), (3, 24, 24, 8), (1, 10, 7, 4), (2, 9, 11, 3), (3, 17, 5, 6), (4, 13, 9, 4), (5, 7, 6, 2), (4, 20, 12, 5),
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


def emulate_pair(st, m, n, p, b, parent, X):
    """The fused last two levels as the pair kernel addresses them: for every unit
    (J, trailing tuples s0 .. s0 + G_s - 1) gather the level m-2 rows through
    level m-2's G and offsets, form U = rows x X^T over all children of J, then
    C[(jb0, jb1, J)][j0 + b j1 + b^2 s] = sum_i0 X[j0g, i0g] U[i0g, j1g, s]."""
    nbar, pbar = -(-n // b), -(-p // b)
    Kt = nbar * b
    Xpad = np.zeros((pbar * b, Kt))
    Xpad[:p, :n] = X
    units, Gs = st.sttsm_plan_pair(m, n, p, b)
    _, G, info = st.sttsm_plan_level(m, n, p, b, st.STTSM_BF16X6, m - 2)
    k, R, bm, P_par, P_out = info["k"], info["R"], info["bm"], info["P_parent"], info["P_out"]
    assert k == 1 and P_out == nbar
    OFF = G[P_out * nbar:].reshape(k + 1, R)
    G = G[: P_out * nbar].reshape(P_out, nbar)
    S_total = R // b
    assert ((Kt + 3) // 4 * 4) * Gs <= 128
    nC = st.bcss_num_elems(m, p, b)
    C = np.zeros(nC)
    count = np.zeros(nC, dtype=np.int64)
    kk = np.arange(Kt)
    ib, a = kk // b, kk % b
    for inst, par, _, s0, children, gs, cbase, _ in units:
        assert inst == 0 and gs == Gs and 0 <= par < info["nodes_parent"]
        s = s0 + np.arange(Gs)
        s = s[s < S_total]
        i0g = np.arange(Kt)
        pr = np.repeat(i0g // b, s.size).reshape(Kt, s.size)
        rr = (i0g % b)[:, None] + b * s[None, :]
        gq = G[pr[..., None], ib[None, None, :]]
        q, rank = gq & 7, gq >> 3
        off = OFF[q, rr[..., None]] + a[None, None, :] * b ** q
        idx = (par * P_par + rank) * bm + off
        assert idx.min() >= 0 and idx.max() < parent.size
        rows = parent[idx]                                   # [i0g, s, kk]
        NA = children * b
        U = np.einsum("isk,jk->ijs", rows, Xpad[:NA])          # [i0g, j1g, s]
        for jb1 in range(children):
            for j1 in range(b):
                Cv = Xpad[: (jb1 + 1) * b] @ U[:, jb1 * b + j1, :]   # [j0g, s]
                j0g = np.arange((jb1 + 1) * b)
                node = cbase + jb1 * (jb1 + 1) // 2 + j0g // b
                cidx = node[:, None] * bm + (j0g % b)[:, None] + b * j1 + b * b * s[None, :]
                assert cidx.min() >= 0 and cidx.max() < nC
                C[cidx] = Cv
                np.add.at(count, cidx.reshape(-1), 1)
    assert np.all(count == 1), "every C entry is written exactly once"
    return C


PAIR_CASES = [(3, 24, 24, 8), (2, 9, 11, 3), (3, 17, 5, 6), (4, 13, 9, 4), (5, 7, 6, 2), (4, 20, 12, 5),
              (3, 40, 40, 4), (3, 40, 12, 1), (2, 30, 20, 1), (4, 21, 21, 7), (5, 16, 16, 8), (6, 6, 5, 2),
              (3, 64, 48, 16), (3, 5, 3, 8), (3, 1, 6, 4), (4, 5, 1, 2)]


@pytest.mark.parametrize("m,n,p,b", PAIR_CASES)
def test_fused_pair_emulation_matches_oracle(st, m, n, p, b):
    A = synth.sym_uniform_dense(m, n, 17)
    X = synth.x_gaussian(18, p, n)
    A_bcss = oracle.bcss_pack(A, m, n, b)
    parent = A_bcss if m == 2 else emulate(st, m, n, p, b, st.STTSM_BF16X6, A_bcss, X, nlev=m - 2)
    C_emu = emulate_pair(st, m, n, p, b, parent, X)
    C_ref = oracle.bcss_pack(oracle.sttsm_chain(A, X, m), m, p, b)
    assert np.linalg.norm(C_emu - C_ref) <= 1e-12 * np.linalg.norm(C_ref)


def test_fused_pair_only_for_short_shapes(st):
    with pytest.raises(st.SttsmError) as e:
        st.sttsm_plan_pair(3, 96, 96, 32)
    assert e.value.code == st.STTSM_ERR_UNSUPPORTED
    with pytest.raises(st.SttsmError):
        st.sttsm_plan_pair(3, 40, 90, 4)          # p-bar b > 64
    with pytest.raises(st.SttsmError):
        st.sttsm_plan_pair(1, 10, 7, 4)           # one level: nothing to fuse


def test_order16x8_only_where_runs_misalign(st):
    """Tiles of 16 fastest x 8 next rows appear exactly at the TMA-fed levels of the
    16-wide slice form whose runs of b^q rows (q >= 1) neither divide 128 nor are
    multiples of it: b = 48 at levels 0 and 1 of m = 3, not at its last level and
    not for b = 16, 32 or 64."""
    for (m, n, p, b), want in (((3, 96, 96, 48), [1, 1, 0]), ((3, 96, 96, 16), [0, 0, 0]),
                               ((3, 96, 96, 32), [0, 0, 0]), ((3, 130, 130, 64), [0, 0, 0])):
        got = [int(st.sttsm_plan_level(m, n, p, b, st.STTSM_BF16X6, d)[0][:, 6].max()) for d in range(m)]
        assert got == want, (m, n, p, b, got)
    # the FP64 path keeps consecutive rows
    assert st.sttsm_plan_level(3, 96, 96, 48, st.STTSM_FP64, 0)[0][:, 6].max() == 0
