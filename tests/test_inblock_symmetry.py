"""In-block symmetry (canonical entries of diagonal blocks only) on the CPU.

T^(k) is symmetric in its k leading modes and in its m - k trailing modes
(Sec. 5.3), so inside a stored block an entry equals the one whose full
indices are non-decreasing within each group.  These tests check, without a
GPU, the plan of the mode that computes those canonical entries only:

* the library's canonical-row map equals the canonical rows written out from
  that definition (sorted tuples of full indices), each exactly once;
* an FP64 emulation of every tile of every level, addressed as the kernel
  addresses it, writes exactly the canonical entries of every temporary,
  reads only entries that were written (each operand at its canonical
  position), copies each canonical entry of the result to the positions it
  equals by symmetry (every entry exactly once) and gives the oracle's C;
* the canonical entries computed per level times 2 n are the minimum flop
  count the paper prints for storing no entry twice (Sec. 6, "analysis
  relative to minimum"), when b divides n and p.
"""
import itertools
from math import comb

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


@pytest.fixture()
def sym_on(st):
    st.sttsm_set_inblock_symmetry(True)
    try:
        yield
    finally:
        st.sttsm_set_inblock_symmetry(False)


def sorted_tuples(nvals, length):
    """Non-decreasing tuples over [0, nvals) in BCSS storage (colex) order: the last entry slowest."""
    out = [tuple(sorted(c, reverse=False)) for c in itertools.combinations_with_replacement(range(nvals), length)]
    return sorted(out, key=lambda s: tuple(reversed(s)))


def canonical_rows(m, n, p, b, d, u):
    """Rows pr * b^(m-1) + rr of level d (k = m - 1 - d) whose full i indices are
    non-decreasing and whose trailing j offsets are non-decreasing where the
    parent's blocks u repeat, written out from the definition."""
    k = m - 1 - d
    nbar = -(-n // b)
    R = b ** (m - 1)
    rows = set()
    prefixes = sorted_tuples(nbar, k) if k > 0 else [()]
    for pr, I in enumerate(prefixes):
        for ri in itertools.product(range(b), repeat=k):
            x = [I[t] * b + ri[t] for t in range(k)]
            if any(x[t] > x[t + 1] for t in range(k - 1)):
                continue
            for sj in itertools.product(range(b), repeat=d):
                y = [u[t] * b + sj[t] for t in range(d)]
                if any(y[t] > y[t + 1] for t in range(d - 1)):
                    continue
                rr = sum(ri[t] * b ** t for t in range(k)) + b ** k * sum(sj[t] * b ** t for t in range(d))
                rows.add(pr * R + rr)
    return rows


ROW_CASES = [(3, 12, 12, 4), (3, 10, 7, 3), (4, 8, 8, 2), (4, 9, 6, 4), (2, 16, 20, 8), (5, 6, 6, 2),
             (3, 16, 16, 16), (1, 8, 5, 4), (4, 4, 4, 4)]


@pytest.mark.parametrize("m,n,p,b", ROW_CASES)
def test_sym_rows_are_the_canonical_rows(st, m, n, p, b):
    pbar = -(-p // b)
    for d in range(m):
        parents = sorted_tuples(pbar, d) if d > 0 else [()]
        for par, u in enumerate(parents):
            g, tie, rows = st.sttsm_plan_sym_rows(m, n, p, b, d, par)
            want = canonical_rows(m, n, p, b, d, u)
            assert rows == len(want) == len(g)
            assert len(set(g.tolist())) == rows and set(g.tolist()) == want
            # past the end: -1
            g2, _, _ = st.sttsm_plan_sym_rows(m, n, p, b, d, par, rows, 3)
            assert (g2 == -1).all()
            # tie bits: trailing modes k+1+t and k+2+t hold the same parent block
            k = m - 1 - d
            for t in range(d - 1):
                assert (((tie >> (k + 1 + t)) & 1) == int(u[t] == u[t + 1])).all()


def test_sym_rows_reject_long_contractions(st):
    with pytest.raises(st.SttsmError):
        st.sttsm_plan_sym_rows(3, 96, 96, 32, 0, 0)      # nbar b = 96 > 64
    with pytest.raises(st.SttsmError):
        st.sttsm_plan_sym_rows(3, 12, 12, 4, 1, 99)      # no such parent


def runs(blocks, lo, hi):
    """Maximal runs [a, z) of equal blocks inside modes lo .. hi-1."""
    out, a = [], lo
    while a < hi:
        z = a + 1
        while z < hi and blocks[z] == blocks[a]:
            z += 1
        out.append((a, z))
        a = z
    return out


def mirrors(o, blocks, k):
    """Offsets equal to the canonical entry o by symmetry: distinct permutations of o
    inside every run of equal blocks within the i group (modes < k) and the j group."""
    groups = runs(blocks, 0, k) + runs(blocks, k, len(o))
    per_run = [sorted(set(itertools.permutations(o[a:z]))) for a, z in groups]
    for choice in itertools.product(*per_run):
        out = []
        for part in choice:
            out.extend(part)
        yield out


def emulate_sym(st, m, n, p, b, A_bcss, X, nlev=None):
    """Every level from the library's plan in the in-block-symmetry mode, addressed as the
    kernel addresses it: tile rows are canonical rows (sttsm_plan_sym_rows); each
    operand entry is read at its canonical position (the contraction offset sorted into
    the run of equal parent blocks it joins) and must have been written; a temporary
    gets its canonical entries only (the diagonal child's columns past the offset of
    mode k+1 dropped), each exactly once; the last level (the result) copies each
    canonical entry to its mirrors, covering every entry exactly once.
    Returns (result, canonical entries computed per level, issued multiply-adds)."""
    nlev = m if nlev is None else nlev
    nbar, pbar = -(-n // b), -(-p // b)
    Kp, Pp = nbar * b, pbar * b
    Xpad = np.zeros((Pp, Kp))
    Xpad[:p, :n] = X
    parent = A_bcss
    written = np.ones(A_bcss.size, dtype=bool)      # A holds every entry
    canon_per_level, issued = [], 0
    for d in range(nlev):
        last = d == nlev - 1
        tiles, G, info = st.sttsm_plan_level(m, n, p, b, st.STTSM_BF16X6, d)
        assert (tiles[:, 6] & 3 == 2).all(), "every tile of the level is in the symmetry mode"
        k, R, bm = info["k"], info["R"], info["bm"]
        P_par, P_out, BM = info["P_parent"], info["P_out"], info["BM"]
        out = np.zeros(info["nodes_out"] * P_out * bm)
        count = np.zeros(out.size, dtype=np.int64)
        OFF = G[P_out * nbar:].reshape(k + 1, R)
        G = G[: P_out * nbar].reshape(P_out, nbar)
        prefixes = sorted_tuples(nbar, k) if k > 0 else [()]
        parents = sorted_tuples(pbar, d) if d > 0 else [()]
        canon = 0
        for inst, par, cb, row0, col0, ncols, pad0, pad1 in tiles:
            u = parents[par]
            assert (pad0 >> 16) == (u[0] if d > 0 else 0)
            g, tie, rows = st.sttsm_plan_sym_rows(m, n, p, b, d, int(par), int(row0), BM)
            assert rows == pad1
            g = g[g >= 0]
            assert g.size > 0
            issued += g.size * int(ncols) * Kp
            ops = np.zeros((g.size, Kp))
            for i, gi in enumerate(g):
                pr, rr = divmod(int(gi), R)
                I = prefixes[pr]
                io = [(rr // b ** t) % b for t in range(k)]
                for ib in range(nbar):
                    q, rank = int(G[pr, ib]) & 7, int(G[pr, ib]) >> 3
                    e = 0
                    while q + e < k and I[q + e] == ib:
                        e += 1
                    for a in range(b):
                        # the run's offsets with a sorted in: modes q .. q+e
                        vals = sorted([a] + io[q:q + e])
                        off = OFF[q, rr] - sum(io[q + t] * b ** (q + 1 + t) for t in range(e))
                        off += sum(vals[t] * b ** (q + t) for t in range(e + 1))
                        idx = (par * P_par + rank) * bm + off
                        assert written[idx], "an operand entry that was never written"
                        ops[i, ib * b + a] = parent[idx]
            T = ops @ Xpad[col0 + np.arange(ncols), :].T
            for i, gi in enumerate(g):
                pr, rr = divmod(int(gi), R)
                I = prefixes[pr]
                digits = [(rr // b ** t) % b for t in range(m - 1)]
                for e in range(ncols):
                    cc = col0 + e
                    jb, c = cc // b, cc % b
                    o = digits[:k] + [c] + digits[k:]
                    blocks = list(I) + [jb] + list(u)
                    if d > 0 and jb == u[0] and c > o[k + 1]:
                        continue            # not canonical: another row's entry
                    canon += 1
                    base = ((cb + jb) * P_out + pr) * bm
                    for o2 in (mirrors(o, blocks, k) if last else [o]):
                        idx = base + sum(o2[t] * b ** t for t in range(m))
                        out[idx] = T[i, e]
                        count[idx] += 1
        assert count.max() == 1, "no entry is written twice"
        if last:
            assert np.all(count == 1), "the mirrors of the canonical entries cover every entry"
        else:
            assert count.sum() == canon == comb(Kp + k - 1, k) * comb(Pp + m - k - 1, m - k)
        canon_per_level.append(canon)
        parent, written = out, count == 1
    return parent, canon_per_level, issued


SYM_CASES = [(3, 12, 12, 4), (3, 10, 7, 3), (4, 8, 8, 2), (4, 9, 6, 4), (2, 16, 20, 8), (5, 6, 6, 2),
             (3, 8, 8, 8), (1, 8, 5, 4), (3, 9, 13, 4), (4, 6, 10, 3)]


@pytest.mark.parametrize("m,n,p,b", SYM_CASES)
def test_sym_emulation_matches_oracle(st, sym_on, m, n, p, b):
    A = synth.sym_uniform_dense(m, n, 11)
    X = synth.x_gaussian(12, p, n)
    A_bcss = oracle.bcss_pack(A, m, n, b)
    C_emu, _, _ = emulate_sym(st, m, n, p, b, A_bcss, X)
    C_ref = oracle.bcss_pack(oracle.sttsm_chain(A, X, m), m, p, b)
    assert np.linalg.norm(C_emu - C_ref) <= 1e-12 * np.linalg.norm(C_ref)


def minimum_flops(m, n, p):
    """Sec. 6 ("analysis relative to minimum"): computing the unique entries only,
    2 n sum_{d=0}^{m-1} C(n + d, d + 1) C(n + m - d - 2, m - d - 1) for p = n; with
    p != n the d + 1 produced modes range over p."""
    return 2 * n * sum(comb(p + d, d + 1) * comb(n + m - d - 2, m - d - 1) for d in range(m))


@pytest.mark.parametrize("m,n,p,b", [(3, 12, 12, 4), (4, 8, 8, 2), (5, 6, 6, 2), (3, 8, 8, 8), (3, 8, 12, 4),
                                     (4, 8, 4, 4), (2, 16, 16, 8)])
def test_sym_work_is_the_paper_minimum(st, sym_on, m, n, p, b):
    """b divides n and p: the canonical entries of each level are the unique entries of
    T^(k), and 2 n per entry gives the paper's minimum; the issued multiply-adds (all
    columns of every canonical row) lie between it and the Tbl. 4 count."""
    A = synth.sym_uniform_dense(m, n, 3)
    X = synth.x_gaussian(4, p, n)
    _, canon, issued = emulate_sym(st, m, n, p, b, oracle.bcss_pack(A, m, n, b), X)
    for d, c in enumerate(canon):
        k = m - 1 - d
        assert c == comb(n + k - 1, k) * comb(p + m - k - 1, m - k)
    assert 2 * n * sum(canon) == minimum_flops(m, n, p)
    if p == n:
        # the printed form, p = n
        assert minimum_flops(m, n, n) == 2 * n * sum(comb(n + d, d + 1) * comb(n + m - d - 2, m - d - 1)
                                                     for d in range(m))
    assert minimum_flops(m, n, p) <= 2 * issued <= int(oracle.bcss_flops(m, n, p, b))


def test_minimum_formula_small_case_by_brute_force():
    """The minimum count on a tiny case, counted by listing the unique entries of every
    temporary T^(k) (k sorted i indices over n, m - k sorted j indices over p)."""
    m, n, p = 3, 4, 3
    total = 0
    for k in range(m):
        ui = len(list(itertools.combinations_with_replacement(range(n), k)))
        uj = len(list(itertools.combinations_with_replacement(range(p), m - k)))
        total += 2 * n * ui * uj
    assert total == minimum_flops(m, n, p)


def test_switch_changes_only_short_contractions(st, sym_on):
    """Shapes whose contraction is longer than 64, the FP64 path and orders above 5
    keep the full tiles."""
    tiles, _, _ = st.sttsm_plan_level(3, 96, 96, 32, st.STTSM_BF16X6, 1)
    assert (tiles[:, 6] & 3 != 2).all()
    tiles, _, _ = st.sttsm_plan_level(3, 12, 12, 4, st.STTSM_FP64, 1)
    assert (tiles[:, 6] == 0).all()
    # orders above 5 keep the full tiles (a row could have more than 4! mirrors)
    tiles, _, _ = st.sttsm_plan_level(6, 8, 8, 4, st.STTSM_BF16X6, 2)
    assert (tiles[:, 6] & 3 != 2).all()
    with pytest.raises(st.SttsmError):
        st.sttsm_plan_sym_rows(6, 8, 8, 4, 0, 0)
    with pytest.raises(st.SttsmError):
        st.sttsm_set_inblock_symmetry(2)


@pytest.mark.parametrize("m,n,p,b", [(3, 12, 12, 4), (4, 9, 6, 4), (5, 6, 6, 2)])
def test_sym_emulation_all_but_one(st, sym_on, m, n, p, b):
    """All modes but one: the result T^(1) (level m-2) gets every entry, the
    temporaries before it their canonical entries only."""
    from helpers import all_but_one_storage
    A = synth.sym_uniform_dense(m, n, 13)
    X = synth.x_gaussian(14, p, n)
    T1, _, _ = emulate_sym(st, m, n, p, b, oracle.bcss_pack(A, m, n, b), X, nlev=m - 1)
    B = oracle.ttm_chain(A, [np.eye(n)] + [X] * (m - 1), m).reshape((n,) + (p,) * (m - 1), order="F")
    ref = all_but_one_storage(B, m, n, p, b)
    assert np.linalg.norm(T1 - ref) <= 1e-12 * np.linalg.norm(ref)
