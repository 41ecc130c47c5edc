"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point the header declares, and its BCSS indexing and cost model
agree with the oracle's independent enumeration."""
import itertools
import math
import re
from pathlib import Path

import numpy as np
import pytest

import oracle

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    pkg._load()
    return pkg


def declared_functions():
    names = []
    for hdr in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", hdr.read_text(), flags=re.S)
        for m in re.finditer(r"^\s*(?:int64_t|int|double|void)\s+\**(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return names


def test_library_exports_every_declared_symbol(st):
    import ctypes
    lib = ctypes.CDLL(str(st.lib_path()))
    names = declared_functions()
    assert "sttsm_bcss" in names and "bcss_pack" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(st.exported_symbols()) == set(names)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_block_counts(st, m):
    for n, b in [(24, 8), (25, 8), (7, 3), (16, 16), (5, 1)]:
        nbar = -(-n // b)
        assert st.bcss_num_blocks(m, n, b) == oracle.bcss_count_blocks(m, nbar)
        assert st.bcss_num_elems(m, n, b) == b ** m * oracle.bcss_count_blocks(m, nbar)


@pytest.mark.parametrize("m,nbar", [(1, 6), (2, 5), (3, 5), (4, 4), (5, 3), (6, 3)])
def test_rank_matches_oracle_storage_order(st, m, nbar):
    """With b = 1 the oracle's BCSS storage order is the order of the stored
    tuples; encode each entry by its sorted tuple and compare with unrank."""
    n = nbar
    dense = np.empty(n ** m)
    for lin in range(n ** m):
        idx = sorted(np.unravel_index(lin, (n,) * m, order="F"))
        dense[lin] = sum(int(v) * (n + 1) ** a for a, v in enumerate(idx))
    packed = oracle.bcss_pack(dense, m, n, 1)
    for r, code in enumerate(packed):
        tup = []
        c = int(code)
        for _ in range(m):
            tup.append(c % (n + 1))
            c //= n + 1
        assert st.bcss_block_unrank(m, r) == tuple(tup)
        assert st.bcss_block_rank(tup) == r


def test_rank_rejects_unsorted(st):
    assert st.bcss_block_rank([2, 1, 3]) == -1
    assert st.bcss_block_rank([-1, 0]) == -1


@pytest.mark.parametrize("m,n,p,b", [(3, 24, 24, 8), (3, 768, 768, 64), (3, 768, 768, 32), (3, 768, 768, 48),
                                     (4, 128, 64, 8), (4, 128, 64, 16), (4, 128, 64, 32), (5, 37, 20, 4), (2, 9, 11, 3),
                                     (1, 10, 7, 4), (6, 20, 12, 8)])
def test_flops_match_oracle_count(st, m, n, p, b):
    assert st.sttsm_flops(m, n, p, b) == pytest.approx(oracle.bcss_flops(m, n, p, b), rel=1e-13)


def test_workspace_sizes(st):
    # FP64 needs the two temporaries buffers; split precisions add X pieces
    ws64 = st.sttsm_workspace_size(3, 24, 24, 8, st.STTSM_FP64)
    ws32 = st.sttsm_workspace_size(3, 24, 24, 8, st.STTSM_BF16X6)
    # level 0 output: C(pbar,1) nodes * C(nbar+1,2) blocks * b^3 ; level 1: C(pbar+1,2) * nbar * b^3
    l0 = 3 * 6 * 512
    l1 = 6 * 3 * 512
    assert ws64 >= 8 * (l0 + l1)
    assert ws32 >= 4 * (l0 + l1) + 3 * 24 * 24 * 2
    with pytest.raises(st.SttsmError) as e:
        st.sttsm_workspace_size(3, 24, 24, 8, st.STTSM_TF32X3)
    assert e.value.code == st.STTSM_ERR_UNSUPPORTED
    with pytest.raises(st.SttsmError):
        st.sttsm_workspace_size(9, 24, 24, 8, st.STTSM_FP64)
    with pytest.raises(st.SttsmError):
        st.sttsm_workspace_size(3, 0, 24, 8, st.STTSM_FP64)


def test_workspace_covers_the_tma_path(st):
    """m=3 n=p=768 b=64 BF16X6 runs on the TMA-fed kernel: the workspace must hold
    the X pieces, A as 3 BF16 pieces per entry and both temporaries as 3 pieces
    per entry (level 0 writes C(pbar,1) * C(nbar+1,2) blocks, level 1
    C(pbar+1,2) * nbar blocks of b^3 entries)."""
    m, n, p, b = 3, 768, 768, 64
    nbar = pbar = 12
    bm = b ** m
    x_pieces = 3 * (pbar * b) * (nbar * b) * 2
    a_pieces = 3 * math.comb(nbar + 2, 3) * bm * 2
    t0 = 3 * math.comb(pbar, 1) * math.comb(nbar + 1, 2) * bm * 2
    t1 = 3 * math.comb(pbar + 1, 2) * nbar * bm * 2
    ws = st.sttsm_workspace_size(m, n, p, b, st.STTSM_BF16X6)
    assert ws >= x_pieces + a_pieces + t0 + t1
    # and not wastefully more (alignment padding only)
    assert ws <= x_pieces + a_pieces + t0 + t1 + 4 * 256


def test_autotune_picks_a_candidate(st):
    for m, n, p in [(3, 20, 12), (4, 64, 40), (5, 33, 33), (3, 768, 768)]:
        cands = (4, 8, 16) if n < 100 else (32, 48, 64)
        b = st.sttsm_autotune_b(m, n, p, st.STTSM_BF16X6, cands)
        assert b in cands
    # the FP64 path minimises the Tbl. 4 flop count
    cands = (4, 8, 16)
    b = st.sttsm_autotune_b(3, 48, 48, st.STTSM_FP64, cands)
    assert b == min(cands, key=lambda c: st.sttsm_flops(3, 48, 48, c))
    with pytest.raises(st.SttsmError):
        st.sttsm_autotune_b(3, 48, 48, st.STTSM_FP64, ())


def test_batch_shapes_follow_the_workload_recipe():
    import collections
    import synth
    sh = synth.batch_shapes(3, 4096)
    cnt = collections.Counter(m for m, _, _ in sh)
    assert set(cnt) == {3, 4, 5}
    assert abs(cnt[3] / 4096 - 0.5) < 0.03 and abs(cnt[4] / 4096 - 0.3) < 0.03
    assert all(8 <= n <= 64 and 8 <= p <= n for _, n, p in sh)
    assert sh == synth.batch_shapes(3, 4096)


def test_serving_arrivals_are_poisson():
    import synth
    rq = synth.serve_requests(4, 2000.0, 5.0)
    t = np.array([r[0] for r in rq])
    assert abs(len(rq) / 5.0 - 2000) < 150 and np.all(np.diff(t) > 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() * 2000 - 1) < 0.05 and abs(gaps.std() / gaps.mean() - 1) < 0.1
    for _, m, n, p in rq:
        lo, hi = {3: (64, 512), 4: (32, 160), 5: (16, 64), 6: (8, 32)}[m]
        assert lo <= n <= hi and lo <= p <= hi


def test_measured_autotune_rejects_bad_arguments_on_the_host(st):
    import ctypes
    import numpy as np
    L = ctypes.CDLL(str(st.lib_path()))
    f = L.sttsm_autotune_b_measured
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_int, ctypes.c_void_p]
    c = np.array([16, 32], dtype=np.int32)
    assert f(3, 100, 100, st.STTSM_BF16X6, None, 2, 3, None) == st.STTSM_ERR_ARG
    assert f(3, 100, 100, st.STTSM_BF16X6, c.ctypes.data, 0, 3, None) == st.STTSM_ERR_ARG
    assert f(3, 100, 100, st.STTSM_BF16X6, c.ctypes.data, 2, 0, None) == st.STTSM_ERR_ARG
    assert f(3, 100, 100, st.STTSM_TF32X3, c.ctypes.data, 2, 3, None) == st.STTSM_ERR_UNSUPPORTED


@pytest.mark.parametrize("m,n,p,b", [(3, 24, 24, 8), (3, 768, 768, 64), (3, 768, 768, 32), (3, 768, 768, 48),
                                     (4, 128, 64, 8), (4, 128, 64, 16), (4, 128, 64, 32), (5, 37, 20, 4),
                                     (2, 9, 11, 3), (1, 10, 7, 4), (6, 20, 12, 8), (3, 320, 320, 32)])
@pytest.mark.parametrize("precname", ["fp64", "bf16x6", "bf16x6_r64"])
def test_work_list_issues_the_table4_count(st, m, n, p, b, precname):
    """The multiply-adds the emitted tiles cover (valid rows x columns x n̄ b, times
    2), summed over every tile of every level, equal the oracle's loop-counted
    Tbl. 4 flop count exactly: the work list neither drops nor repeats work."""
    prec = {"fp64": st.STTSM_FP64, "bf16x6": st.STTSM_BF16X6, "bf16x6_r64": st.STTSM_BF16X6_R64}[precname]
    nbar = -(-n // b)
    total = 0
    for d in range(m):
        tiles, _, info = st.sttsm_plan_level(m, n, p, b, prec, d)
        rows = np.minimum(info["BM"], info["rows_per_parent"] - tiles[:, 3].astype(np.int64))
        rows = np.where(tiles[:, 6] == 1, 128, rows)    # tiles of 16 x 8 rows are always full
        assert (rows > 0).all()
        total += int(2 * (rows * tiles[:, 5].astype(np.int64)).sum()) * nbar * b
    assert total == int(oracle.bcss_flops(m, n, p, b))
