"""Multiplication in all modes but one (Sec. 2.5): B = A x_1 X ... x_{m-1} X, mode 0
untransformed, returned in its partially symmetric block storage.  Pinned on the
CPU by emulating the library's level plans (levels 0 .. m-2) against the oracle's
dense chain with the identity on mode 0; on the GPU, every level kernel path
against the same oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import all_but_one_storage, colex_tuples, rel_fro


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def oracle_all_but_one(A, X, m):
    """Dense B = A x_1 X ... x_{m-1} X as an n x p x ... x p array (the oracle's
    chain with the identity on mode 0; its output is in dimensional order)."""
    p, n = X.shape
    B = oracle.ttm_chain(A, [np.eye(n)] + [X] * (m - 1), m)
    return B.reshape((n,) + (p,) * (m - 1), order="F")


def test_colex_enumeration_matches_rank_formula():
    """The pure-Python colex enumeration used by the layout map agrees with
    rank = sum_t C(s_t + t, t + 1) (the block order of Sec. 3.3's picture)."""
    from math import comb
    for L, nb in [(1, 5), (2, 4), (3, 3), (4, 3)]:
        for r, t in enumerate(colex_tuples(L, nb)):
            assert sum(comb(t[k] + k, k + 1) for k in range(L)) == r


def test_sizes(st):
    from math import comb
    for m, n, p, b in [(3, 24, 24, 8), (4, 13, 9, 4), (2, 10, 7, 3), (5, 7, 6, 2)]:
        nbar, pbar = -(-n // b), -(-p // b)
        assert st.sttsm_all_but_one_elems(m, n, p, b) == comb(pbar + m - 2, m - 1) * nbar * b ** m
        f = st.sttsm_all_but_one_flops(m, n, p, b)
        full = st.sttsm_flops(m, n, p, b)
        last = 2 * nbar * b ** (m + 1) * comb(pbar + m - 1, m)
        assert abs(full - f - last) <= 1e-9 * full
    assert st.sttsm_all_but_one_elems(1, 10, 10, 2) == -1


CPU_CASES = [(3, 24, 24, 8), (2, 9, 11, 3), (4, 13, 9, 4), (3, 17, 5, 6), (5, 7, 6, 2)]


@pytest.mark.parametrize("m,n,p,b", CPU_CASES)
def test_layout_emulated_levels_match_oracle(st, m, n, p, b):
    from test_plan_emulation import emulate
    A = synth.sym_uniform_dense(m, n, 11)
    X = synth.x_gaussian(12, p, n)
    T = emulate(st, m, n, p, b, st.STTSM_FP64, oracle.bcss_pack(A, m, n, b), X, nlev=m - 1)
    ref = all_but_one_storage(oracle_all_but_one(A, X, m), m, n, p, b)
    assert T.size == ref.size == st.sttsm_all_but_one_elems(m, n, p, b)
    assert np.linalg.norm(T - ref) <= 1e-12 * np.linalg.norm(ref)


GPU_CASES = [(3, 24, 24, 8), (2, 130, 70, 32), (3, 100, 90, 16), (3, 96, 96, 32), (3, 100, 100, 48),
             (4, 70, 40, 16), (4, 20, 12, 5), (5, 16, 16, 8)]


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,p,b", GPU_CASES)
@pytest.mark.parametrize("precname", ["fp64", "bf16x6"])
def test_all_but_one_matches_oracle(st, m, n, p, b, precname):
    torch = pytest.importorskip("torch")
    from helpers import device_bcss_from_dense, xcol
    prec = st.STTSM_FP64 if precname == "fp64" else st.STTSM_BF16X6
    dt = torch.float64 if precname == "fp64" else torch.float32
    A = synth.sym_uniform_dense(m, n, 21 + m)
    X = synth.x_gaussian(22 + n, p, n)
    if precname != "fp64":
        X = X.astype(np.float32).astype(np.float64)
    Ab = device_bcss_from_dense(st, A, m, n, b, dt)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=dt)
    T = torch.full((st.sttsm_all_but_one_elems(m, n, p, b),), float("nan"), dtype=dt, device="cuda")
    st.sttsm_bcss_all_but_one(Ab, dX, m, n, p, b, T, prec, st.workspace_tensor(m, n, p, b, prec))
    torch.cuda.synchronize()
    got = T.double().cpu().numpy()
    assert not np.isnan(got).any()
    ref = all_but_one_storage(oracle_all_but_one(A, X, m), m, n, p, b)
    assert rel_fro(got, ref) <= (1e-12 if precname == "fp64" else 1e-6)
    assert st.sttsm_device_status() == 0
