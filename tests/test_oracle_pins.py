"""Pins for the FP64 oracle: each check is fixed by the paper or by mathematics,
never by the oracle itself (nor by the GPU library, which is not imported here).

Paper: Schatz, Low, van de Geijn, Kolda, arXiv 1301.7744.
"""
import itertools
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
import synth

GOLDEN = Path(__file__).resolve().parent / "golden"


def nd(a, m, n):
    return np.asarray(a).reshape((n,) * m, order="F")


def flat(t):
    return np.asarray(t).reshape(-1, order="F")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def closed_form_rank_r(lams, vecs, X, m):
    """[sum_r lam_r a_r^{(x)m}; X, ..., X] = sum_r lam_r (X a_r)^{(x)m} (multilinearity)."""
    p = X.shape[0]
    C = np.zeros((p,) * m)
    for lam, a in zip(lams, vecs):
        y = X @ a
        t = np.array(lam, dtype=np.float64)
        for _ in range(m):
            t = np.multiply.outer(t, y)
        C = C + t
    return flat(C)


def random_symmetric(m, n, seed):
    return synth.sym_uniform_dense(m, n, seed)


# ---------------------------------------------------------------- generator

def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the Random123 library (SC'11)."""
    ctr = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint32)
    keys = [[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]]
    want = [[0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8],
            [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD],
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]]
    for c, k, w in zip(ctr, keys, want):
        assert synth.philox4x32_10(c[None], k)[0].tolist() == w


def test_symmetric_draws_are_symmetric_and_fp32_exact():
    m, n = 4, 7
    A = nd(random_symmetric(m, n, 0), m, n)
    for perm in itertools.permutations(range(m)):
        assert np.array_equal(A, np.transpose(A, perm))
    a = A.reshape(-1)
    assert np.all(np.abs(a) < 1.0)
    assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
    assert abs(a.mean()) < 0.05 and 0.3 < a.var() < 0.37   # U(-1,1): mean 0, variance 1/3


def test_gaussian_moments():
    g = synth.gaussian(1, 300, 400, 1.0)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.02


# ---------------------------------------------------------------- eq. (cob)

@pytest.mark.parametrize("m,n,p,R", [(1, 5, 3, 2), (2, 4, 6, 1), (3, 4, 3, 2), (3, 5, 5, 3), (4, 3, 4, 2)])
def test_bruteforce_rank_r_closed_form(m, n, p, R):
    vecs = synth.rank_r_factors(11 + m, R, n)
    lams = np.linspace(1.0, -0.5, R)
    X = synth.gaussian(5 + m, p, n)
    A = synth.rank_r_dense(m, n, lams, vecs)
    C = oracle.sttsm_bruteforce(A, X, m)
    assert rel(C, closed_form_rank_r(lams, vecs, X, m)) < 1e-13


def test_bruteforce_m2_is_X_A_Xt():
    """Sec. 3.1: for m = 2, [A; X, X] = X A X^T."""
    n, p = 6, 5
    A = nd(random_symmetric(2, n, 3), 2, n)
    X = synth.gaussian(4, p, n)
    C = oracle.sttsm_bruteforce(flat(A), X, 2)
    assert rel(nd(C, 2, p), X @ A @ X.T) < 1e-14


def test_bruteforce_m1_is_matvec():
    n, p = 7, 4
    a = synth.gaussian(2, n, 1)[:, 0]
    X = synth.gaussian(3, p, n)
    assert rel(oracle.sttsm_bruteforce(a, X, 1), X @ a) < 1e-15


def test_bruteforce_special_matrices():
    m, n = 3, 5
    A = random_symmetric(m, n, 9)
    # identity: C = A exactly
    assert np.array_equal(oracle.sttsm_bruteforce(A, np.eye(n), m), A)
    # diagonal: gamma_j = alpha_j prod_k d_{j_k}
    d = np.array([1.0, -2.0, 0.5, 3.0, -1.5])
    want = nd(A, m, n) * np.einsum("i,j,k->ijk", d, d, d)
    assert rel(oracle.sttsm_bruteforce(A, np.diag(d), m), flat(want)) < 1e-15
    # selection of the first p rows of I: the leading p^m sub-tensor
    p = 3
    got = nd(oracle.sttsm_bruteforce(A, np.eye(n)[:p], m), m, p)
    assert np.array_equal(got, nd(A, m, n)[:p, :p, :p])
    # permutation matrix: gamma_j = alpha_{pi(j)}
    perm = np.array([3, 0, 4, 1, 2])
    P = np.eye(n)[perm]
    got = nd(oracle.sttsm_bruteforce(A, P, m), m, n)
    assert np.array_equal(got, nd(A, m, n)[np.ix_(perm, perm, perm)])


def test_C_is_symmetric():
    """Sec. 2.5: C inherits the symmetry of A."""
    m, n, p = 3, 5, 4
    C = nd(oracle.sttsm_bruteforce(random_symmetric(m, n, 1), synth.gaussian(2, p, n), m), m, p)
    for perm in itertools.permutations(range(m)):
        assert rel(np.transpose(C, perm), C) < 1e-14


def test_homogeneity_in_X():
    m, n, p = 3, 4, 3
    A = random_symmetric(m, n, 4)
    X = synth.gaussian(6, p, n)
    assert np.array_equal(oracle.sttsm_bruteforce(A, 2.0 * X, m), 8.0 * oracle.sttsm_bruteforce(A, X, m))


# ---------------------------------------------------------------- successive mode products

def test_chain_per_mode_matrices_match_einsum():
    """App. A mode-k products with a different matrix per mode on a non-symmetric tensor."""
    n = 5
    A = synth.gaussian(1, n ** 3, 1)[:, 0]
    Xs = [synth.gaussian(2, 3, n), synth.gaussian(3, 4, n), synth.gaussian(4, 2, n)]
    got = oracle.ttm_chain(A, Xs, 3)
    want = np.einsum("abc,ia,jb,kc->ijk", nd(A, 3, n), *Xs)
    assert rel(got, flat(want)) < 1e-14


@pytest.mark.parametrize("m,n,p", [(2, 7, 5), (3, 6, 4), (3, 5, 7), (4, 4, 3), (5, 3, 3)])
def test_chain_equals_bruteforce(m, n, p):
    A = random_symmetric(m, n, 20 + m)
    X = synth.gaussian(30 + m, p, n)
    assert rel(oracle.sttsm_chain(A, X, m), oracle.sttsm_bruteforce(A, X, m)) < 1e-13


def test_chain_rank2_config1_closed_form():
    """m = 3, n = p = 24: A = a_0^{(x)3} - 0.5 a_1^{(x)3}, a_r ~ N(0,1)."""
    m, n = 3, 24
    vecs = synth.rank_r_factors(0, 2, n)
    lams = [1.0, -0.5]
    X = synth.x_gaussian(1, n, n)
    C = oracle.sttsm_chain(synth.rank_r_dense(m, n, lams, vecs), X, m)
    assert rel(C, closed_form_rank_r(lams, vecs, X, m)) < 1e-13


def test_chain_rank8_compressing_closed_form():
    """m = 4 with p < n and orthonormal rows (shape of the compressing workload)."""
    m, n, p = 4, 24, 12
    vecs = synth.rank_r_factors(7, 8, n)
    lams = np.linspace(1.0, -1.0, 8)
    X = synth.x_orthonormal_rows(3, p, n)
    assert np.allclose(X @ X.T, np.eye(p), atol=1e-13)
    C = oracle.sttsm_chain(synth.rank_r_dense(m, n, lams, vecs), X, m)
    assert rel(C, closed_form_rank_r(lams, vecs, X, m)) < 1e-13


def test_entries_equal_chain():
    m, n, p = 3, 9, 7
    A = random_symmetric(m, n, 2)
    X = synth.gaussian(3, p, n)
    C = nd(oracle.sttsm_chain(A, X, m), m, p)
    rng = np.random.default_rng(0)
    J = rng.integers(0, p, size=(40, m))
    got = oracle.sttsm_entries(A, X, m, J)
    want = C[tuple(J.T)]
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(C))


# ---------------------------------------------------------------- BCSS layout

def read_golden(name):
    rows = []
    for line in (GOLDEN / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_bcss_b1_m2_order_matches_paper_picture():
    """Sec. 3.3's element ordering of a packed upper triangle; BCSS with b = 1."""
    n = 3
    pic = read_golden("m2_element_order.txt")
    # encode each (i, j) position by a distinct value in a symmetric matrix
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            A[i, j] = A[j, i] = 10 * i + j
    packed = oracle.bcss_pack(flat(A), 2, n, 1)
    for i in range(n):
        for j in range(n):
            if pic[i][j] != ".":
                assert packed[int(pic[i][j])] == 10 * i + j


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_bcss_block_count_is_binomial(m):
    """Tbl. 1: BCSS stores C(nbar + m - 1, m) blocks."""
    for nbar in range(1, 8):
        assert oracle.bcss_count_blocks(m, nbar) == math.comb(nbar + m - 1, m)


def test_fig2_storage_ratios():
    n = 512
    for nbar, to_min, to_dense in read_golden("fig2_storage_ratios.txt"):
        nbar = int(nbar)
        b = n // nbar
        bcss = b * b * oracle.bcss_count_blocks(2, nbar)
        assert round(n * (n + 1) / 2 / bcss, 2) == float(to_min)
        assert round(n * n / bcss, 2) == float(to_dense)


@pytest.mark.parametrize("m,n,b", [(2, 7, 3), (3, 10, 4), (3, 8, 4), (4, 5, 2)])
def test_bcss_pack_blocks_and_padding(m, n, b):
    """Each stored block is the dense b^m sub-block at its sorted block index,
    blocks ordered with the last block index slowest; entries past n are zero."""
    A = nd(random_symmetric(m, n, 5), m, n)
    nbar = -(-n // b)
    pad = np.zeros((nbar * b,) * m)
    pad[(slice(0, n),) * m] = A
    tuples = sorted(itertools.combinations_with_replacement(range(nbar), m), key=lambda t: t[::-1])
    want = np.concatenate([flat(pad[tuple(slice(t[k] * b, t[k] * b + b) for k in range(m))]) for t in tuples])
    got = oracle.bcss_pack(flat(A), m, n, b)
    assert got.size == b ** m * math.comb(nbar + m - 1, m)
    assert np.array_equal(got, want)


# ---------------------------------------------------------------- cost model

def mincosts_flops(m, n, p, bA, bC):
    """Tbl. 4 (MinCosts), BCSS computation row."""
    nbar, pbar = -(-n // bA), -(-p // bC)
    s = sum(math.comb(pbar + d, d + 1) * math.comb(nbar + m - d - 2, m - d - 1) * (bC / bA) ** d for d in range(m))
    return 2 * nbar * bC * bA ** m * s


@pytest.mark.parametrize("m,n,p,b", [(2, 16, 16, 4), (3, 24, 24, 8), (3, 768, 768, 64), (3, 768, 768, 48),
                                     (4, 128, 64, 16), (5, 20, 13, 4), (6, 9, 9, 2), (3, 10, 7, 3)])
def test_flop_count_matches_mincosts_table(m, n, p, b):
    assert oracle.bcss_flops(m, n, p, b) == pytest.approx(mincosts_flops(m, n, p, b, b), rel=1e-15)


def test_flop_count_unequal_blocks():
    assert oracle.bcss_flops(3, 12, 8, 4, 2) == pytest.approx(mincosts_flops(3, 12, 8, 4, 2), rel=1e-15)


def test_flop_count_config1_value():
    assert oracle.bcss_flops(3, 24, 24, 8) == 1130496


@pytest.mark.parametrize("m,n", [(2, 5), (3, 6), (4, 7), (5, 4)])
def test_flop_count_b1_exact_identity(m, n):
    """Sec. 6.5 (b = 1, p = n): the sum collapses by the Chu-Vandermonde identity to
    2n [C(2n+m-1, m) - C(n+m-1, m)]."""
    exact = 2 * n * (math.comb(2 * n + m - 1, m) - math.comb(n + m - 1, m))
    assert oracle.bcss_flops(m, n, n, 1) == exact


def test_flop_count_fig3D_structure_m3():
    """Fig. 4 (3D): level flops 2 b n^3 ... with the executed-count column C(pbar+d, d+1);
    with b = n (one block) the algorithm is the dense chain on one block."""
    n = 8
    assert oracle.bcss_flops(3, n, n, n) == 3 * 2 * n ** 4
