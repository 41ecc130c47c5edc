"""GPU parity of the in-block-symmetry mode (sttsm_set_inblock_symmetry).

With the mode on, short contractions (n̄ b <= 64) compute the canonical entries
of each stored block only and copy them to the rest of the block.  Checked
against the FP64 oracle at the split-precision tolerance (1e-6), for exact
symmetry of every stored block of C (each entry bitwise equal to its canonical
entry), against the full computation (rounding-level difference), and for
bit-equality between single calls, batch plans and serving.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from helpers import colex_tuples, device_bcss_from_dense, inputs, oracle_C_bcss, rel_fro, rel_max, run_sttsm, xcol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    assert torch.cuda.is_available()
    return pkg


@pytest.fixture()
def sym_on(st):
    st.sttsm_set_inblock_symmetry(True)
    try:
        yield
    finally:
        st.sttsm_set_inblock_symmetry(False)


def canonical_offsets(tup, b):
    """For every in-block offset of the stored block with sorted block tuple tup, the
    offset of its canonical entry (full indices sorted; for C all modes are one group)."""
    m = len(tup)
    off = np.arange(b ** m)
    loc = np.array([(off // b ** t) % b for t in range(m)])
    full = np.array([tup[t] * b + loc[t] for t in range(m)])
    full.sort(axis=0)
    return sum((full[t] - tup[t] * b) * b ** t for t in range(m))


def assert_blocks_symmetric(C, m, p, b):
    pbar = -(-p // b)
    bm = b ** m
    for r, tup in enumerate(colex_tuples(m, pbar)):
        if len(set(tup)) == m:
            continue               # no repeated block index: nothing to check inside
        blk = C[r * bm:(r + 1) * bm]
        assert np.array_equal(blk, blk[canonical_offsets(tup, b)]), tup


SHAPES = [(3, 24, 24, 8), (3, 12, 12, 4), (4, 16, 16, 4), (4, 13, 9, 4), (5, 12, 12, 4), (5, 9, 7, 3),
          (3, 64, 64, 16), (3, 64, 40, 16), (3, 10, 7, 3), (2, 40, 40, 8), (1, 30, 20, 8),
          (3, 5, 3, 8), (4, 32, 32, 16), (5, 16, 16, 16), (3, 17, 30, 6)]


@pytest.mark.parametrize("m,n,p,b", SHAPES)
@pytest.mark.parametrize("precname", ["bf16x6", "bf16x6_r64"])
def test_sym_single_call_matches_oracle(st, sym_on, m, n, p, b, precname):
    prec = {"bf16x6": st.STTSM_BF16X6, "bf16x6_r64": st.STTSM_BF16X6_R64}[precname]
    A, X = inputs(m, n, p, 31 + m, 32 + n, fp32=True)
    Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
    got = run_sttsm(st, Ab, X, m, n, p, b, prec)
    assert not np.isnan(got).any()
    ref = oracle_C_bcss(A, X, m, p, b)
    assert rel_fro(got, ref) <= 1e-6 and rel_max(got, ref) <= 1e-5
    assert_blocks_symmetric(got, m, p, b)
    # the full computation differs by rounding only
    st.sttsm_set_inblock_symmetry(False)
    full = run_sttsm(st, Ab, X, m, n, p, b, prec)
    st.sttsm_set_inblock_symmetry(True)
    assert rel_fro(got, full) <= 1e-6
    assert st.sttsm_device_status() == 0


def test_sym_rank_one_closed_form(st, sym_on):
    """A = a^(x)m: C = (X a)^(x)m exactly in exact arithmetic (the rank-1 closed form)."""
    m, n, p, b = 4, 20, 12, 4
    rng = np.random.default_rng(5)
    a = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    A = a
    for _ in range(m - 1):
        A = np.multiply.outer(A, a)
    A = A.reshape(-1, order="F")
    X = synth.x_gaussian(6, p, n).astype(np.float32).astype(np.float64)
    Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
    got = run_sttsm(st, Ab, X, m, n, p, b, st.STTSM_BF16X6)
    y = X @ a
    Y = y
    for _ in range(m - 1):
        Y = np.multiply.outer(Y, y)
    ref = oracle.bcss_pack(Y.reshape(-1, order="F"), m, p, b)
    assert rel_fro(got, ref) <= 1e-6


def test_sym_all_but_one_matches_full(st, sym_on):
    """T^(1) (all modes but one) in the symmetry mode equals the full computation to rounding."""
    m, n, p, b = 4, 24, 16, 8
    A, X = inputs(m, n, p, 41, 42, fp32=True)
    Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
    outs = []
    for on in (True, False):
        st.sttsm_set_inblock_symmetry(on)
        T = torch.full((st.sttsm_all_but_one_elems(m, n, p, b),), float("nan"), dtype=torch.float32, device="cuda")
        st.sttsm_bcss_all_but_one(Ab, dX, m, n, p, b, T, st.STTSM_BF16X6,
                                  st.workspace_tensor(m, n, p, b, st.STTSM_BF16X6))
        torch.cuda.synchronize()
        outs.append(T.double().cpu().numpy())
    st.sttsm_set_inblock_symmetry(True)
    assert not np.isnan(outs[0]).any()
    assert rel_fro(outs[0], outs[1]) <= 1e-6


def _batch(st, count, seed):
    insts, host = [], []
    for i, (m, n, p) in enumerate(synth.batch_shapes(seed, count)):
        n, p = min(n, 24), min(p, 24)
        b = st.sttsm_autotune_b(m, n, p, st.STTSM_BF16X6, (4, 8, 16))
        A = synth.sym_uniform_dense(m, n, 700 + i)
        X = synth.x_gaussian(800 + i, p, n).astype(np.float32).astype(np.float64)
        Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
        dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
        C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=torch.float32, device="cuda")
        insts.append((Ab, dX, C, m, n, p, b))
        host.append((A, X))
    return insts, host


@pytest.mark.parametrize("precname", ["bf16x6", "bf16x6_r64"])
def test_sym_batch_equals_single_calls(st, sym_on, precname):
    prec = {"bf16x6": st.STTSM_BF16X6, "bf16x6_r64": st.STTSM_BF16X6_R64}[precname]
    insts, host = _batch(st, 40, 9)
    plan = st.BatchPlan(insts, prec)
    ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    plan.run(ws)
    torch.cuda.synchronize()
    for i, ((Ab, dX, C, m, n, p, b), (A, X)) in enumerate(zip(insts, host)):
        got = C.double().cpu().numpy()
        Cs = torch.empty_like(C)
        st.sttsm_bcss(Ab, dX, m, n, p, b, Cs, prec, st.workspace_tensor(m, n, p, b, prec))
        torch.cuda.synchronize()
        assert np.array_equal(got, Cs.double().cpu().numpy()), i
        if i % 5 == 0:
            assert rel_fro(got, oracle_C_bcss(A, X, m, p, b)) <= 1e-6
            assert_blocks_symmetric(got, m, p, b)
    plan.destroy()


def test_sym_serving_equals_alone(st, sym_on):
    """Short-contraction requests in the symmetry mode beside long ones (TMA and gathered
    kernels, unaffected by the switch) give the bits of the same request alone."""
    shapes = [(5, 16, 16, 4), (6, 10, 8, 4), (4, 40, 30, 8), (3, 64, 64, 16), (3, 100, 90, 16), (5, 24, 20, 8),
              (4, 16, 16, 16), (3, 70, 60, 8)]
    reqs = []
    for i, (m, n, p, b) in enumerate(shapes):
        A, X = inputs(m, n, p, 900 + i, 950 + i, fp32=True)
        Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
        dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
        C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=torch.float32, device="cuda")
        reqs.append(dict(A=A, X=X, Ab=Ab, dX=dX, C=C, m=m, n=n, p=p, b=b))
    torch.cuda.synchronize()
    srv = st.Server(4 << 30)
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
    t0 = time.time()
    done = set()
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done and srv.poll(t)[0]:
                done.add(t)
        assert time.time() - t0 < 120.0
        time.sleep(0.001)
    srv.destroy()
    for r in reqs:
        got = r["C"].double().cpu().numpy()
        alone = run_sttsm(st, r["Ab"], r["X"], r["m"], r["n"], r["p"], r["b"], st.STTSM_BF16X6)
        assert np.array_equal(got, alone), (r["m"], r["n"], r["b"])
        assert rel_fro(got, oracle_C_bcss(r["A"], r["X"], r["m"], r["p"], r["b"])) <= 1e-6


def test_sym_batch_config_shapes_sampled(st, sym_on):
    """Full-size batch shapes (m up to 5, n up to 64): 64 seeded C entries per sampled
    instance against the oracle's entry contraction, and exact in-block symmetry."""
    insts, host = [], []
    shapes = [(5, 64, 60, 16), (5, 48, 40, 8), (4, 64, 64, 16), (3, 64, 50, 4)]
    for i, (m, n, p, b) in enumerate(shapes):
        A, X = inputs(m, n, p, 1000 + i, 1100 + i, fp32=True)
        Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
        dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
        C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=torch.float32, device="cuda")
        insts.append((Ab, dX, C, m, n, p, b))
        host.append((A, X))
    plan = st.BatchPlan(insts, st.STTSM_BF16X6)
    ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    plan.run(ws)
    torch.cuda.synchronize()
    plan.destroy()
    rng = np.random.default_rng(17)
    for (Ab, dX, C, m, n, p, b), (A, X) in zip(insts, host):
        got = C.double().cpu().numpy()
        assert not np.isnan(got).any()
        pbar = -(-p // b)
        tups = colex_tuples(m, pbar)
        J = np.sort(rng.integers(0, p, size=(64, m)), axis=1)
        ref = oracle.sttsm_entries(A, X, m, J)
        pos = [tups.index(tuple(int(v) // b for v in j)) * b ** m + sum((int(j[t]) % b) * b ** t for t in range(m))
               for j in J]
        assert rel_max(got[pos], ref) <= 1e-5
        # exact symmetry on the diagonal blocks of a few sampled tuples
        for tup in [t for t in tups if len(set(t)) < m][:6]:
            r = tups.index(tup)
            blk = got[r * b ** m:(r + 1) * b ** m]
            assert np.array_equal(blk, blk[canonical_offsets(tup, b)])
