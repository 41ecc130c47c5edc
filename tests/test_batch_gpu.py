"""Batches of independent instances (different m, n, p, b) in one graph-captured
launch sequence: every instance's C equals sttsm_bcss on that instance alone
(bit for bit: same tiles, same arithmetic), and a sample equals the oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import device_bcss_from_dense, oracle_C_bcss, rel_fro, xcol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def make_batch(st, count, seed, fp64, cands=(4, 8, 16), small=True):
    prec = st.STTSM_FP64 if fp64 else st.STTSM_BF16X6
    dt = torch.float64 if fp64 else torch.float32
    insts, host = [], []
    for i, (m, n, p) in enumerate(synth.batch_shapes(seed, count)):
        if small:                       # keep the oracle cheap
            n, p = min(n, 24), min(p, 24)
            m = min(m, 4)
        b = st.sttsm_autotune_b(m, n, p, prec, cands)
        A = synth.sym_uniform_dense(m, n, 100 + i)
        X = synth.x_gaussian(200 + i, p, n)
        if not fp64:
            X = X.astype(np.float32).astype(np.float64)
        Ab = device_bcss_from_dense(st, A, m, n, b, dt)
        dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=dt)
        C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=dt, device="cuda")
        insts.append((Ab, dX, C, m, n, p, b))
        host.append((A, X))
    return prec, insts, host


@pytest.mark.parametrize("fp64,kind,r64", [(False, 0, False), (False, 1, False), (True, 0, False), (False, 0, True)])
def test_batch_equals_single_instance_runs(st, fp64, kind, r64):
    st.sttsm_set_small_kernel(kind)
    try:
        _batch_equals_single(st, fp64, r64)
    finally:
        st.sttsm_set_small_kernel(0)


def _batch_equals_single(st, fp64, r64=False):
    prec, insts, host = make_batch(st, 48, 3, fp64)
    if r64:
        prec = st.STTSM_BF16X6_R64
    plan = st.BatchPlan(insts, prec)
    ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    plan.run(ws)
    torch.cuda.synchronize()
    tol = 1e-12 if fp64 else 1e-6
    for i, ((Ab, dX, C, m, n, p, b), (A, X)) in enumerate(zip(insts, host)):
        got = C.double().cpu().numpy()
        Cs = torch.empty_like(C)
        st.sttsm_bcss(Ab, dX, m, n, p, b, Cs, prec, st.workspace_tensor(m, n, p, b, prec))
        torch.cuda.synchronize()
        assert np.array_equal(got, Cs.double().cpu().numpy()), i
        if i % 6 == 0:
            assert rel_fro(got, oracle_C_bcss(A, X, m, p, b)) <= tol
    plan.destroy()


def test_batch_waves_and_graph_replay(st):
    prec, insts, host = make_batch(st, 40, 5, False)
    one = st.BatchPlan(insts, prec)
    ws1 = torch.empty(max(one.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    one.run(ws1)
    torch.cuda.synchronize()
    ref = [C.clone() for (_, _, C, *_rest) in insts]
    budget = one.workspace_size() // 4
    many = st.BatchPlan(insts, prec, ws_budget=budget)
    assert many.info()["waves"] >= 3 and many.workspace_size() <= budget
    ws2 = torch.empty(max(many.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    for _ in range(3):                  # first run captures the graph, then replays
        for (_, _, C, *_rest) in insts:
            C.fill_(float("nan"))
        many.run(ws2)
        torch.cuda.synchronize()
        for r, (_, _, C, *_rest) in zip(ref, insts):
            assert torch.equal(r, C)
    assert abs(many.info()["useful_flops"] - sum(st.sttsm_flops(m, n, p, b) for (_, _, _, m, n, p, b) in insts)) < 1.0


def test_batch_config_shapes_sampled_against_oracle(st):
    """Full-size shapes of the batched workload (n up to 64, m up to 5), oracle on a sample."""
    prec, insts, host = make_batch(st, 24, 3, False, small=False)
    plan = st.BatchPlan(insts, prec)
    ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
    plan.run(ws)
    torch.cuda.synchronize()
    checked = 0
    for (Ab, dX, C, m, n, p, b), (A, X) in zip(insts, host):
        if n ** m > 3e7:
            continue
        got = C.double().cpu().numpy()
        assert rel_fro(got, oracle_C_bcss(A, X, m, p, b)) <= 1e-6
        checked += 1
    assert checked >= 8


def test_one_shot_batch(st):
    prec, insts, host = make_batch(st, 12, 7, False)
    plan = st.BatchPlan(insts, prec)
    need = plan.workspace_size()
    plan.destroy()
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    st.sttsm_batch(insts, prec, ws)
    for (Ab, dX, C, m, n, p, b), (A, X) in zip(insts, host):
        assert rel_fro(C.double().cpu().numpy(), oracle_C_bcss(A, X, m, p, b)) <= 1e-6


def test_batch_fused_tail_equals_two_launches(st):
    """A batch whose short instances run their last two levels fused gives the same
    bits as the same batch planned with the fused launch switched off."""
    prec, insts, host = make_batch(st, 48, 5, False)
    outs = []
    for fused in (st.FUSED_TAIL_ALL, st.FUSED_TAIL_OFF):
        st.sttsm_set_fused_tail(fused)
        try:
            plan = st.BatchPlan(insts, prec)
            ws = torch.empty(max(plan.workspace_size(), 1), dtype=torch.uint8, device="cuda")
            for (_, _, C, *_rest) in insts:
                C.fill_(float("nan"))
            plan.run(ws)
            torch.cuda.synchronize()
            outs.append([C.double().cpu().numpy() for (_, _, C, *_rest) in insts])
            plan.destroy()
        finally:
            st.sttsm_set_fused_tail(st.FUSED_TAIL_CALLS)
    for a, b in zip(*outs):
        assert not np.isnan(a).any() and np.array_equal(a, b)
