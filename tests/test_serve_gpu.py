"""Continuous-batching server: requests of mixed sizes submitted while others
run must give the same C as the same request run alone (same tiles, same
arithmetic: bit for bit), and the oracle's within the split-path tolerance;
admission waits for workspace under the HBM budget; a full queue says BUSY
and an over-budget request says NOMEM — all decided on the host."""
import time

import numpy as np
import pytest

import synth
from helpers import device_bcss_from_dense, oracle_C_bcss, rel_fro, xcol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLASSES = {3: (64, 112), 4: (32, 48), 5: (16, 24), 6: (8, 12)}   # sizes kept oracle-friendly


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def make_request(st, i, m, n, p, b=None):
    cands = {3: (16, 32), 4: (8, 16), 5: (4, 8), 6: (4, 8)}[m]
    if b is None:
        b = st.sttsm_autotune_b(m, n, p, st.STTSM_BF16X6, cands)
    A = synth.sym_uniform_dense(m, n, 300 + i)
    X = synth.x_gaussian(400 + i, p, n).astype(np.float32).astype(np.float64)
    Ab = device_bcss_from_dense(st, A, m, n, b, torch.float32)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
    C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=torch.float32, device="cuda")
    return dict(A=A, X=X, Ab=Ab, dX=dX, C=C, m=m, n=n, p=p, b=b)


def requests(st, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = [3, 4, 5, 6][i % 4]
        lo, hi = CLASSES[m]
        out.append(make_request(st, seed * 1000 + i, m, int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))))
    return out


def wait_all(srv, tickets, timeout=120.0):
    t0 = time.time()
    lat = {}
    while len(lat) < len(tickets):
        for t in tickets:
            if t not in lat:
                done, ms = srv.poll(t)
                if done:
                    lat[t] = ms
        assert time.time() - t0 < timeout, "requests did not complete"
        time.sleep(0.001)
    return lat


def alone(st, r):
    C = torch.empty_like(r["C"])
    st.sttsm_bcss(r["Ab"], r["dX"], r["m"], r["n"], r["p"], r["b"], C, st.STTSM_BF16X6,
                  st.workspace_tensor(r["m"], r["n"], r["p"], r["b"], st.STTSM_BF16X6))
    torch.cuda.synchronize()
    return C.double().cpu().numpy()


def test_mixed_requests_equal_alone_and_oracle(st):
    reqs = requests(st, 24, 1)
    torch.cuda.synchronize()
    srv = st.Server(2 << 30)
    tickets = []
    for k, r in enumerate(reqs):                 # three bursts: later ones join running steps
        tickets.append(srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]))
        if k % 8 == 7:
            time.sleep(0.002)
    lat = wait_all(srv, tickets)
    assert all(v > 0 for v in lat.values())
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["queued"] == 0 and stats["active"] == 0
    assert stats["arena_bytes"] == 0
    srv.destroy()
    for k, r in enumerate(reqs):
        got = r["C"].double().cpu().numpy()
        assert np.array_equal(got, alone(st, r)), k
        if k % 3 == 0:
            assert rel_fro(got, oracle_C_bcss(r["A"], r["X"], r["m"], r["p"], r["b"])) <= 1e-6


def test_admission_waits_under_a_tight_budget(st):
    reqs = requests(st, 12, 2)
    need = max(st.sttsm_workspace_size(r["m"], r["n"], r["p"], r["b"], st.STTSM_BF16X6) for r in reqs)
    srv = st.Server(need + need // 2)            # room for about one request at a time
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
    peak_queue = srv.stats()["queued"]
    wait_all(srv, tickets)
    srv.destroy()
    assert peak_queue >= 1
    for r in reqs:
        assert np.array_equal(r["C"].double().cpu().numpy(), alone(st, r))


def test_busy_queue_and_over_budget_request(st):
    big = make_request(st, 9000, 3, 400, 400)
    small = [make_request(st, 9001 + i, 5, 16, 16) for i in range(4)]
    need = st.sttsm_workspace_size(big["m"], big["n"], big["p"], big["b"], st.STTSM_BF16X6)
    srv = st.Server(need, queue_cap=2)
    t_big = srv.submit(big["Ab"], big["dX"], big["C"], big["m"], big["n"], big["p"], big["b"])
    codes = []                                    # the big request holds the whole arena for ~1 ms
    for r in small:
        try:
            srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"])
            codes.append(0)
        except st.SttsmError as e:
            codes.append(e.code)
    huge = make_request(st, 9100, 3, 512, 512)
    with pytest.raises(st.SttsmError) as e:
        srv.submit(huge["Ab"], huge["dX"], huge["C"], huge["m"], huge["n"], huge["p"], huge["b"])
    assert e.value.code == st.STTSM_ERR_NOMEM
    wait_all(srv, [t_big])
    srv.destroy()
    assert st.STTSM_ERR_BUSY in codes and 0 in codes


def test_both_tma_forms_and_small_tiles_in_one_step(st):
    """Requests that run on the TMA-fed kernel with b = 16 and with b = 32, and on the
    short-contraction kernel, admitted together: every step launches each form over its
    own requests; each result equals the request run alone and the oracle's."""
    shapes = [(3, 100, 90, 16), (3, 96, 96, 32), (4, 70, 40, 16), (3, 130, 70, 32), (5, 16, 16, 4), (3, 24, 24, 8)]
    reqs = [make_request(st, 7000 + i, m, n, p, b) for i, (m, n, p, b) in enumerate(shapes)]
    torch.cuda.synchronize()
    srv = st.Server(4 << 30)
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
    wait_all(srv, tickets)
    srv.destroy()
    for r in reqs:
        got = r["C"].double().cpu().numpy()
        assert np.array_equal(got, alone(st, r)), (r["m"], r["n"], r["b"])
        assert rel_fro(got, oracle_C_bcss(r["A"], r["X"], r["m"], r["p"], r["b"])) <= 1e-6


def test_later_small_requests_pass_one_that_does_not_fit_yet(st):
    """Budget for one big request plus a margin: while the first big request runs,
    a second big one cannot be admitted; small requests submitted after it are
    admitted in the margin and finish before it (admission lets them pass a
    request whose workspace does not fit yet, within the age cap)."""
    big = [make_request(st, 9500 + i, 3, 384, 384, 16) for i in range(2)]
    small = [make_request(st, 9600 + i, 5, 16, 16, 4) for i in range(6)]
    torch.cuda.synchronize()
    need_big = st.sttsm_workspace_size(3, 384, 384, 16, st.STTSM_BF16X6)
    need_small = st.sttsm_workspace_size(5, 16, 16, 4, st.STTSM_BF16X6)
    srv = st.Server(need_big + 8 * need_small + (1 << 20))
    order = []
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in big]
    tickets += [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in small]
    t0 = time.time()
    while len(order) < len(tickets):
        for t in tickets:
            if t not in order and srv.poll(t)[0]:
                order.append(t)
        assert time.time() - t0 < 60.0
    srv.destroy()
    second_big = tickets[1]
    assert any(order.index(t) < order.index(second_big) for t in tickets[2:])
    for r in big + small:
        assert np.array_equal(r["C"].double().cpu().numpy(), alone(st, r))


def test_full_size_classes_sampled_against_oracle(st):
    """One request at the top of each serving class (m=3 n up to 512, m=4 up to
    160, m=5 up to 64, m=6 up to 32), served together; 32 sampled C entries of each
    against the FP64 oracle's entry contraction, and each result equal to the
    request run alone."""
    import oracle
    from helpers import bcss_pos, rel_max
    shapes = [(3, 512, 448, 16), (4, 128, 160, 16), (5, 48, 64, 4), (6, 24, 32, 4)]
    reqs = []
    for i, (m, n, p, b) in enumerate(shapes):
        d = torch.empty(n ** m, dtype=torch.float32, device="cuda")
        synth.dev_sym_uniform_dense(d.data_ptr(), m, n, 9700 + i, "f32", torch.cuda.current_stream().cuda_stream)
        Ab = torch.empty(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
        st.bcss_pack(d, Ab, m, n, b)
        del d
        X = synth.x_gaussian(9800 + i, p, n).astype(np.float32).astype(np.float64)
        dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float32)
        C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=torch.float32, device="cuda")
        reqs.append(dict(Ab=Ab, dX=dX, C=C, X=X, m=m, n=n, p=p, b=b, seed=9700 + i))
    torch.cuda.synchronize()
    srv = st.Server(8 << 30)
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
    wait_all(srv, tickets)
    srv.destroy()
    rng = np.random.default_rng(5)
    for r in reqs:
        m, n, p, b = r["m"], r["n"], r["p"], r["b"]
        got = r["C"].double().cpu().numpy()
        assert np.array_equal(got, alone(st, r))
        J = np.sort(rng.integers(0, p, size=(32, m)), axis=1)
        A = synth.sym_uniform_dense(m, n, r["seed"])
        ref = oracle.sttsm_entries(A, r["X"], m, J)
        del A
        vals = np.array([got[bcss_pos(j, m, b)] for j in J])
        assert rel_fro(vals, ref) <= 1e-6 and rel_max(vals, ref) <= 1e-6, (m, n, p, b)


def test_fused_tail_in_serving_equals_two_launches(st):
    """With the fused last two levels switched on for serving (mode 2), short requests
    finish in m - 1 steps and give the same bits as with two launches."""
    reqs = requests(st, 8, 7)
    torch.cuda.synchronize()
    outs = []
    for mode in (st.FUSED_TAIL_ALL, st.FUSED_TAIL_OFF):
        st.sttsm_set_fused_tail(mode)
        try:
            srv = st.Server(2 << 30)
            for r in reqs:
                r["C"].fill_(float("nan"))
            tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
            wait_all(srv, tickets)
            srv.destroy()
            outs.append([r["C"].double().cpu().numpy() for r in reqs])
        finally:
            st.sttsm_set_fused_tail(st.FUSED_TAIL_CALLS)
    for a, b in zip(*outs):
        assert not np.isnan(a).any() and np.array_equal(a, b)


def test_r64_serving_equals_alone_and_oracle(st):
    """A server in BF16X6_R64 (the final C-block reduction in FP64): requests on the TMA
    kernel (b = 16, 32), the gathered kernel (b = 8) and the FP32 short kernel give the
    same bits as the same request alone in BF16X6_R64, and the oracle's C."""
    shapes = [(3, 100, 90, 16), (3, 96, 96, 32), (3, 70, 60, 8), (5, 16, 16, 4), (4, 40, 30, 8)]
    reqs = [make_request(st, 7500 + i, m, n, p, b) for i, (m, n, p, b) in enumerate(shapes)]
    torch.cuda.synchronize()
    prec = st.STTSM_BF16X6_R64
    srv = st.Server(4 << 30, prec)
    tickets = [srv.submit(r["Ab"], r["dX"], r["C"], r["m"], r["n"], r["p"], r["b"]) for r in reqs]
    wait_all(srv, tickets)
    srv.destroy()
    for r in reqs:
        got = r["C"].double().cpu().numpy()
        C = torch.empty_like(r["C"])
        st.sttsm_bcss(r["Ab"], r["dX"], r["m"], r["n"], r["p"], r["b"], C, prec,
                      st.workspace_tensor(r["m"], r["n"], r["p"], r["b"], prec))
        torch.cuda.synchronize()
        assert np.array_equal(got, C.double().cpu().numpy()), (r["m"], r["n"], r["b"])
        assert rel_fro(got, oracle_C_bcss(r["A"], r["X"], r["m"], r["p"], r["b"])) <= 1e-6
