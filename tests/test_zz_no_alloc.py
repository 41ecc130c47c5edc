"""The allocation-free entry point sttsm_bcss_noalloc, for callers that may not
allocate device memory where they call sttsm (fixed memory budgets,
framework-owned allocators).  Its results must match sttsm_bcss (which takes a
caller workspace) within the tolerances of the other GPU tests, on two calls in
a row, whether this file runs alone in a fresh process or after the others.
This file is named to be collected last."""
import numpy as np
import pytest

from helpers import device_bcss_from_dense, inputs, rel_fro, xcol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# BF16X3 keeps 16 significand bits of each operand in two BF16 pieces and drops
# the lo x lo product: about 3 x 2^-16 = 4.6e-5 relative per product at worst.
# This entry point and sttsm_bcss run different kernels for it (gather-fed and
# TMA-fed), which may differ by that much; 1e-4 bounds it.
TOL = {"fp64": 1e-12, "bf16x6": 1e-6, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def _prec(st, name):
    return {"fp64": st.STTSM_FP64, "bf16x6": st.STTSM_BF16X6, "bf16x3": st.STTSM_BF16X3}[name]


def _operands(st, m, n, p, b, precname):
    fp64 = precname == "fp64"
    dt = torch.float64 if fp64 else torch.float32
    A, X = inputs(m, n, p, seed_a=m + n, seed_x=p, fp32=not fp64)
    Ab = device_bcss_from_dense(st, A, m, n, b, dt)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=dt)
    return Ab, dX, dt


def _with_workspace(st, Ab, dX, m, n, p, b, prec, dt):
    ref = torch.empty(st.bcss_num_elems(m, p, b), dtype=dt, device="cuda")
    st.sttsm_bcss(Ab, dX, m, n, p, b, ref, prec, st.workspace_tensor(m, n, p, b, prec))
    torch.cuda.synchronize()
    return ref.double().cpu().numpy()


def _noalloc(st, Ab, dX, m, n, p, b, prec, dt):
    out = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=dt, device="cuda")
    st.sttsm_bcss_noalloc(Ab, dX, m, n, p, b, out, prec)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert not np.isnan(got).any()
    return got


@pytest.mark.parametrize("m,n,p,b,precname", [(3, 96, 80, 32, "bf16x6"), (4, 20, 12, 5, "bf16x6"),
                                              (3, 40, 40, 8, "fp64"), (3, 96, 80, 32, "bf16x3")])
def test_noalloc_matches_workspace_entry_point(st, m, n, p, b, precname):
    prec = _prec(st, precname)
    Ab, dX, dt = _operands(st, m, n, p, b, precname)
    ref = _with_workspace(st, Ab, dX, m, n, p, b, prec, dt)
    for _ in range(2):
        assert rel_fro(_noalloc(st, Ab, dX, m, n, p, b, prec, dt), ref) <= TOL[precname]


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_short_contractions_under_both_kernels(st, kind):
    """n̄ b <= 64: the FP32 CUDA-core kernel (0) and the tcgen05 small-tile kernel (1)."""
    m, n, p, b = 4, 30, 20, 4
    prec = st.STTSM_BF16X6
    st.sttsm_set_small_kernel(kind)
    try:
        Ab, dX, dt = _operands(st, m, n, p, b, "bf16x6")
        ref = _with_workspace(st, Ab, dX, m, n, p, b, prec, dt)
        for _ in range(2):
            assert rel_fro(_noalloc(st, Ab, dX, m, n, p, b, prec, dt), ref) <= 1e-6
    finally:
        st.sttsm_set_small_kernel(0)


def test_noalloc_shape_changes_replace_the_resident_plans(st):
    """S1, then S2, then S1 again: the second S1 call re-installs S1's plans and
    gives S1's bits."""
    s1, s2 = (3, 96, 80, 32), (4, 20, 12, 5)
    prec = st.STTSM_BF16X6
    ops1 = _operands(st, *s1, "bf16x6")
    ops2 = _operands(st, *s2, "bf16x6")
    first = _noalloc(st, ops1[0], ops1[1], *s1, prec, ops1[2])
    second = _noalloc(st, ops2[0], ops2[1], *s2, prec, ops2[2])
    again = _noalloc(st, ops1[0], ops1[1], *s1, prec, ops1[2])
    assert np.array_equal(first, again)
    assert rel_fro(second, _with_workspace(st, ops2[0], ops2[1], *s2, prec, ops2[2])) <= 1e-6


def test_noalloc_reports_a_timed_out_wait_once(st):
    """A bounded wait that runs out on this entry point's status word (the
    self-test's wait on an mbarrier nothing arrives on, 50 ms) is reported by the
    next sttsm_bcss_noalloc call as STTSM_ERR_TIMEOUT; the call after that runs
    and is correct, and sttsm_bcss's own status word is untouched."""
    m, n, p, b = 3, 96, 80, 32
    prec = st.STTSM_BF16X6
    Ab, dX, dt = _operands(st, m, n, p, b, "bf16x6")
    ref = _with_workspace(st, Ab, dX, m, n, p, b, prec, dt)
    st.sttsm_noalloc_selftest_wait_timeout(50.0)
    out = torch.empty(st.bcss_num_elems(m, p, b), dtype=dt, device="cuda")
    with pytest.raises(st.SttsmError) as e:
        st.sttsm_bcss_noalloc(Ab, dX, m, n, p, b, out, prec)
    assert e.value.code == st.STTSM_ERR_TIMEOUT
    assert st.sttsm_device_status() == 0
    assert rel_fro(_noalloc(st, Ab, dX, m, n, p, b, prec, dt), ref) <= 1e-6


def test_noalloc_rejects_shapes_beyond_its_scratch(st):
    m, n, p, b = 3, 768, 768, 64
    A = torch.zeros(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
    X = torch.zeros(p * n, dtype=torch.float32, device="cuda")
    C = torch.zeros(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda")
    with pytest.raises(st.SttsmError) as e:
        st.sttsm_bcss_noalloc(A, X, m, n, p, b, C, st.STTSM_BF16X6)
    assert e.value.code == st.STTSM_ERR_NOMEM


def test_noalloc_selftest_rejects_bad_limits(st):
    for limit in (0.0, -1.0, 5000.0):
        with pytest.raises(st.SttsmError) as e:
            st.sttsm_noalloc_selftest_wait_timeout(limit)
        assert e.value.code == st.STTSM_ERR_ARG
