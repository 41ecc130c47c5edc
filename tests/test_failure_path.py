"""Failure detection without a GPU fault: every spin-wait in the level kernels
is bounded and, when it runs out, raises a status word that the next library
call reports as STTSM_ERR_TIMEOUT.  The self-test launches a wait on an
mbarrier that nothing arrives on, with a short limit."""
import time

import numpy as np
import pytest

import synth
from helpers import device_bcss_from_dense, oracle_C_bcss, rel_fro, xcol


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


def test_selftest_rejects_bad_limits_on_the_host(st):
    """Argument checks happen before any CUDA call."""
    assert st.sttsm_selftest_wait_timeout(0.0) == st.STTSM_ERR_ARG
    assert st.sttsm_selftest_wait_timeout(-1.0) == st.STTSM_ERR_ARG
    assert st.sttsm_selftest_wait_timeout(5000.0) == st.STTSM_ERR_ARG


@pytest.mark.gpu
def test_wait_runs_out_status_reported_context_usable(st):
    torch = pytest.importorskip("torch")
    assert st.sttsm_device_status() == 0
    t0 = time.time()
    rc = st.sttsm_selftest_wait_timeout(50.0)
    dt = time.time() - t0
    assert rc == st.STTSM_ERR_TIMEOUT
    assert dt < 5.0
    assert st.sttsm_device_status() == 0          # reported once, then cleared
    # the context is still usable: a full sttsm call right after is correct
    m, n, p, b = 3, 24, 24, 8
    A = synth.sym_uniform_dense(m, n, 3)
    X = synth.x_gaussian(4, p, n)
    Ab = device_bcss_from_dense(st, A, m, n, b, torch.float64)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=torch.float64)
    C = torch.empty(st.bcss_num_elems(m, p, b), dtype=torch.float64, device="cuda")
    st.sttsm_bcss(Ab, dX, m, n, p, b, C, st.STTSM_FP64, st.workspace_tensor(m, n, p, b, st.STTSM_FP64))
    torch.cuda.synchronize()
    assert rel_fro(C.cpu().numpy(), oracle_C_bcss(A, X, m, p, b)) <= 1e-12
    assert st.sttsm_device_status() == 0
