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


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_7744_gb300 as pkg
    return pkg


@pytest.mark.parametrize("m,n,p,b,precname", [(3, 96, 80, 32, "bf16x6"), (4, 20, 12, 5, "bf16x6"),
                                              (3, 40, 40, 8, "fp64")])
def test_noalloc_matches_workspace_entry_point(st, m, n, p, b, precname):
    fp64 = precname == "fp64"
    prec = st.STTSM_FP64 if fp64 else st.STTSM_BF16X6
    dt = torch.float64 if fp64 else torch.float32
    tol = 1e-12 if fp64 else 1e-6
    A, X = inputs(m, n, p, seed_a=m + n, seed_x=p, fp32=not fp64)
    Ab = device_bcss_from_dense(st, A, m, n, b, dt)
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=dt)
    ref = torch.empty(st.bcss_num_elems(m, p, b), dtype=dt, device="cuda")
    st.sttsm_bcss(Ab, dX, m, n, p, b, ref, prec, st.workspace_tensor(m, n, p, b, prec))
    torch.cuda.synchronize()
    ref_np = ref.double().cpu().numpy()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        st.sttsm_bcss_noalloc(Ab, dX, m, n, p, b, out, prec)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert not np.isnan(got).any()
        assert rel_fro(got, ref_np) <= tol


def test_noalloc_rejects_shapes_beyond_its_scratch(st):
    m, n, p, b = 3, 768, 768, 64
    A = torch.zeros(st.bcss_num_elems(m, n, b), dtype=torch.float32, device="cuda")
    X = torch.zeros(p * n, dtype=torch.float32, device="cuda")
    C = torch.zeros(st.bcss_num_elems(m, p, b), dtype=torch.float32, device="cuda")
    with pytest.raises(st.SttsmError) as e:
        st.sttsm_bcss_noalloc(A, X, m, n, p, b, C, st.STTSM_BF16X6)
    assert e.value.code == st.STTSM_ERR_NOMEM
