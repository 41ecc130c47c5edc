"""Shared helpers of the GPU tests: inputs from synth/, expected values from
oracle/ only, results read back from the library through its C ABI."""
import math

import numpy as np

import oracle
import synth


def xcol(X):
    """X (p x n) as the flat column-major buffer the C ABI takes."""
    return np.asfortranarray(X).reshape(-1, order="F")


def bcss_pos(j, m, b):
    """BCSS position of entry j (any order): sorted indices -> block tuple ->
    colex rank, plus the in-block dimensional offset (restated here, not
    taken from the library)."""
    s = sorted(int(x) for x in j)
    rank = sum(math.comb(s[t] // b + t, t + 1) for t in range(m))
    loc = sum((s[t] % b) * b ** t for t in range(m))
    return rank * b ** m + loc


def rel_fro(got, ref):
    return float(np.linalg.norm(np.asarray(got) - np.asarray(ref)) / np.linalg.norm(ref))


def device_bcss_from_dense(st, dense_np, m, n, b, dtype):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(dense_np)).to(device="cuda", dtype=dtype)
    out = torch.empty(st.bcss_num_elems(m, n, b), dtype=dtype, device="cuda")
    st.bcss_pack(d, out, m, n, b)
    return out


def run_sttsm(st, A_bcss_dev, X, m, n, p, b, prec, stream=None):
    """Runs sttsm_bcss on a device BCSS A and host X; returns C (BCSS) as FP64 numpy."""
    import torch
    dt = A_bcss_dev.dtype
    dX = torch.from_numpy(xcol(X)).to(device="cuda", dtype=dt)
    C = torch.full((st.bcss_num_elems(m, p, b),), float("nan"), dtype=dt, device="cuda")
    ws = st.workspace_tensor(m, n, p, b, prec)
    st.sttsm_bcss(A_bcss_dev, dX, m, n, p, b, C, prec, ws, stream)
    torch.cuda.synchronize()
    return C.double().cpu().numpy()


def oracle_C_bcss(A, X, m, p, b):
    return oracle.bcss_pack(oracle.sttsm_chain(A, X, m), m, p, b)


def inputs(m, n, p, seed_a=0, seed_x=1, fp32=False):
    """Symmetric Uniform(-1,1) A (exact in FP32) and N(0,1/n) X; for fp32 the
    X the oracle sees is the FP32-rounded one the GPU sees."""
    A = synth.sym_uniform_dense(m, n, seed_a)
    X = synth.x_gaussian(seed_x, p, n)
    if fp32:
        X = X.astype(np.float32).astype(np.float64)
    return A, X
