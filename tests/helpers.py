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


def rel_max(got, ref):
    """Elementwise bound beside the Frobenius one: max |got - ref| / max |ref|
    (a wrong block among many right ones shows here even where a norm over all
    entries would hide it)."""
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


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


def colex_tuples(length, nb):
    """Sorted block tuples (t_0 <= ... <= t_{length-1}) over [0, nb) in colex order
    (last index most significant), enumerated directly."""
    import itertools
    tups = list(itertools.combinations_with_replacement(range(nb), length))
    return sorted(tups, key=lambda t: tuple(reversed(t)))


def all_but_one_storage(B, m, n, p, b):
    """The dense all-but-one result B (n x p x ... x p, symmetric in modes 1..m-1)
    laid out as the library's partially symmetric storage [node][ib][b^m]: node =
    colex rank of the sorted p-block tuple of modes 1..m-1, ib = block of mode 0,
    in-block offset i_0 + sum_t j_t b^t; zero past n or p."""
    nbar, pbar = -(-n // b), -(-p // b)
    nodes = colex_tuples(m - 1, pbar)
    out = np.zeros((len(nodes), nbar, b ** m))
    off = np.arange(b ** m)
    loc = np.array([(off // b ** t) % b for t in range(m)])   # local index of mode t at in-block offset e
    for r, tup in enumerate(nodes):
        for ib in range(nbar):
            idx = [ib * b + loc[0]] + [tup[t - 1] * b + loc[t] for t in range(1, m)]
            ok = (idx[0] < n)
            for t in range(1, m):
                ok &= idx[t] < p
            vals = np.zeros(b ** m)
            sel = np.nonzero(ok)[0]
            vals[sel] = B[tuple(ix[sel] for ix in idx)]
            out[r, ib] = vals
    return out.reshape(-1)
