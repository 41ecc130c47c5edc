"""Seeded synthetic inputs for sttsm tests and benchmarks.

Shared by the FP64 oracle and by the GPU tests/benchmark; it holds no
arithmetic of the method, only the counter-based generator (Philox4x32-10)
and the map from index tuples to draws (see ``synth.h``).

Layouts: dense tensors are flat arrays in dimensional order (mode 0
fastest); matrices are returned as (rows, cols) numpy arrays and callers pass
them column-major where a C interface wants X (chi_{j,i} at j + i*p).

Workload recipes (paper Sec. 7 used "randomized" FP64 data; these stand in):
  * symmetric A: Uniform(-1,1) per unique entry (sorted index tuple);
  * X: N(0, 1/n) entries, or orthonormal rows (QR of a Gaussian);
  * rank-R symmetric A = sum_r lambda_r a_r^{(x)m}, a_r ~ N(0,1).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_DIR = _HERE / "_lib"
_HOST = _LIB_DIR / "libsynth_host.so"
_DEV = _LIB_DIR / "libsynth_dev.so"
_host = None
_dev = None

CUDA_ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _stale(out: Path, *srcs: Path) -> bool:
    return not out.exists() or any(out.stat().st_mtime < s.stat().st_mtime for s in srcs)


def build_host(force: bool = False) -> None:
    _LIB_DIR.mkdir(exist_ok=True)
    srcs = [_HERE / "synth_host.c", _HERE / "synth.h"]
    if force or _stale(_HOST, *srcs):
        tmp = _HOST.with_suffix(".so.tmp%d" % os.getpid())
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        str(srcs[0]), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _HOST)


def build_dev_cmd() -> list[str] | None:
    """nvcc command for the device generator, or None if it is up to date."""
    srcs = [_HERE / "synth_dev.cu", _HERE / "synth.h"]
    if not _stale(_DEV, *srcs):
        return None
    _LIB_DIR.mkdir(exist_ok=True)
    return ["nvcc", CUDA_ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC",
            str(srcs[0]), "-o", str(_DEV)]


def build(force: bool = False) -> None:
    build_host(force)
    cmd = build_dev_cmd() if not force else build_dev_cmd() or [
        "nvcc", CUDA_ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC",
        str(_HERE / "synth_dev.cu"), "-o", str(_DEV)]
    if cmd is not None and shutil.which("nvcc"):
        subprocess.run(cmd, check=True)


def _h():
    global _host
    if _host is None:
        build_host()
        lib = ctypes.CDLL(str(_HOST))
        P, i64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
        lib.synth_philox_batch.argtypes = [P, P, i64, P]
        lib.synth_sym_uniform_dense_f64.argtypes = [ctypes.c_int, i64, u64, P]
        lib.synth_sym_uniform_values.argtypes = [ctypes.c_int, i64, u64, P, i64, P]
        lib.synth_gaussian.argtypes = [u64, i64, ctypes.c_double, P]
        lib.synth_rank_r_dense.argtypes = [ctypes.c_int, i64, ctypes.c_int, P, P, P]
        for f in ("synth_philox_batch", "synth_sym_uniform_dense_f64", "synth_sym_uniform_values",
                  "synth_gaussian", "synth_rank_r_dense"):
            getattr(lib, f).restype = None
        _host = lib
    return _host


def _d():
    global _dev
    if _dev is None:
        if not _DEV.exists():
            raise RuntimeError("libsynth_dev.so is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(str(_DEV))
        lib.synth_dev_sym_uniform_dense.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                                    ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        lib.synth_dev_sym_uniform_dense.restype = ctypes.c_int
        _dev = lib
    return _dev


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 on counters ctr (count x 4, uint32) with key (2 words)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    _h().synth_philox_batch(_p(ctr), _p(key), ctr.shape[0], _p(out))
    return out


def sym_uniform_dense(m: int, n: int, seed: int) -> np.ndarray:
    """Dense symmetric Uniform(-1,1) tensor, FP64, flat dimensional order."""
    out = np.empty(n ** m, dtype=np.float64)
    _h().synth_sym_uniform_dense_f64(m, n, seed, _p(out))
    return out


def sym_uniform_values(m: int, n: int, seed: int, idx: np.ndarray) -> np.ndarray:
    """Values of the symmetric Uniform(-1,1) tensor at index tuples idx (count x m)."""
    idx = np.ascontiguousarray(idx, dtype=np.int64).reshape(-1, m)
    out = np.empty(idx.shape[0], dtype=np.float64)
    _h().synth_sym_uniform_values(m, n, seed, _p(idx), idx.shape[0], _p(out))
    return out


def gaussian(seed: int, rows: int, cols: int, scale: float = 1.0) -> np.ndarray:
    """(rows, cols) matrix of N(0, scale^2) draws; entry (r, c) uses counter r + c*rows."""
    out = np.empty(rows * cols, dtype=np.float64)
    _h().synth_gaussian(seed, rows * cols, scale, _p(out))
    return out.reshape(cols, rows).T.copy()


def x_gaussian(seed: int, p: int, n: int) -> np.ndarray:
    """X (p x n) with entries N(0, 1/n)."""
    return gaussian(seed, p, n, 1.0 / np.sqrt(n))


def x_orthonormal_rows(seed: int, p: int, n: int) -> np.ndarray:
    """X (p x n, p <= n) with orthonormal rows: Q of the QR of a seeded n x p Gaussian, transposed."""
    q, _ = np.linalg.qr(gaussian(seed, n, p))
    return np.ascontiguousarray(q.T)


def rank_r_dense(m: int, n: int, lambdas, vecs: np.ndarray) -> np.ndarray:
    """Dense sum_r lambda_r a_r^{(x)m} (vecs: R x n), FP64, flat dimensional order."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(-1)
    vecs = np.ascontiguousarray(vecs, dtype=np.float64).reshape(lam.size, n)
    out = np.empty(n ** m, dtype=np.float64)
    _h().synth_rank_r_dense(m, n, lam.size, _p(lam), _p(vecs), _p(out))
    return out


def rank_r_factors(seed: int, R: int, n: int) -> np.ndarray:
    """R x n matrix of N(0,1) factor vectors a_r."""
    return gaussian(seed, R, n, 1.0)


def dev_sym_uniform_dense(ptr: int, m: int, n: int, seed: int, dtype: str, stream: int = 0) -> None:
    """Fill device memory at ptr with the same tensor as sym_uniform_dense (FP64 or FP32)."""
    code = {"f64": 0, "f32": 1}[dtype]
    rc = _d().synth_dev_sym_uniform_dense(ctypes.c_void_p(ptr), m, n, seed, code, ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError("synth_dev_sym_uniform_dense failed with CUDA error %d" % rc)


def _uniform01(seed: int, count: int, stream: int) -> np.ndarray:
    """count Uniform[0,1) draws from Philox word 0, counters (t, 0, stream, 0), key (seed, 2)."""
    ctr = np.zeros((count, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(count, dtype=np.uint32)
    ctr[:, 2] = stream
    w = philox4x32_10(ctr, [seed & 0xFFFFFFFF, 2])[:, 0]
    return w.astype(np.float64) / 4294967296.0


def batch_shapes(seed: int, count: int):
    """Shapes of the batched workload: m in {3,4,5} with weights {.5,.3,.2},
    n uniform in {8..64}, p uniform in {8..n}.  Returns a list of (m, n, p)."""
    u = _uniform01(seed, count, 0)
    v = _uniform01(seed, count, 1)
    w = _uniform01(seed, count, 2)
    m = np.where(u < 0.5, 3, np.where(u < 0.8, 4, 5))
    n = 8 + np.floor(v * 57).astype(int)
    p = 8 + np.floor(w * (n - 7)).astype(int)
    return [(int(a), int(b), int(c)) for a, b, c in zip(m, n, p)]


SERVE_CLASSES = ((3, 64, 512), (4, 32, 160), (5, 16, 64), (6, 8, 32))


def serve_requests(seed: int, rate: float, seconds: float):
    """Poisson arrivals at `rate` per second over `seconds`; each request is
    uniform over the four (m, range) classes with n, p uniform in the class
    range.  Returns a list of (arrival_s, m, n, p)."""
    expect = int(rate * seconds * 1.2) + 64
    u = _uniform01(seed, expect, 0)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    t = t[t < seconds]
    k = len(t)
    cls = np.minimum((_uniform01(seed, k, 1) * 4).astype(int), 3)
    a = _uniform01(seed, k, 2)
    c = _uniform01(seed, k, 3)
    out = []
    for i in range(k):
        m, lo, hi = SERVE_CLASSES[cls[i]]
        n = lo + int(a[i] * (hi - lo + 1))
        p = lo + int(c[i] * (hi - lo + 1))
        out.append((float(t[i]), m, min(n, hi), min(p, hi)))
    return out
