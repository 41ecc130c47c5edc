"""FP64 CPU oracle for sttsm (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU
library and the GPU library never imports it.

The C source ``oracle.c`` holds the arithmetic; this module only builds it
with gcc and marshals numpy arrays.  Conventions (paper Sec. 2.1, App. A):
dense tensors are flat arrays in dimensional order (mode 0 fastest), and X
is a (p, n) matrix passed column-major (chi_{j,i} at j + i*p).

Functions and what pins them are listed in the header of ``oracle.c``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_DIR = _HERE / "_lib"
_LIB_PATH = _LIB_DIR / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile oracle.c into oracle/_lib/liboracle.so with gcc (OpenMP)."""
    src = _HERE / "oracle.c"
    if not force and _LIB_PATH.exists() and _LIB_PATH.stat().st_mtime >= src.stat().st_mtime:
        return _LIB_PATH
    _LIB_DIR.mkdir(exist_ok=True)
    tmp = _LIB_PATH.with_suffix(".so.tmp%d" % os.getpid())
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           str(src), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declares the C signatures on a loaded build of oracle.c."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.oracle_sttsm_bruteforce.argtypes = [ctypes.c_int, i64, i64, P, P, P]
    lib.oracle_sttsm_bruteforce.restype = None
    lib.oracle_ttm_chain.argtypes = [ctypes.c_int, i64, P, P, P, P]
    lib.oracle_ttm_chain.restype = ctypes.c_int
    lib.oracle_sttsm_entries.argtypes = [ctypes.c_int, i64, i64, P, P, P, i64, P]
    lib.oracle_sttsm_entries.restype = ctypes.c_int
    lib.oracle_bcss_count_blocks.argtypes = [ctypes.c_int, i64]
    lib.oracle_bcss_count_blocks.restype = i64
    lib.oracle_bcss_pack.argtypes = [ctypes.c_int, i64, ctypes.c_int, P, P]
    lib.oracle_bcss_pack.restype = None
    lib.oracle_bcss_flops.argtypes = [ctypes.c_int, i64, i64, ctypes.c_int, ctypes.c_int]
    lib.oracle_bcss_flops.restype = ctypes.c_double
    return lib


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(ctypes.CDLL(str(_LIB_PATH)))
    return _lib


@contextlib.contextmanager
def library(path):
    """Runs this module's functions on another build of oracle.c (the tests
    that plant a mistake in a copy of the source use it to show that the pins
    catch it); the default build is restored afterwards."""
    global _lib
    prev = _load()
    _lib = _bind(ctypes.CDLL(str(path)))
    try:
        yield
    finally:
        _lib = prev


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _xcol(X) -> np.ndarray:
    """X as a column-major (p, n) FP64 buffer."""
    return np.asfortranarray(np.asarray(X, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    """Threads used by the oracle's OpenMP loops (0 = library default)."""
    if n > 0:
        os.environ["OMP_NUM_THREADS"] = str(n)


def sttsm_bruteforce(A: np.ndarray, X: np.ndarray, m: int) -> np.ndarray:
    """Eq. (cob) summed term by term; A dense (n^m, dimensional order)."""
    lib = _load()
    X = _xcol(X)
    p, n = X.shape
    A = _f64(A).reshape(-1)
    assert A.size == n ** m
    C = np.empty(p ** m, dtype=np.float64)
    lib.oracle_sttsm_bruteforce(m, n, p, _ptr(A), _ptr(X), _ptr(C))
    return C


def ttm_chain(A: np.ndarray, Xs: list, m: int) -> np.ndarray:
    """A x_{m-1} Xs[m-1] ... x_0 Xs[0] by successive mode products."""
    lib = _load()
    Xs = [_xcol(x) for x in Xs]
    n = Xs[0].shape[1]
    A = _f64(A).reshape(-1)
    assert A.size == n ** m and len(Xs) == m
    q = np.array([x.shape[0] for x in Xs], dtype=np.int64)
    ptrs = (ctypes.c_void_p * m)(*[x.ctypes.data for x in Xs])
    out = np.empty(int(np.prod(q)), dtype=np.float64)
    rc = lib.oracle_ttm_chain(m, n, _ptr(A), _ptr(q), ptrs, _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_ttm_chain could not allocate a temporary")
    return out


def sttsm_chain(A: np.ndarray, X: np.ndarray, m: int) -> np.ndarray:
    """[A; X, ..., X] by the dense successive-mode-product algorithm."""
    return ttm_chain(A, [X] * m, m)


def sttsm_entries(A: np.ndarray, X: np.ndarray, m: int, J: np.ndarray) -> np.ndarray:
    """Entries gamma_j for the index tuples J (count x m)."""
    lib = _load()
    X = _xcol(X)
    p, n = X.shape
    A = _f64(A).reshape(-1)
    J = np.ascontiguousarray(J, dtype=np.int64).reshape(-1, m)
    out = np.empty(J.shape[0], dtype=np.float64)
    rc = lib.oracle_sttsm_entries(m, n, p, _ptr(A), _ptr(X), _ptr(J), J.shape[0], _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_sttsm_entries could not allocate a temporary")
    return out


def bcss_count_blocks(m: int, nbar: int) -> int:
    return int(_load().oracle_bcss_count_blocks(m, nbar))


def bcss_pack(dense: np.ndarray, m: int, n: int, b: int) -> np.ndarray:
    """Dense symmetric tensor -> BCSS array (stored blocks in loop order)."""
    lib = _load()
    nbar = -(-n // b)
    nblk = bcss_count_blocks(m, nbar)
    dense = _f64(dense).reshape(-1)
    out = np.empty(nblk * b ** m, dtype=np.float64)
    lib.oracle_bcss_pack(m, n, b, _ptr(dense), _ptr(out))
    return out


def bcss_flops(m: int, n: int, p: int, b: int, bC: int | None = None) -> float:
    """Flops of the algorithm-by-blocks with partially symmetric temporaries."""
    return float(_load().oracle_bcss_flops(m, n, p, b, b if bC is None else bC))
