"""Python binding of libsttsm (the C ABI in include/sttsm.h).

Argument marshalling only: every step of sttsm runs in the library's CUDA
kernels.  Device buffers are torch tensors (their data_ptr is passed);
streams are torch CUDA streams (default: the current stream).  Names and
argument order follow the C ABI.

Paper: Schatz, Low, van de Geijn, Kolda, "Exploiting Symmetry in Tensors for
High Performance: Multiplication with Symmetric Tensors", arXiv 1301.7744.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
_LIB_PATH = _PKG / "_lib" / "libsttsm.so"

STTSM_OK = 0
STTSM_ERR_ARG = -1
STTSM_ERR_UNSUPPORTED = -2
STTSM_ERR_NOMEM = -3
STTSM_ERR_TIMEOUT = -4
STTSM_ERR_CUDA = -5
STTSM_ERR_BUSY = -6

STTSM_FP64 = 0
STTSM_BF16X6 = 1
STTSM_TF32X3 = 2
STTSM_BF16X3 = 3
STTSM_BF16X6_R64 = 4
STTSM_BF16X3_R64 = 5

DTYPE_F64 = 0
DTYPE_F32 = 1

PREC_NAMES = {STTSM_FP64: "fp64", STTSM_BF16X6: "bf16x6", STTSM_TF32X3: "tf32x3", STTSM_BF16X3: "bf16x3",
              STTSM_BF16X6_R64: "bf16x6_r64", STTSM_BF16X3_R64: "bf16x3_r64"}
_ERRORS = {STTSM_ERR_ARG: "invalid argument", STTSM_ERR_UNSUPPORTED: "unsupported",
           STTSM_ERR_NOMEM: "workspace too small or allocation failed", STTSM_ERR_TIMEOUT: "device wait timed out",
           STTSM_ERR_CUDA: "CUDA call failed", STTSM_ERR_BUSY: "queue full"}


class SttsmError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__("%s returned %d (%s)" % (fn, code, _ERRORS.get(code, "?")))
        self.code = code


_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError("libsttsm.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    L = ctypes.CDLL(str(_LIB_PATH))
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.bcss_num_blocks.argtypes = [i32, i64, i32]
    L.bcss_num_blocks.restype = i64
    L.bcss_num_elems.argtypes = [i32, i64, i32]
    L.bcss_num_elems.restype = i64
    L.bcss_block_rank.argtypes = [i32, P]
    L.bcss_block_rank.restype = i64
    L.bcss_block_unrank.argtypes = [i32, i64, P]
    L.bcss_block_unrank.restype = i32
    L.sttsm_flops.argtypes = [i32, i64, i64, i32]
    L.sttsm_flops.restype = ctypes.c_double
    L.bcss_pack.argtypes = [P, P, i32, i64, i32, i32, P]
    L.bcss_pack.restype = i32
    L.bcss_unpack.argtypes = [P, P, i32, i64, i32, i32, P]
    L.bcss_unpack.restype = i32
    L.sttsm_workspace_size.argtypes = [i32, i64, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    L.sttsm_workspace_size.restype = i32
    L.sttsm_bcss.argtypes = [P, P, i32, i64, i64, i32, P, i32, P, ctypes.c_size_t, P]
    L.sttsm_bcss.restype = i32
    L.sttsm_bcss_host.argtypes = [P, P, i32, i64, i64, i32, P, i32, P, P, P, P, ctypes.c_size_t, P]
    L.sttsm_bcss_host.restype = i32
    L.sttsm_bcss_all_but_one.argtypes = [P, P, i32, i64, i64, i32, P, i32, P, ctypes.c_size_t, P]
    L.sttsm_bcss_all_but_one.restype = i32
    L.sttsm_all_but_one_elems.argtypes = [i32, i64, i64, i32]
    L.sttsm_all_but_one_elems.restype = i64
    L.sttsm_all_but_one_flops.argtypes = [i32, i64, i64, i32]
    L.sttsm_all_but_one_flops.restype = ctypes.c_double
    L.sttsm_device_status.argtypes = []
    L.sttsm_device_status.restype = i32
    L.sttsm_selftest_wait_timeout.argtypes = [ctypes.c_double]
    L.sttsm_selftest_wait_timeout.restype = i32
    L.sttsm_autotune_b.argtypes = [i32, i64, i64, i32, P, i32]
    L.sttsm_autotune_b.restype = i32
    L.sttsm_autotune_b_measured.argtypes = [i32, i64, i64, i32, P, i32, i32, P]
    L.sttsm_autotune_b_measured.restype = i32
    L.sttsm_batch_plan_create.argtypes = [P, i32, i32, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]
    L.sttsm_batch_plan_create.restype = i32
    L.sttsm_batch_workspace_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.sttsm_batch_workspace_size.restype = i32
    L.sttsm_batch_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.sttsm_batch_info.restype = i32
    L.sttsm_batch_run.argtypes = [P, P, ctypes.c_size_t, P]
    L.sttsm_batch_run.restype = i32
    L.sttsm_batch_plan_destroy.argtypes = [P]
    L.sttsm_batch_plan_destroy.restype = i32
    L.sttsm_batch.argtypes = [P, i32, i32, P, ctypes.c_size_t, P]
    L.sttsm_batch.restype = i32
    L.sttsm_serve_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(ctypes.c_void_p)]
    L.sttsm_serve_create.restype = i32
    L.sttsm_serve_submit.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
    L.sttsm_serve_submit.restype = i32
    L.sttsm_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.sttsm_serve_poll.restype = i32
    L.sttsm_serve_stats.argtypes = [P, P]
    L.sttsm_serve_stats.restype = i32
    L.sttsm_serve_destroy.argtypes = [P]
    L.sttsm_serve_destroy.restype = i32
    L.sttsm_set_small_kernel.argtypes = [i32]
    L.sttsm_set_small_kernel.restype = i32
    L.sttsm_set_fused_tail.argtypes = [i32]
    L.sttsm_set_fused_tail.restype = i32
    L.sttsm_bcss_noalloc.argtypes = [P, P, i32, i64, i64, i32, P, i32, P]
    L.sttsm_bcss_noalloc.restype = i32
    L.sttsm_noalloc_selftest_wait_timeout.argtypes = [ctypes.c_double]
    L.sttsm_noalloc_selftest_wait_timeout.restype = i32
    L.sttsm_profile_enable.argtypes = [i32]
    L.sttsm_profile_enable.restype = i32
    L.sttsm_profile_read.argtypes = [i32, P, P, P, P, P]
    L.sttsm_profile_read.restype = i32
    L.sttsm_plan_level.argtypes = [i32, i64, i64, i32, i32, i32, P, i64, P, i64, P, P, P]
    L.sttsm_plan_level.restype = i32
    L.sttsm_plan_pair.argtypes = [i32, i64, i64, i32, P, i64, P, P]
    L.sttsm_plan_pair.restype = i32
    L.sttsm_set_inblock_symmetry.argtypes = [i32]
    L.sttsm_set_inblock_symmetry.restype = i32
    L.sttsm_plan_sym_rows.argtypes = [i32, i64, i64, i32, i32, i64, i64, i64, P, P, P]
    L.sttsm_plan_sym_rows.restype = i32
    _lib = L
    return L


def exported_symbols() -> list[str]:
    """Names of the C-ABI entry points this binding loads."""
    return ["bcss_num_blocks", "bcss_num_elems", "bcss_block_rank", "bcss_block_unrank", "sttsm_flops",
            "bcss_pack", "bcss_unpack", "sttsm_workspace_size", "sttsm_bcss", "sttsm_bcss_all_but_one",
            "sttsm_all_but_one_elems", "sttsm_all_but_one_flops", "sttsm_bcss_host", "sttsm_autotune_b",
            "sttsm_autotune_b_measured", "sttsm_batch_plan_create", "sttsm_batch_workspace_size",
            "sttsm_batch_info", "sttsm_batch_run", "sttsm_batch_plan_destroy", "sttsm_batch", "sttsm_serve_create",
            "sttsm_serve_submit", "sttsm_serve_poll", "sttsm_serve_stats", "sttsm_serve_destroy",
            "sttsm_bcss_noalloc", "sttsm_noalloc_selftest_wait_timeout", "sttsm_set_small_kernel", "sttsm_set_fused_tail", "sttsm_set_inblock_symmetry", "sttsm_device_status", "sttsm_selftest_wait_timeout",
            "sttsm_plan_level", "sttsm_plan_pair", "sttsm_plan_sym_rows", "sttsm_profile_enable", "sttsm_profile_read"]


def _check(fn: str, rc: int) -> None:
    if rc != STTSM_OK:
        raise SttsmError(fn, rc)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a) -> ctypes.c_void_p:
    """Host buffer pointer: a CPU torch tensor or a numpy array."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return DTYPE_F64
    if t.dtype == torch.float32:
        return DTYPE_F32
    raise ValueError("BCSS tensors hold float64 or float32")


# ---------------------------------------------------------------- BCSS indexing (host)

def bcss_num_blocks(m: int, n: int, b: int) -> int:
    return int(_load().bcss_num_blocks(m, n, b))


def bcss_num_elems(m: int, n: int, b: int) -> int:
    return int(_load().bcss_num_elems(m, n, b))


def bcss_block_rank(sorted_blk_idx) -> int:
    idx = list(sorted_blk_idx)
    arr = (ctypes.c_int32 * len(idx))(*idx)
    return int(_load().bcss_block_rank(len(idx), arr))


def bcss_block_unrank(m: int, rank: int) -> tuple:
    arr = (ctypes.c_int32 * m)()
    _check("bcss_block_unrank", _load().bcss_block_unrank(m, rank, arr))
    return tuple(arr)


def sttsm_flops(m: int, n: int, p: int, b: int) -> float:
    return float(_load().sttsm_flops(m, n, p, b))


# ---------------------------------------------------------------- device calls

def bcss_pack(dense, bcss, m: int, n: int, b: int, stream=None) -> None:
    if dense.dtype != bcss.dtype:
        raise ValueError("dense and bcss must have the same dtype")
    if dense.numel() != n ** m or bcss.numel() != bcss_num_elems(m, n, b):
        raise ValueError("size mismatch")
    _check("bcss_pack", _load().bcss_pack(_dptr(dense), _dptr(bcss), m, n, b, _dtype_code(dense), _stream(stream)))


def bcss_unpack(bcss, dense, m: int, n: int, b: int, stream=None) -> None:
    if dense.dtype != bcss.dtype:
        raise ValueError("dense and bcss must have the same dtype")
    if dense.numel() != n ** m or bcss.numel() != bcss_num_elems(m, n, b):
        raise ValueError("size mismatch")
    _check("bcss_unpack", _load().bcss_unpack(_dptr(bcss), _dptr(dense), m, n, b, _dtype_code(dense), _stream(stream)))


def sttsm_workspace_size(m: int, n: int, p: int, b: int, prec: int) -> int:
    out = ctypes.c_size_t(0)
    _check("sttsm_workspace_size", _load().sttsm_workspace_size(m, n, p, b, prec, ctypes.byref(out)))
    return int(out.value)


def _check_operands(A, X, C, m, n, p, b, prec):
    import torch
    want = torch.float64 if prec == STTSM_FP64 else torch.float32
    for name, t in (("A", A), ("X", X), ("C", C)):
        if t.dtype != want:
            raise ValueError("%s must be %s for precision %s" % (name, want, PREC_NAMES.get(prec, prec)))
    if A.numel() != bcss_num_elems(m, n, b) or C.numel() != bcss_num_elems(m, p, b) or X.numel() != p * n:
        raise ValueError("size mismatch")


def sttsm_bcss(A, X, m: int, n: int, p: int, b: int, C, prec: int, workspace, stream=None) -> None:
    """C := [A; X, ..., X] on BCSS.  X: p*n elements, column-major (chi_{j,i} at j + i*p)."""
    _check_operands(A, X, C, m, n, p, b, prec)
    ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None and workspace.numel() else ctypes.c_void_p(0)
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("sttsm_bcss", _load().sttsm_bcss(_dptr(A), _dptr(X), m, n, p, b, _dptr(C), prec, ws, nbytes,
                                            _stream(stream)))


def sttsm_all_but_one_elems(m: int, n: int, p: int, b: int) -> int:
    return int(_load().sttsm_all_but_one_elems(m, n, p, b))


def sttsm_all_but_one_flops(m: int, n: int, p: int, b: int) -> float:
    return float(_load().sttsm_all_but_one_flops(m, n, p, b))


def sttsm_bcss_all_but_one(A, X, m: int, n: int, p: int, b: int, T, prec: int, workspace, stream=None) -> None:
    """T := A x_1 X ... x_{m-1} X (mode 0 untransformed) in the partially symmetric
    block storage [node][ib][b^m] of the header; T holds sttsm_all_but_one_elems
    elements.  X: p*n elements, column-major."""
    import torch
    want = torch.float64 if prec == STTSM_FP64 else torch.float32
    for name, t in (("A", A), ("X", X), ("T", T)):
        if t.dtype != want:
            raise ValueError("%s must be %s for precision %s" % (name, want, PREC_NAMES.get(prec, prec)))
    if A.numel() != bcss_num_elems(m, n, b) or X.numel() != p * n or T.numel() != sttsm_all_but_one_elems(m, n, p, b):
        raise ValueError("size mismatch")
    ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None and workspace.numel() else ctypes.c_void_p(0)
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("sttsm_bcss_all_but_one",
           _load().sttsm_bcss_all_but_one(_dptr(A), _dptr(X), m, n, p, b, _dptr(T), prec, ws, nbytes, _stream(stream)))


def sttsm_bcss_noalloc(A, X, m: int, n: int, p: int, b: int, C, prec: int, stream=None) -> None:
    """sttsm_bcss without a caller workspace and without allocating: for callers
    that may not allocate device memory at the call site (fixed memory budgets,
    framework-owned allocators).  Uses the library's fixed 64 MiB device scratch
    array; calls that overlap on the GPU race on it.  The first call on a device
    sets the array up and should come before any stream capture."""
    _check_operands(A, X, C, m, n, p, b, prec)
    _check("sttsm_bcss_noalloc", _load().sttsm_bcss_noalloc(_dptr(A), _dptr(X), m, n, p, b, _dptr(C), prec,
                                                            _stream(stream)))


def sttsm_noalloc_selftest_wait_timeout(limit_ms: float) -> None:
    """Runs the bounded-wait self-test on sttsm_bcss_noalloc's status word; the next
    sttsm_bcss_noalloc call on this device then reports STTSM_ERR_TIMEOUT."""
    _check("sttsm_noalloc_selftest_wait_timeout", _load().sttsm_noalloc_selftest_wait_timeout(float(limit_ms)))


def sttsm_bcss_host(A, X, m: int, n: int, p: int, b: int, C, prec: int, dA, dX, dC, workspace, stream=None) -> None:
    """End-to-end call on host buffers A, X, C (pinned CPU tensors or numpy arrays)."""
    ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None and workspace.numel() else ctypes.c_void_p(0)
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("sttsm_bcss_host", _load().sttsm_bcss_host(_hptr(A), _hptr(X), m, n, p, b, _hptr(C), prec,
                                                      _dptr(dA), _dptr(dX), _dptr(dC), ws, nbytes, _stream(stream)))


class SttsmDesc(ctypes.Structure):
    """sttsm_desc: one instance of a batch (device pointers)."""
    _fields_ = [("A", ctypes.c_void_p), ("X", ctypes.c_void_p), ("C", ctypes.c_void_p), ("m", ctypes.c_int),
                ("n", ctypes.c_int64), ("p", ctypes.c_int64), ("b", ctypes.c_int)]


def sttsm_autotune_b(m: int, n: int, p: int, prec: int, cands=(4, 8, 16)) -> int:
    arr = (ctypes.c_int * len(cands))(*cands)
    rc = _load().sttsm_autotune_b(m, n, p, prec, arr, len(cands))
    if rc <= 0:
        raise SttsmError("sttsm_autotune_b", rc)
    return int(rc)


def sttsm_autotune_b_measured(m: int, n: int, p: int, prec: int, cands=(16, 32, 64), reps: int = 3,
                              with_times: bool = True):
    """Block size by timing each candidate on the device (see the header); returns
    (b, {candidate: median ms or None}) with with_times, else (b, None) using the
    library's cache when it has this shape."""
    import numpy as np
    c = np.array(cands, dtype=np.int32)
    t = np.full(len(cands), -1.0) if with_times else None
    b = _load().sttsm_autotune_b_measured(m, n, p, prec, c.ctypes.data, len(cands), reps,
                                          t.ctypes.data if t is not None else None)
    if b < 0:
        _check("sttsm_autotune_b_measured", b)
    times = {int(k): (float(v) if v >= 0 else None) for k, v in zip(cands, t)} if t is not None else None
    return int(b), times


def _descs(instances):
    """instances: iterables of (A, X, C, m, n, p, b) with CUDA tensors."""
    arr = (SttsmDesc * len(instances))()
    for i, (A, X, C, m, n, p, b) in enumerate(instances):
        arr[i] = SttsmDesc(_dptr(A).value, _dptr(X).value, _dptr(C).value, m, n, p, b)
    return arr


class BatchPlan:
    """sttsm_batch_plan_*: plan once, run (graph replay) many times."""

    def __init__(self, instances, prec: int, ws_budget: int = 0):
        self._keep = list(instances)
        arr = _descs(self._keep)
        h = ctypes.c_void_p(0)
        _check("sttsm_batch_plan_create", _load().sttsm_batch_plan_create(arr, len(self._keep), prec, ws_budget,
                                                                          ctypes.byref(h)))
        self.handle = h
        self.prec = prec

    def workspace_size(self) -> int:
        out = ctypes.c_size_t(0)
        _check("sttsm_batch_workspace_size", _load().sttsm_batch_workspace_size(self.handle, ctypes.byref(out)))
        return int(out.value)

    def info(self) -> dict:
        w, f = ctypes.c_int(0), ctypes.c_double(0.0)
        _check("sttsm_batch_info", _load().sttsm_batch_info(self.handle, ctypes.byref(w), ctypes.byref(f)))
        return {"waves": w.value, "useful_flops": f.value}

    def run(self, workspace, stream=None) -> None:
        nbytes = workspace.numel() * workspace.element_size()
        _check("sttsm_batch_run", _load().sttsm_batch_run(self.handle, ctypes.c_void_p(workspace.data_ptr()), nbytes,
                                                          _stream(stream)))

    def destroy(self) -> None:
        if self.handle:
            _load().sttsm_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sttsm_batch(instances, prec: int, workspace, stream=None) -> None:
    arr = _descs(list(instances))
    nbytes = workspace.numel() * workspace.element_size()
    _check("sttsm_batch", _load().sttsm_batch(arr, len(arr), prec, ctypes.c_void_p(workspace.data_ptr()), nbytes,
                                              _stream(stream)))


class Server:
    """sttsm_serve_*: continuous-batching server under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, prec: int = STTSM_BF16X6, queue_cap: int = 1 << 20):
        h = ctypes.c_void_p(0)
        _check("sttsm_serve_create", _load().sttsm_serve_create(hbm_budget_bytes, prec, queue_cap, ctypes.byref(h)))
        self.handle = h
        self.prec = prec

    def submit(self, A, X, C, m: int, n: int, p: int, b: int) -> int:
        """Queues C := [A; X, ..., X]; returns a ticket.  Raises SttsmError (code STTSM_ERR_BUSY) if full."""
        d = SttsmDesc(_dptr(A).value, _dptr(X).value, _dptr(C).value, m, n, p, b)
        t = ctypes.c_uint64(0)
        _check("sttsm_serve_submit", _load().sttsm_serve_submit(self.handle, ctypes.byref(d), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int):
        """(done, latency_ms)."""
        done, lat = ctypes.c_int(0), ctypes.c_double(0.0)
        _check("sttsm_serve_poll", _load().sttsm_serve_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(lat)))
        return bool(done.value), float(lat.value)

    def stats(self) -> dict:
        out = (ctypes.c_uint64 * 6)()
        _check("sttsm_serve_stats", _load().sttsm_serve_stats(self.handle, out))
        return dict(zip(["submitted", "admitted", "completed", "queued", "active", "arena_bytes"], [int(v) for v in out]))

    def destroy(self) -> None:
        if self.handle:
            _load().sttsm_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


SMALL_F32 = 0
SMALL_TCGEN05 = 1


def sttsm_set_small_kernel(kind: int) -> None:
    """Kernel for contractions n̄ b <= 64 under split precisions: SMALL_F32 (default) or SMALL_TCGEN05."""
    _check("sttsm_set_small_kernel", _load().sttsm_set_small_kernel(kind))


FUSED_TAIL_OFF = 0
FUSED_TAIL_CALLS = 1      # single calls (default)
FUSED_TAIL_ALL = 2        # batch plans and serving too


def sttsm_set_fused_tail(mode: int) -> None:
    """Short contractions: levels m-2 and m-1 as one launch with T^(1) in shared
    memory, or as two launches through the workspace (same bits).  mode:
    FUSED_TAIL_OFF, FUSED_TAIL_CALLS (default), FUSED_TAIL_ALL (True/False map to
    FUSED_TAIL_CALLS/FUSED_TAIL_OFF)."""
    mode = {True: FUSED_TAIL_CALLS, False: FUSED_TAIL_OFF}.get(mode, mode) if isinstance(mode, bool) else int(mode)
    _check("sttsm_set_fused_tail", _load().sttsm_set_fused_tail(mode))


def sttsm_set_inblock_symmetry(on: bool) -> None:
    """Short contractions under split precisions: compute only the canonical entries of
    diagonal blocks (full indices non-decreasing within each symmetric group) and copy
    them to the rest of the block (on), or compute every entry (off, default)."""
    _check("sttsm_set_inblock_symmetry", _load().sttsm_set_inblock_symmetry(int(on)))


def sttsm_selftest_wait_timeout(limit_ms: float) -> int:
    """Runs the bounded-wait self-test; returns the status code (STTSM_ERR_TIMEOUT expected)."""
    return int(_load().sttsm_selftest_wait_timeout(float(limit_ms)))


def sttsm_device_status() -> int:
    return int(_load().sttsm_device_status())


def sttsm_plan_level(m: int, n: int, p: int, b: int, prec: int, d: int):
    """Level-d plan as numpy arrays: (tiles [ntiles x 8] int32, G [P_out x nbar] int32, info dict)."""
    import numpy as np
    L = _load()
    nt, ng = ctypes.c_int64(0), ctypes.c_int64(0)
    info = (ctypes.c_int64 * 9)()
    _check("sttsm_plan_level", L.sttsm_plan_level(m, n, p, b, prec, d, None, 0, None, 0, ctypes.byref(nt),
                                                  ctypes.byref(ng), info))
    tiles = np.zeros((nt.value, 8), dtype=np.int32)
    G = np.zeros(ng.value, dtype=np.int32)
    _check("sttsm_plan_level", L.sttsm_plan_level(m, n, p, b, prec, d, tiles.ctypes.data, nt.value, G.ctypes.data,
                                                  ng.value, None, None, info))
    keys = ["k", "P_parent", "P_out", "rows_per_parent", "nodes_parent", "nodes_out", "R", "bm", "BM"]
    return tiles, G, dict(zip(keys, [int(v) for v in info]))


def sttsm_plan_pair(m: int, n: int, p: int, b: int):
    """Units of the fused last-two-levels launch: (tiles [ntiles x 8] int32, tuples per
    unit); raises SttsmError (STTSM_ERR_UNSUPPORTED) for shapes that do not take it."""
    import numpy as np
    L = _load()
    nt, g = ctypes.c_int64(0), ctypes.c_int32(0)
    _check("sttsm_plan_pair", L.sttsm_plan_pair(m, n, p, b, None, 0, ctypes.byref(nt), ctypes.byref(g)))
    tiles = np.zeros((nt.value, 8), dtype=np.int32)
    _check("sttsm_plan_pair", L.sttsm_plan_pair(m, n, p, b, tiles.ctypes.data, nt.value, None, None))
    return tiles, int(g.value)


def sttsm_plan_sym_rows(m: int, n: int, p: int, b: int, d: int, parent: int, rho0: int = 0, count: int | None = None):
    """Canonical-row map of the in-block-symmetry mode at level d for one parent node:
    (g [count] int64 rows pr * b^(m-1) + rr, -1 past the end; tie [count] uint32; rows of
    the parent).  count None: all of the parent's canonical rows from rho0."""
    import numpy as np
    L = _load()
    rows = ctypes.c_int64(0)
    _check("sttsm_plan_sym_rows", L.sttsm_plan_sym_rows(m, n, p, b, d, parent, 0, 0, None, None, ctypes.byref(rows)))
    if count is None:
        count = max(rows.value - rho0, 0)
    g = np.zeros(count, dtype=np.int64)
    tie = np.zeros(count, dtype=np.uint32)
    _check("sttsm_plan_sym_rows", L.sttsm_plan_sym_rows(m, n, p, b, d, parent, rho0, count, g.ctypes.data,
                                                        tie.ctypes.data, None))
    return g, tie, int(rows.value)


def sttsm_profile_enable(on: bool) -> None:
    _check("sttsm_profile_enable", _load().sttsm_profile_enable(1 if on else 0))


def sttsm_profile_read() -> list[dict]:
    """Recorded launches: dicts with kind ('fp64' | 'tc' | 'tma' | 'split'), level, useful_flops, ms."""
    import numpy as np
    L = _load()
    cnt = ctypes.c_int(0)
    _check("sttsm_profile_read", L.sttsm_profile_read(0, None, None, None, None, ctypes.byref(cnt)))
    n = cnt.value
    kind = np.zeros(n, dtype=np.int32)
    level = np.zeros(n, dtype=np.int32)
    flops = np.zeros(n, dtype=np.float64)
    ms = np.zeros(n, dtype=np.float32)
    _check("sttsm_profile_read", L.sttsm_profile_read(n, kind.ctypes.data, level.ctypes.data, flops.ctypes.data,
                                                      ms.ctypes.data, ctypes.byref(cnt)))
    names = {0: "fp64", 1: "tc", 2: "split", 3: "tma", 4: "pair"}
    return [dict(kind=names[int(k)], level=int(l), useful_flops=float(f), ms=float(t))
            for k, l, f, t in zip(kind, level, flops, ms)]


def workspace_tensor(m: int, n: int, p: int, b: int, prec: int, device=None):
    """A uint8 CUDA tensor of sttsm_workspace_size bytes (torch allocations are 256-byte aligned)."""
    import torch
    return torch.empty(max(sttsm_workspace_size(m, n, p, b, prec), 1), dtype=torch.uint8,
                       device=device if device is not None else "cuda")
