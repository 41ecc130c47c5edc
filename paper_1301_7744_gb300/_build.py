"""Builds libsttsm.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units compile in parallel into ``_build/``; the shared library
lands in ``_lib/libsttsm.so``.  Both folders are git-ignored.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "_lib" / "libsttsm.so"
SOURCES = ["plan.cu", "capi.cu", "kernels_simt.cu", "kernels_tc.cu", "noalloc.cu", "batch.cu", "serve.cu", "kernels_tma.cu",
           "autotune.cu", "kernels_pair.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I" + str(ROOT / "include"), "-I" + str(CSRC)]


def _headers() -> list[Path]:
    return sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh")) + [ROOT / "include" / "sttsm.h"]


def _stale(out: Path, deps: list[Path]) -> bool:
    return not out.exists() or any(out.stat().st_mtime < d.stat().st_mtime for d in deps)


def compile_commands(force: bool = False) -> list[tuple[list[str], Path]]:
    """nvcc -c commands for the out-of-date objects."""
    BUILD.mkdir(exist_ok=True)
    hdrs = _headers()
    cmds = []
    for src in SOURCES:
        obj = BUILD / (Path(src).stem + ".o")
        if force or _stale(obj, [CSRC / src] + hdrs):
            cmds.append((["nvcc", *NVCC_FLAGS, "-c", str(CSRC / src), "-o", str(obj)], obj))
    return cmds


def link() -> Path:
    objs = [BUILD / (Path(s).stem + ".o") for s in SOURCES]
    if _stale(LIB, objs):
        LIB.parent.mkdir(exist_ok=True)
        tmp = LIB.with_suffix(".so.tmp%d" % os.getpid())
        subprocess.run(["nvcc", ARCH, "-shared", *map(str, objs), "-o", str(tmp)], check=True)
        os.replace(tmp, LIB)
    return LIB


def run_parallel(cmds: list[list[str]]) -> None:
    procs = [(c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for c in cmds]
    failed = []
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((c, out.decode(errors="replace")))
    if failed:
        msg = "\n".join("$ %s\n%s" % (" ".join(c), o) for c, o in failed)
        raise RuntimeError("build failed:\n" + msg)


def build(force: bool = False, extra: list[list[str]] | None = None) -> Path:
    """Compile every out-of-date translation unit (plus any extra commands) in parallel, then link."""
    cmds = [c for c, _ in compile_commands(force)] + list(extra or [])
    if cmds:
        run_parallel(cmds)
    return link()
