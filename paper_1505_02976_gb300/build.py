"""Build of the CUDA library (``liblbm_gb300.so``) for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library inside the package (``_build/``), so the
library that the binding loads is always the in-tree one.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-ftz=true", "-prec-div=false", "-prec-sqrt=false",
              "-I", INCLUDE] + ARCH
_lock = threading.Lock()


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    d = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    d.append(os.path.join(INCLUDE, "lbm.h"))
    return d


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link the library; returns its path."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(OUT, exist_ok=True)
        nvcc = _nvcc()
        procs, objs = [], []
        for src in sources():
            obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        errors = []
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose and out:
                print(out.decode(errors="replace"))
            if p.returncode != 0:
                errors.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"], check=True)
        os.replace(tmp, LIB)
        return LIB
