"""Build libfstat.so in-tree with nvcc for sm_103a (no CMake).

Each translation unit under csrc/ compiles in parallel to an object file in
_build/, then nvcc links the shared library next to this file.  A rebuild
happens only when a source or header is newer than the library.
"""

from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libfstat.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no floating-point contraction, so host arithmetic (template
# shifts, validation) rounds the same on x86-64 and aarch64
# host code: hidden visibility, so only the fstat_* entry points (declared
# default-visible in fstat.h) are exported and template statics stay private
# to each build of the library
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr", "-I" + INCLUDE] + ARCH


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfstat")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [
        os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every CUDA source and link libfstat.so; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def build_variant(tag: str, defines, units=("sky.cu",), verbose: bool = False) -> str:
    """A second build of the library in which ``units`` are compiled with
    the extra preprocessor ``defines`` (the other objects are the regular
    build's): _build/libfstat_<tag>.so.  ``units``: file names under csrc/.  Used by tests that need a
    deliberately degraded library (the precision negative control)."""
    build(verbose=verbose)
    nvcc = _nvcc()
    out_dir = os.path.join(BUILD, tag)
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(BUILD, f"libfstat_{tag}.so")
    flags = [f"-D{d}" for d in defines]
    objs = []
    for src in sources():
        name = os.path.basename(src)
        if name in units:
            obj = os.path.join(out_dir, name + ".o")
            r = subprocess.run([nvcc, *NVCC_FLAGS, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {name} ({tag}):\n" + r.stdout + r.stderr)
        else:
            obj = os.path.join(BUILD, name + ".o")
        objs.append(obj)
    r = subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", lib, *objs,
                        "-Xlinker", "-rpath,/usr/local/cuda/lib64"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
