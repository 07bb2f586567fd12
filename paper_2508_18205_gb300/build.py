"""Builds libmfd.so (the CUDA library behind include/mfd.h) in-tree for sm_103a.

Each translation unit (CUDA .cu, host-only .cpp) is compiled by its own nvcc
process (in parallel), then
linked into paper_2508_18205_gb300/_build/libmfd.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmfd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-Wall"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _stale(lib_path, deps):
    if not os.path.exists(lib_path):
        return True
    t = os.path.getmtime(lib_path)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), bounds: bool = False) -> str:
    """Compiles libmfd.so; with bounds=True the bounds-checked debug build
    (MFD_BOUNDS_CHECK, every stencil index tested before a gather) into
    _build_bounds/libmfd.so instead (load it with MFD_LIB=<path>)."""
    if bounds:
        return _build(os.path.join(HERE, "_build_bounds"), force, verbose, (*extra, "-DMFD_BOUNDS_CHECK"))
    return _build(OUT, force, verbose, extra)


def _build(out_dir, force, verbose, extra):
    lib_path = os.path.join(out_dir, "libmfd.so")
    srcs = sources()
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(HERE, "..", "include", "mfd.h"))
    deps.append(os.path.abspath(__file__))
    if not force and not _stale(lib_path, deps):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    objs = [os.path.join(out_dir, os.path.splitext(os.path.basename(s))[0] + ".o") for s in srcs]

    def one(args):
        src, obj = args
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(one, zip(srcs, objs)))
    bad = [(s, out) for s, rc, out in results if rc != 0]
    for s, rc, out in results:
        if verbose and out.strip():
            print(f"--- {os.path.basename(s)}\n{out}", file=sys.stderr)
    if bad:
        msg = "\n".join(f"{os.path.basename(s)}:\n{out}" for s, out in bad)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    v = "-v" in sys.argv
    ex = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(ex), extra=ex))
