"""Build libfntrs.so (sm_103a) in-tree with nvcc.

Translation units are compiled in parallel, then linked into
``paper_0907_1788_gb300/_build/libfntrs.so``.  No CMake, no torch extension:
the library exposes a plain C ABI (``include/fnt_rs.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfntrs.so")
# debug build: device index checks (FNTRS_DEBUG_BOUNDS, csrc/dbg.cuh) in a folder of its own
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libfntrs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills"]
SOURCES = ["plan.cu", "pattern.cu", "inst_small.cu", "inst_mid.cu", "inst_big.cu",
           "inst_huge.cu", "inst_split.cu", "noalloc.cu", "ragged.cu", "ragged_kernel.cu", "server.cu",
           "systematic.cu", "wire.cu",
           "hostpipe.cu", "paper_route.cu",
           "direct.cu",
           "inst_fold.cu"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfntrs")
    return cand


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(os.path.dirname(HERE), "include", "fnt_rs.h"))
    return files


def build(force: bool = False, verbose: bool = False, extra_flags=(),
          debug_bounds: bool = False) -> str:
    """Compile and link the library; returns its path.

    debug_bounds=True builds the variant with device index checks
    (-DFNTRS_DEBUG_BOUNDS=1) into _build_debug/ instead of _build/."""
    out_dir, lib_path = (OUT_DEBUG, LIB_DEBUG) if debug_bounds else (OUT, LIB)
    if debug_bounds:
        extra_flags = (*extra_flags, "-DFNTRS_DEBUG_BOUNDS=1")
    os.makedirs(out_dir, exist_ok=True)
    stamp = os.path.join(out_dir, "stamp.txt")
    digest = _digest(_inputs()) + ("|" + " ".join(extra_flags) if extra_flags else "")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        if open(stamp).read() == digest:
            return lib_path
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
