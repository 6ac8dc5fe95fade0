"""Compile the CUDA sources into ``_build/libldpc_gb300.so`` for sm_103a.

Each translation unit is compiled by its own ``nvcc -c`` in parallel and the
objects are linked with ``nvcc -shared``; nothing is rebuilt when the library
is newer than every source and header.  Besides ``csrc/*.cu`` the build
writes one small translation unit per unroll width listed in
``csrc/maxh.cuh`` (``_build/gen/maxh_<width>.cu``), each instantiating the
batch and the persistent decoder of that width, so that the many kernel
instances compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import re
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB_NAME = "libldpc_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the decoder")


GEN_DIR = os.path.join(OUT_DIR, "gen")
_GEN_TEMPLATE = """// Written by build.py: the batch and persistent decoders of unroll width {m}.
#include "decode_persistent.cuh"

template int ldpc_dec::decode_launch<{m}>(const ldpc_code*, const ldpc_dec::DecodeArgs&, int, int, bool,
                                          cudaStream_t);
template int ldpc_dec::persist_launch<{m}>(const ldpc_code*, const ldpc_dec::PersistArgs&, int, int, int, int*,
                                           bool, cudaStream_t);
"""


def unroll_widths():
    """The widths of LDPC_MAXH_LIST in csrc/maxh.cuh."""
    with open(os.path.join(CSRC, "maxh.cuh")) as fh:
        txt = fh.read()
    line = re.search(r"#define LDPC_MAXH_LIST\(X\)(.*)", txt)
    if not line:
        raise RuntimeError("csrc/maxh.cuh: LDPC_MAXH_LIST not found")
    return [int(x) for x in re.findall(r"X\((\d+)\)", line.group(1))]


def _generated():
    """Write (only when changed) and list the per-width translation units."""
    os.makedirs(GEN_DIR, exist_ok=True)
    out = []
    for m in unroll_widths():
        path = os.path.join(GEN_DIR, f"maxh_{m}.cu")
        body = _GEN_TEMPLATE.format(m=m)
        if not os.path.exists(path) or open(path).read() != body:
            with open(path, "w") as fh:
                fh.write(body)
        out.append(path)
    return out


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
            + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Build the library unless it is up to date; returns its path.  Processes
    that start together (ranks of one job, test workers) take a file lock, so
    one of them compiles and the others find the library built."""
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and up_to_date():
                return LIB_PATH
            return _build_locked(verbose, extra)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(verbose: bool, extra) -> str:
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    srcs = _generated() + _sources()  # the big instantiation units first
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]  # cudart linked statically (nvcc default)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    try:  # launch shapes tuned for the previous kernels no longer apply
        os.remove(os.path.join(OUT_DIR, "autotune.json"))
    except FileNotFoundError:
        pass
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
