"""Build of the in-tree shared library ``libcde.so`` (sm_103a only).

Each ``csrc/*.cu`` / ``csrc/*.cpp`` translation unit is compiled in parallel
with nvcc, then linked into ``paper_1206_5278_gb300/libcde.so``.  Objects go to
``paper_1206_5278_gb300/_build/`` and are rebuilt when a source or header is
newer than them.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcde.so")
# checked build: device index checks (-DCDE_CHECKS), its own objects and library
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libcde_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                     "-Xcompiler", "-Wno-unused-function"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def build(verbose: bool = False, jobs: int = 0, checks: bool = False) -> str:
    """Compile and link libcde.so (checks=True: libcde_checked.so with the
    device index checks of cde_check_status)."""
    bdir, lib_out = (BUILD_CHECKED, LIB_CHECKED) if checks else (BUILD, LIB)
    flags = NVCC_FLAGS + (["-DCDE_CHECKS"] if checks else [])
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    hdr_t = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    nvcc = _nvcc()

    def obj_of(s):
        return os.path.join(bdir, os.path.basename(s) + ".o")

    def compile_one(s):
        o = obj_of(s)
        if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr_t):
            return o, ""
        cmd = [nvcc] + flags + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (s, r.stdout, r.stderr))
        os.replace(o + ".tmp", o)
        return o, r.stderr

    n = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=n) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(lib_out) or os.path.getmtime(lib_out) < newest:
        tmp = lib_out + ".tmp.%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_out)
    return lib_out


if __name__ == "__main__":
    print(build(verbose=True))
