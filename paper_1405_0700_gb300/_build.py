"""Build libplq.so (the CUDA library behind the C ABI in include/plq.h).

Compiles every ``csrc/*.cu`` for sm_103a with nvcc, in parallel, into
``_build/`` and links them into ``libplq.so`` next to this file.  Objects are
rebuilt when a source or header is newer than them.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libplq.so")
INCLUDE = os.path.join(ROOT, "include")
# The debug build: the same sources compiled with -DPLQ_DEBUG (device bounds
# guards that record PLQ_ERR_BOUNDS in the context's status word instead of
# accessing out of range), in its own object folder and library.
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libplq_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
    "-I" + INCLUDE, "-I" + CSRC,
]


def nvcc():
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libplq.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, jobs=None, extra_flags=(), debug=False):
    """Compile and link libplq.so (with debug=True: libplq_debug.so, the
    PLQ_DEBUG build); returns its path."""
    build_dir, lib_path = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if debug:
        extra_flags = tuple(extra_flags) + ("-DPLQ_DEBUG",)
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = _headers()
    nv = nvcc()
    jobs_todo = []
    objs = []
    for src in srcs:
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if _stale(obj, [src] + hdrs):
            jobs_todo.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nv] + NVCC_FLAGS + list(extra_flags) + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        os.replace(obj + ".tmp", obj)
        return src, r.stderr

    n = jobs or min(len(jobs_todo), os.cpu_count() or 4) or 1
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        for src, err in ex.map(compile_one, jobs_todo):
            if verbose:
                print("compiled", os.path.basename(src), err.strip())
    if _stale(lib_path, objs) or jobs_todo:
        tmp = lib_path + ".tmp%d" % os.getpid()
        cmd = [nv] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys

    print(build(verbose="-v" in sys.argv))
