"""Builds the in-tree CUDA library ``libcf.so`` (sm_103a) from ``csrc/``.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically.  Re-running is cheap:
objects are rebuilt only when a source or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf_futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", os.path.join(os.path.dirname(HERE), "include")]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_header():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "cf.h")]
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, ptxas_info: bool = False, jobs: int | None = None, defines=(),
          out: str | None = None, build_dir: str | None = None) -> str:
    """Compiles csrc/ into LIB (or `out`); `defines` are extra -D macros
    (build-time tunables such as CF_E32 or CF_ROWS_MINB) compiled into a
    separate object directory."""
    lib = out or LIB
    bdir = build_dir or BUILD
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_time = _newest_header()
    objs, todo = [], []
    for src in srcs:
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if (not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time)
                or ptxas_info):
            todo.append((src, obj))

    def compile_one(item):
        src, obj = item
        cmd = [_nvcc()] + ARCH + NVCC_FLAGS + ["-D" + d for d in defines] + \
            (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return src, r.stderr

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf_futures.ThreadPoolExecutor(max_workers=n) as ex:
            for src, err in ex.map(compile_one, todo):
                if verbose or ptxas_info:
                    sys.stderr.write("== %s\n%s" % (os.path.basename(src), err))
    if todo or not os.path.exists(lib):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
