"""Build libafd.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
object next to this file.  The CUDA runtime is linked statically; the driver
is reached at run time through the runtime's entry-point query.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libafd.so")
# the debug build with bounds checks in the kernels (-DAFD_CHECK)
LIB_CHECKED = os.path.join(HERE, "libafd_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["afd_api.cu", "pm_simple.cu", "pm_stream.cu", "reduce.cu", "selftest.cu",
           "noalloc.cu", "quant.cu", "tb_host.cu", "pm_tb_f32.cu", "pm_tb_f16.cu",
           "pm_tb_bf16.cu", "pm_tb_i16.cu", "pm_batch.cu",
           "serve.cu", "fdiag.cu", "smooth.cu", "smooth_direct.cu", "passes.cu",
           "pm_wide.cu", "pm_wide2.cu"]
HEADERS = ["afd_math.cuh", "afd_ptx.cuh", "afd_internal.h", "afd_store.cuh", "pm_tb.cuh",
           "pm_tb_impl.cuh", "afd_ctx.h", "afd_batch.h", "afd_trace.h", "afd_check.cuh",
           "pm_block.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no multiply/add contraction of scalar code anywhere; every FMA
# the kernels want is written explicitly (afd_math.cuh also guards the packed
# f32x2 products, which this flag does not cover, by forming them as FMAs).
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libafd.so")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(INCLUDE, "afd.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def up_to_date(lib: str = LIB) -> bool:
    return os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input()


def _extra_flags():
    """Extra nvcc flags from AFD_NVCC_FLAGS (tuning builds, e.g.
    -DAFD_STREAM_SLOTS=4 -DAFD_STREAM_MIN_BLOCKS=3)."""
    return os.environ.get("AFD_NVCC_FLAGS", "").split()


def _compile(src: str, verbose: bool, objdir: str = BUILD, defines=()) -> str:
    obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *defines, *_extra_flags(), "-c", os.path.join(CSRC, src),
           "-o", obj]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, res.stdout, res.stderr))
    if verbose and res.stderr:
        print(res.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every kernel and the C ABI into libafd.so (in-tree); with
    checked=True, the bounds-checked debug build libafd_check.so instead."""
    lib = LIB_CHECKED if checked else LIB
    objdir = os.path.join(BUILD, "checked") if checked else BUILD
    defines = ("-DAFD_CHECK",) if checked else ()
    if not force and up_to_date(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, objdir, defines), SOURCES))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt",
           "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (res.stdout, res.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
