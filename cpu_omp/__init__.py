"""Multithreaded FP32 CPU build of the per-face filter (OpenMP, portable C).

The host-side baseline the GPU library is measured against: the same method
(Sec. 3.3, per-face conductance, zero-flux faces, n Jacobi iterations) in
float32 on every host core, in the role of the paper's OpenMP implementation
(Sec. 6).  It shares no code with the CUDA library or with the FP64 oracle;
``bench.py`` times it and the CPU tests check it against the oracle.

filter(cube, K, dt, n_iter, conductance, spacing, threads) -> new array
max_threads()                  OpenMP's default thread count
stream_copy_gbs(bytes, reps)   host STREAM-copy bandwidth (read + write GB/s)
cpu_model()                    the host CPU's name (from /proc/cpuinfo or lscpu)
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afd_omp.c")
_LIB = os.path.join(_HERE, "libafd_omp.so")
_lock = threading.Lock()
_lib = None
_COND = {"exponential": 0, "rational": 1}


def build(force: bool = False) -> str:
    """Compile with gcc: -O3 (vectorised x loops), OpenMP, no FP contraction,
    no target-specific flags (the same source builds on x86-64 and arm64)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, c_int, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.afd_omp_filter.argtypes = [vp, i64, i64, i64, vp, ctypes.c_float,
                                           ctypes.c_float, c_int, c_int, c_int]
            lib.afd_omp_filter.restype = c_int
            lib.afd_omp_max_threads.restype = c_int
            lib.afd_omp_stream_copy.argtypes = [i64, c_int, c_int]
            lib.afd_omp_stream_copy.restype = ctypes.c_double
            _lib = lib
    return _lib


def filter_inplace(cube: np.ndarray, K: float, dt: float, n_iter: int,
                   conductance: str = "rational", spacing=None, threads: int = 0) -> None:
    """The filter on a C-contiguous float32 (nz, ny, nx) array, in place."""
    if cube.dtype != np.float32 or cube.ndim != 3 or not cube.flags["C_CONTIGUOUS"]:
        raise ValueError("cube must be a C-contiguous float32 (nz, ny, nx) array")
    nz, ny, nx = cube.shape
    sp = None
    if spacing is not None:
        sp = (ctypes.c_float * 3)(*[float(h) for h in spacing])
    rc = _load().afd_omp_filter(cube.ctypes.data, nx, ny, nz, sp, float(K), float(dt),
                                int(n_iter), _COND[conductance], int(threads))
    if rc == -1:
        raise ValueError("invalid argument")
    if rc != 0:
        raise MemoryError("afd_omp_filter could not allocate its buffers")


def filter(cube: np.ndarray, K: float, dt: float, n_iter: int, conductance: str = "rational",
           spacing=None, threads: int = 0) -> np.ndarray:
    """n_iter iterations on a float32 copy of `cube`; returns the copy."""
    out = np.array(cube, dtype=np.float32, order="C", copy=True)
    filter_inplace(out, K, dt, n_iter, conductance, spacing, threads)
    return out


def max_threads() -> int:
    return int(_load().afd_omp_max_threads())


def stream_copy_gbs(nbytes: int = 1 << 30, reps: int = 5, threads: int = 0) -> float:
    return float(_load().afd_omp_stream_copy(int(nbytes), int(reps), int(threads)))


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()
