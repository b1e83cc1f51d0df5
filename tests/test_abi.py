"""The C-ABI library builds, loads and exports every entry point declared in
include/afd.h (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afd.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(afd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1609_03782_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("afd_create", "afd_filter", "afd_destroy", "afd_filter_host",
                     "afd_stats", "afd_noise_rms", "afd_sum", "afd_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (afd_[a-z0-9_]+)\b", out))
    assert set(declared_entry_points()) <= exported


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "afd.h"\nint main(void){ afd_ctx *c = 0; (void)c;'
                   ' return (int)afd_status_str(AFD_OK)[0] == 0; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(src), "-o", str(tmp_path / "use.o")], check=True)


def test_host_side_rejections_need_no_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.afd_status_str.restype = ctypes.c_char_p
    assert lib.afd_status_str(0) == b"AFD_OK"
    assert lib.afd_status_str(1).startswith(b"AFD_EINVAL")
    lib.afd_filter.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                               ctypes.c_int, ctypes.c_int]
    # a null context is rejected before any CUDA call
    assert lib.afd_filter(None, None, 4, 4, 4, None, 1.0, 0.1, 1, 1) == 1
    lib.afd_destroy.argtypes = [ctypes.c_void_p]
    assert lib.afd_destroy(None) == 0
    lib.afd_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.afd_create(None, 0, None) == 1
    vp, i64, f32, ci, f64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_int,
                             ctypes.c_double)
    # the other compute entry points reject a null context the same way
    calls = {
        "afd_filter_rel": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, ci, ci, vp],
                           (None, None, None, 4, 4, 4, None, 1.0, 0.1, 1, 1, None)),
        "afd_filter_host_async": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, ci, ci],
                                  (None, None, None, 4, 4, 4, None, 1.0, 0.1, 1, 1)),
        "afd_filter_slabs": ([vp, vp, vp, vp, i64, i64, i64, vp, f32, f32, ci, ci, i64, ci],
                             (None, None, None, None, 4, 4, 4, None, 1.0, 0.1, 1, 1, 2, 1)),
        "afd_filter_intensity_slabs": ([vp, vp, vp, vp, i64, i64, i64, vp, f32, f32, f32, ci,
                                        i64, ci],
                                       (None, None, None, None, 4, 4, 4, None, 1.5, 1.0, 0.03,
                                        2, 2, 1)),
        "afd_smooth_box": ([vp, vp, vp, i64, i64, i64, vp], (None, None, None, 4, 4, 4, None)),
        "afd_smooth_gauss": ([vp, vp, vp, i64, i64, i64, vp, vp, f32],
                             (None, None, None, 4, 4, 4, None, None, 3.0)),
        "afd_f_diagnostic": ([vp, vp, vp, vp, i64, i64, i64, vp, f64, f64, f64, f64, vp],
                             (None, None, None, None, 4, 4, 4, None, 1.0, 1.0, 2.0, 1.0, None)),
    }
    for name, (argtypes, args) in calls.items():
        fn = getattr(lib, name)
        fn.argtypes = argtypes
        fn.restype = ctypes.c_int
        assert fn(*args) == 1, name


def test_python_binding_has_every_entry_point():
    src = open(os.path.join(ROOT, "paper_1609_03782_gb300", "afd.py")).read()
    for n in declared_entry_points():
        assert ('"%s"' % n) in src, n
