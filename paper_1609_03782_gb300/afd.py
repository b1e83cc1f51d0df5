"""Python binding of libafd.so: argument marshalling only.

Every function has the name of the C entry point it calls (include/afd.h) and
does no arithmetic of its own: it turns tensors into pointers and sizes, the
calling thread's current torch CUDA stream into the context's stream, and
non-zero status codes into ``AfdError``.  Cubes are torch tensors shaped
(nz, ny, nx), x fastest, as the C ABI lays them out.  There is no CPU
fallback: if libafd.so is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafd.so")
# AFD_LIB selects another build of the same ABI (the bounds-checked debug
# build, libafd_check.so); there is no fallback if it is missing either.
LIB_PATH = os.environ.get("AFD_LIB", LIB_PATH)

AFD_OK, AFD_EINVAL, AFD_ENOMEM, AFD_ECUDA, AFD_ETIMEOUT, AFD_EBUSY = range(6)
COND = {"exponential": 0, "rational": 1}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2, "i16": 3}
KERNEL = {"auto": 0, "simple": 1, "stream": 2, "two_stage": 3}


class AfdError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = "%s failed: %s" % (what, _lib.afd_status_str(status).decode())
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libafd.so is not built (run __graft_entry__.build() or "
                          "python -m paper_1609_03782_gb300._build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, f32, c_int, dp = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                               ctypes.c_int, ctypes.c_void_p)
    sig = {
        "afd_create": ([ctypes.POINTER(vp), c_int, vp], c_int),
        "afd_destroy": ([vp], c_int),
        "afd_set_stream": ([vp, vp], c_int),
        "afd_set_kernel": ([vp, c_int], c_int),
        "afd_set_stream_zchunk": ([vp, c_int], c_int),
        "afd_filter": ([vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int], c_int),
        "afd_filter_out": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int], c_int),
        "afd_filter_host": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int], c_int),
        "afd_filter_host_async": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int], c_int),
        "afd_filter_slabs": ([vp, vp, vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int, i64,
                              c_int], c_int),
        "afd_filter_rel": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int, vp], c_int),
        "afd_f_diagnostic": ([vp, vp, vp, vp, i64, i64, i64, vp, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, vp], c_int),
        "afd_smooth_box": ([vp, vp, vp, i64, i64, i64, vp], c_int),
        "afd_smooth_gauss": ([vp, vp, vp, i64, i64, i64, vp, vp, f32], c_int),
        "afd_pass_timing": ([vp, c_int], c_int),
        "afd_check_violations": ([vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                  ctypes.POINTER(c_int)], c_int),
        "afd_checked_build": ([], c_int),
        "afd_pass_timing_read": ([vp, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64)], c_int),
        "afd_filter_intensity": ([vp, vp, vp, i64, i64, i64, vp, f32, f32, f32, c_int], c_int),
        "afd_filter_intensity_slabs": ([vp, vp, vp, vp, i64, i64, i64, vp, f32, f32, f32, c_int,
                                        i64, c_int], c_int),
        "afd_selftest_wait": ([vp, i64], c_int),
        "afd_quantize": ([vp, vp, vp, i64, c_int, f32], c_int),
        "afd_dequantize": ([vp, vp, vp, i64, c_int, f32], c_int),
        "afd_filter_ex": ([vp, vp, vp, c_int, f32, i64, i64, i64, vp, f32, f32, c_int, c_int,
                           c_int], c_int),
        "afd_batch_create": ([vp, ctypes.POINTER(vp), c_int, vp, c_int, f32], c_int),
        "afd_batch_set": ([vp, c_int, vp], c_int),
        "afd_batch_get": ([vp, c_int, vp], c_int),
        "afd_batch_filter": ([vp, vp, vp, f32, c_int, c_int], c_int),
        "afd_batch_k": ([vp, vp], c_int),
        "afd_batch_set_zchunk": ([vp, c_int], c_int),
        "afd_batch_set_tiles": ([vp, c_int], c_int),
        "afd_batch_destroy": ([vp], c_int),
        "afd_serve_create": ([vp, vp, ctypes.c_size_t, c_int, ctypes.POINTER(vp)], c_int),
        "afd_serve_submit": ([vp, c_int, f32, f32, c_int, c_int,
                              ctypes.POINTER(ctypes.c_uint64)], c_int),
        "afd_serve_step": ([vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)], c_int),
        "afd_serve_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(c_int),
                            ctypes.POINTER(ctypes.c_double)], c_int),
        "afd_serve_times": ([vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)], c_int),
        "afd_serve_result": ([vp, ctypes.c_uint64, vp], c_int),
        "afd_serve_release": ([vp, ctypes.c_uint64], c_int),
        "afd_serve_free_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], c_int),
        "afd_serve_destroy": ([vp], c_int),
        "afd_filter_noalloc": ([vp, vp, i64, i64, i64, vp, f32, f32, c_int, c_int, vp], c_int),
        "afd_stats": ([vp, vp, i64, vp], c_int),
        "afd_noise_rms": ([vp, vp, i64, dp], c_int),
        "afd_sum": ([vp, vp, i64, dp], c_int),
        "afd_sync": ([vp], c_int),
        "afd_launch_count": ([vp, ctypes.POINTER(ctypes.c_uint64)], c_int),
        "afd_status_str": ([c_int], ctypes.c_char_p),
        "afd_last_error_string": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def exported_symbols():
    """Names of the entry points this binding declares."""
    return sorted(n for n in dir(_lib) if n.startswith("afd_"))


class Context:
    """Owns one afd_ctx*.  Not thread-safe: use one per host thread."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = ctypes.c_void_p()
        _check(_lib.afd_create(ctypes.byref(h), self.device, None), "afd_create", None)
        self.handle = h

    def close(self):
        if self.handle:
            _lib.afd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check(status: int, what: str, ctx: Context | None):
    if status != AFD_OK:
        detail = ""
        if ctx is not None and ctx.handle:
            detail = _lib.afd_last_error_string(ctx.handle).decode()
        raise AfdError(status, what, detail)


def _use_current_stream(ctx: Context, t: torch.Tensor | None = None):
    dev = t.device if t is not None and t.is_cuda else torch.device("cuda", ctx.device)
    s = torch.cuda.current_stream(dev).cuda_stream
    _check(_lib.afd_set_stream(ctx.handle, ctypes.c_void_p(s)), "afd_set_stream", ctx)


def _cube_args(cube: torch.Tensor):
    if cube.dim() != 3:
        raise ValueError("cube must be 3-D, shaped (nz, ny, nx)")
    if not cube.is_contiguous():
        raise ValueError("cube must be contiguous")
    nz, ny, nx = cube.shape
    return ctypes.c_void_p(cube.data_ptr()), nx, ny, nz


def _spacing(spacing):
    if spacing is None:
        return None
    arr = (ctypes.c_float * 3)(*[float(s) for s in spacing])
    return arr


def afd_create(device: int = 0) -> Context:
    return Context(device)


def afd_destroy(ctx: Context) -> None:
    ctx.close()


def afd_set_kernel(ctx: Context, kernel: str) -> None:
    _check(_lib.afd_set_kernel(ctx.handle, KERNEL[kernel]), "afd_set_kernel", ctx)


def afd_set_stream_zchunk(ctx: Context, zc: int) -> None:
    _check(_lib.afd_set_stream_zchunk(ctx.handle, int(zc)), "afd_set_stream_zchunk", ctx)


def afd_filter(ctx: Context, cube: torch.Tensor, K: float, dt: float, n_iter: int,
               conductance: str = "rational", spacing=None) -> torch.Tensor:
    """Filter a float32 CUDA tensor in place on the current stream; returns it."""
    if cube.dtype != torch.float32 or not cube.is_cuda:
        raise ValueError("afd_filter takes a float32 CUDA tensor")
    p, nx, ny, nz = _cube_args(cube)
    _use_current_stream(ctx, cube)
    sp = _spacing(spacing)
    _check(_lib.afd_filter(ctx.handle, p, nx, ny, nz, sp, float(K), float(dt), int(n_iter),
                           COND[conductance]), "afd_filter", ctx)
    return cube


def afd_filter_out(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor, K: float,
                   dt: float, n_iter: int, conductance: str = "rational",
                   spacing=None) -> torch.Tensor:
    """Out-of-place filter of float32 CUDA tensors on the current stream."""
    for t in (cube_in, cube_out):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError("afd_filter_out takes float32 CUDA tensors")
    if cube_in.shape != cube_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    _use_current_stream(ctx, cube_in)
    _check(_lib.afd_filter_out(ctx.handle, p_in, p_out, nx, ny, nz, _spacing(spacing),
                               float(K), float(dt), int(n_iter), COND[conductance]),
           "afd_filter_out", ctx)
    return cube_out


def afd_filter_intensity(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor,
                         K: float, rms: float, tau: float, n_iter: int,
                         C=(5.0, 5.0, 5.0)) -> torch.Tensor:
    """The paper's intensity-driven filter (K in units of rms), out of place."""
    for t in (cube_in, cube_out):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError("afd_filter_intensity takes float32 CUDA tensors")
    if cube_in.shape != cube_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    _use_current_stream(ctx, cube_in)
    c = (ctypes.c_float * 3)(*[float(v) for v in C])
    _check(_lib.afd_filter_intensity(ctx.handle, p_in, p_out, nx, ny, nz, c, float(K),
                                     float(rms), float(tau), int(n_iter)),
           "afd_filter_intensity", ctx)
    return cube_out


def afd_filter_host(ctx: Context, host_in: torch.Tensor, host_out: torch.Tensor, K: float,
                    dt: float, n_iter: int, conductance: str = "rational",
                    spacing=None) -> torch.Tensor:
    """Filter float32 CPU tensors (pinned or pageable) through the device;
    synchronous, host<->device copies included."""
    for t in (host_in, host_out):
        if t.dtype != torch.float32 or t.is_cuda:
            raise ValueError("afd_filter_host takes float32 CPU tensors")
    if host_in.shape != host_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(host_in)
    p_out, _, _, _ = _cube_args(host_out)
    _use_current_stream(ctx)
    _check(_lib.afd_filter_host(ctx.handle, p_in, p_out, nx, ny, nz, _spacing(spacing),
                                float(K), float(dt), int(n_iter), COND[conductance]),
           "afd_filter_host", ctx)
    return host_out


def afd_filter_rel(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor, k_rms: float,
                   dt: float, n_iter: int, conductance: str = "rational", spacing=None,
                   K_out: torch.Tensor | None = None) -> torch.Tensor:
    """afd_filter_out with K = k_rms x (noise rms of cube_in), computed on the
    device; K_out (a CUDA float32 tensor of one element) receives K."""
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    if cube_in.shape != cube_out.shape or cube_in.dtype != torch.float32 or \
            cube_out.dtype != torch.float32:
        raise ValueError("float32 cubes of one shape expected")
    kp = None
    if K_out is not None:
        if not K_out.is_cuda or K_out.dtype != torch.float32 or K_out.numel() < 1:
            raise ValueError("K_out must be a CUDA float32 tensor")
        kp = ctypes.c_void_p(K_out.data_ptr())
    _use_current_stream(ctx, cube_in)
    _check(_lib.afd_filter_rel(ctx.handle, p_in, p_out, nx, ny, nz, _spacing(spacing),
                               float(k_rms), float(dt), int(n_iter), COND[conductance], kp),
           "afd_filter_rel", ctx)
    return cube_out


def _smooth_args(cube_in: torch.Tensor, cube_out: torch.Tensor):
    for t in (cube_in, cube_out):
        if not t.is_cuda or t.dtype != torch.float32:
            raise ValueError("CUDA float32 cubes expected")
    if cube_in.shape != cube_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    return p_in, p_out, nx, ny, nz


def afd_smooth_box(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor, N) -> torch.Tensor:
    """Box (mean) filter of odd window N = (N_x, N_y, N_z) (Sec. 3.1)."""
    p_in, p_out, nx, ny, nz = _smooth_args(cube_in, cube_out)
    n = (ctypes.c_int * 3)(*[int(v) for v in N])
    _use_current_stream(ctx, cube_in)
    _check(_lib.afd_smooth_box(ctx.handle, p_in, p_out, nx, ny, nz, n), "afd_smooth_box", ctx)
    return cube_out


def afd_smooth_gauss(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor, fwhm,
                     angles_deg=None, truncate: float = 0.0) -> torch.Tensor:
    """Gaussian filter (Sec. 3.2): FWHM per axis, optional Euler rotation
    (degrees), truncation in sigma (0 = 3)."""
    p_in, p_out, nx, ny, nz = _smooth_args(cube_in, cube_out)
    f = (ctypes.c_float * 3)(*[float(v) for v in fwhm])
    a = None if angles_deg is None else (ctypes.c_float * 3)(*[float(v) for v in angles_deg])
    _use_current_stream(ctx, cube_in)
    _check(_lib.afd_smooth_gauss(ctx.handle, p_in, p_out, nx, ny, nz, f, a, float(truncate)),
           "afd_smooth_gauss", ctx)
    return cube_out


class FDiag(ctypes.Structure):
    _fields_ = [("S_of", ctypes.c_double), ("S_oo", ctypes.c_double),
                ("S_mf", ctypes.c_double), ("S_m", ctypes.c_double),
                ("N_o", ctypes.c_int64), ("N_f", ctypes.c_int64),
                ("rms_o", ctypes.c_double), ("rms_f", ctypes.c_double),
                ("F", ctypes.c_double), ("sigma_F", ctypes.c_double),
                ("F_M", ctypes.c_double)]


def afd_f_diagnostic(ctx: Context, orig: torch.Tensor, filt: torch.Tensor,
                     model: torch.Tensor | None = None, roi=None, rms_o: float = 0.0,
                     rms_f: float = 0.0, nsig: float = 3.0, beam: float = 1.0) -> dict:
    """F, sigma_F and F_M (and the sums behind them) of a filtered cube
    against its original over roi = (x0, x1, y0, y1, z0, z1); rms <= 0 means
    estimate it on the full cube."""
    cubes = [orig, filt] + ([model] if model is not None else [])
    for t in cubes:
        if not t.is_cuda or t.dtype != torch.float32 or t.shape != orig.shape:
            raise ValueError("CUDA float32 cubes of one shape expected")
    p_o, nx, ny, nz = _cube_args(orig)
    p_f, _, _, _ = _cube_args(filt)
    p_m = _cube_args(model)[0] if model is not None else None
    box = None
    if roi is not None:
        box = (ctypes.c_int64 * 6)(*[int(v) for v in roi])
    _use_current_stream(ctx, orig)
    r = FDiag()
    _check(_lib.afd_f_diagnostic(ctx.handle, p_o, p_f, p_m, nx, ny, nz, box, float(rms_o),
                                 float(rms_f), float(nsig), float(beam), ctypes.byref(r)),
           "afd_f_diagnostic", ctx)
    return {name: getattr(r, name) for name, _ in FDiag._fields_}


def afd_check_violations(ctx: Context):
    """(count, first code, first index) of the bounds-check violations since
    the last call (always count 0 in the release build); clears them."""
    n, code, idx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.afd_check_violations(ctx.handle, ctypes.byref(n), ctypes.byref(code),
                                     ctypes.byref(idx)), "afd_check_violations", ctx)
    return n.value, code.value, idx.value


def afd_checked_build() -> bool:
    return bool(_lib.afd_checked_build())


def afd_pass_timing(ctx: Context, on: bool) -> None:
    _check(_lib.afd_pass_timing(ctx.handle, 1 if on else 0), "afd_pass_timing", ctx)


def afd_pass_timing_read(ctx: Context):
    """(summed device ms, passes) of the pass sequences recorded since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.afd_pass_timing_read(ctx.handle, ctypes.byref(ms), ctypes.byref(n)),
           "afd_pass_timing_read", ctx)
    return ms.value, n.value


def afd_filter_host_async(ctx: Context, host_in: torch.Tensor, host_out: torch.Tensor,
                          K: float, dt: float, n_iter: int, conductance: str = "rational",
                          spacing=None) -> torch.Tensor:
    """Enqueue afd_filter_host without waiting (copies on context-owned copy
    streams, passes on the current stream); host_out is valid after
    afd_sync.  Pinned tensors let consecutive calls overlap."""
    for t in (host_in, host_out):
        if t.dtype != torch.float32 or t.is_cuda:
            raise ValueError("afd_filter_host_async takes float32 CPU tensors")
    if host_in.shape != host_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(host_in)
    p_out, _, _, _ = _cube_args(host_out)
    _use_current_stream(ctx)
    _check(_lib.afd_filter_host_async(ctx.handle, p_in, p_out, nx, ny, nz, _spacing(spacing),
                                      float(K), float(dt), int(n_iter), COND[conductance]),
           "afd_filter_host_async", ctx)
    return host_out


def afd_filter_slabs(ctx: Context, host_in: torch.Tensor, host_out: torch.Tensor, K: float,
                     dt: float, n_iter: int, conductance: str = "rational", spacing=None,
                     slab_nz: int = 64, halo: int = 8, host_tmp: torch.Tensor = None
                     ) -> torch.Tensor:
    """Filter a float32 CPU cube through the device in z-slabs of slab_nz
    planes, in rounds of up to `halo` iterations (device memory: four slabs
    of slab_nz + 2 halo planes); synchronous.  Bit-identical to afd_filter on
    the whole cube.  host_tmp (a cube-sized CPU tensor) is needed when
    n_iter > halo; pinned tensors let the copies overlap the passes."""
    for t in (host_in, host_out) + ((host_tmp,) if host_tmp is not None else ()):
        if t.dtype != torch.float32 or t.is_cuda:
            raise ValueError("afd_filter_slabs takes float32 CPU tensors")
        if t.shape != host_in.shape:
            raise ValueError("afd_filter_slabs: shapes differ")
    p_in, nx, ny, nz = _cube_args(host_in)
    p_out, _, _, _ = _cube_args(host_out)
    p_tmp = _cube_args(host_tmp)[0] if host_tmp is not None else None
    _use_current_stream(ctx)
    _check(_lib.afd_filter_slabs(ctx.handle, p_in, p_out, p_tmp, nx, ny, nz, _spacing(spacing),
                                 float(K), float(dt), int(n_iter), COND[conductance],
                                 int(slab_nz), int(halo)),
           "afd_filter_slabs", ctx)
    return host_out


def afd_filter_intensity_slabs(ctx: Context, host_in: torch.Tensor, host_out: torch.Tensor,
                               K: float, rms: float, tau: float, n_iter: int,
                               C=(5.0, 5.0, 5.0), slab_nz: int = 64, halo: int = 8,
                               host_tmp: torch.Tensor = None) -> torch.Tensor:
    """The paper's intensity-driven filter on a float32 CPU cube, through the
    device in z-slabs as afd_filter_slabs; synchronous.  Bit-identical to
    afd_filter_intensity on the whole cube."""
    for t in (host_in, host_out) + ((host_tmp,) if host_tmp is not None else ()):
        if t.dtype != torch.float32 or t.is_cuda:
            raise ValueError("afd_filter_intensity_slabs takes float32 CPU tensors")
        if t.shape != host_in.shape:
            raise ValueError("afd_filter_intensity_slabs: shapes differ")
    p_in, nx, ny, nz = _cube_args(host_in)
    p_out, _, _, _ = _cube_args(host_out)
    p_tmp = _cube_args(host_tmp)[0] if host_tmp is not None else None
    _use_current_stream(ctx)
    c = (ctypes.c_float * 3)(*[float(v) for v in C])
    _check(_lib.afd_filter_intensity_slabs(ctx.handle, p_in, p_out, p_tmp, nx, ny, nz, c,
                                           float(K), float(rms), float(tau), int(n_iter),
                                           int(slab_nz), int(halo)),
           "afd_filter_intensity_slabs", ctx)
    return host_out


STORAGE_DTYPE = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16,
                 "i16": torch.int16}


def _storage_tensor(t: torch.Tensor, storage: str, what: str):
    if STORAGE_DTYPE[storage] != t.dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s: expected a contiguous %s CUDA tensor for storage %r"
                         % (what, STORAGE_DTYPE[storage], storage))


def afd_quantize(ctx: Context, cube: torch.Tensor, out: torch.Tensor, storage: str,
                 scale: float) -> torch.Tensor:
    """float32 CUDA tensor -> 2-byte storage tensor (float16, bfloat16 or
    int16 counts of scale/1024), on the current stream."""
    if cube.dtype != torch.float32 or not cube.is_cuda or not cube.is_contiguous():
        raise ValueError("afd_quantize takes a contiguous float32 CUDA tensor")
    _storage_tensor(out, storage, "afd_quantize")
    if out.numel() != cube.numel():
        raise ValueError("sizes differ")
    _use_current_stream(ctx, cube)
    _check(_lib.afd_quantize(ctx.handle, ctypes.c_void_p(cube.data_ptr()),
                             ctypes.c_void_p(out.data_ptr()), cube.numel(), STORAGE[storage],
                             float(scale)), "afd_quantize", ctx)
    return out


def afd_dequantize(ctx: Context, q: torch.Tensor, out: torch.Tensor, storage: str,
                   scale: float) -> torch.Tensor:
    """2-byte storage tensor -> float32 CUDA tensor, on the current stream."""
    _storage_tensor(q, storage, "afd_dequantize")
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() != q.numel():
        raise ValueError("out must be a float32 CUDA tensor of the same size")
    _use_current_stream(ctx, q)
    _check(_lib.afd_dequantize(ctx.handle, ctypes.c_void_p(q.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), q.numel(), STORAGE[storage],
                               float(scale)), "afd_dequantize", ctx)
    return out


def afd_filter_ex(ctx: Context, cube_in: torch.Tensor, cube_out: torch.Tensor, storage: str,
                  scale: float, K: float, dt: float, n_iter: int, conductance: str = "rational",
                  spacing=None, t_block: int = 0) -> torch.Tensor:
    """Filter a cube stored as float32, float16, bfloat16 or int16 counts,
    T = t_block iterations per pass; K in value units."""
    _storage_tensor(cube_in, storage, "afd_filter_ex")
    _storage_tensor(cube_out, storage, "afd_filter_ex")
    if cube_in.shape != cube_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    _use_current_stream(ctx, cube_in)
    _check(_lib.afd_filter_ex(ctx.handle, p_in, p_out, STORAGE[storage], float(scale), nx, ny, nz,
                              _spacing(spacing), float(K), float(dt), int(n_iter),
                              COND[conductance], int(t_block)), "afd_filter_ex", ctx)
    return cube_out


class Batch:
    """A resident batch of cubes (afd_batch*).  `shapes` are (nz, ny, nx)."""

    def __init__(self, ctx: Context, shapes, storage: str = "f32", scale: float = 1.0):
        import numpy as _np
        self.ctx = ctx
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.storage = storage
        dims = _np.array([[s[2], s[1], s[0]] for s in self.shapes], dtype=_np.int64).ravel()
        h = ctypes.c_void_p()
        _check(_lib.afd_batch_create(ctx.handle, ctypes.byref(h), len(self.shapes),
                                     ctypes.c_void_p(dims.ctypes.data), STORAGE[storage],
                                     float(scale)), "afd_batch_create", ctx)
        self.handle = h

    def close(self):
        if self.handle:
            _lib.afd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afd_batch_create(ctx: Context, shapes, storage: str = "f32", scale: float = 1.0) -> Batch:
    return Batch(ctx, shapes, storage, scale)


def afd_batch_set(b: Batch, i: int, cube: torch.Tensor) -> None:
    """Copy cube i (CUDA or CPU tensor in the batch's storage dtype, shape
    (nz, ny, nx)) into the batch; asynchronous on the current stream."""
    if tuple(cube.shape) != b.shapes[i] or cube.dtype != STORAGE_DTYPE[b.storage]:
        raise ValueError("cube %d must have shape %s and dtype %s"
                         % (i, b.shapes[i], STORAGE_DTYPE[b.storage]))
    if not cube.is_contiguous():
        raise ValueError("cube must be contiguous")
    _use_current_stream(b.ctx, cube if cube.is_cuda else None)
    _check(_lib.afd_batch_set(b.handle, int(i), ctypes.c_void_p(cube.data_ptr())),
           "afd_batch_set", b.ctx)


def afd_batch_get(b: Batch, i: int, out: torch.Tensor) -> torch.Tensor:
    if tuple(out.shape) != b.shapes[i] or out.dtype != STORAGE_DTYPE[b.storage]:
        raise ValueError("out must have shape %s and dtype %s" % (b.shapes[i],
                                                                  STORAGE_DTYPE[b.storage]))
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    _use_current_stream(b.ctx, out if out.is_cuda else None)
    _check(_lib.afd_batch_get(b.handle, int(i), ctypes.c_void_p(out.data_ptr())),
           "afd_batch_get", b.ctx)
    return out


def afd_batch_filter(b: Batch, K, dt: float, n_iter: int, conductance: str = "rational",
                     spacing=None) -> None:
    """K: sequence of per-cube K (> 0: value units; < 0: -K times the cube's
    noise rms, measured on the GPU)."""
    import numpy as _np
    k = _np.ascontiguousarray(_np.asarray(K, dtype=_np.float32).reshape(-1))
    if k.size != len(b.shapes):
        raise ValueError("need one K per cube")
    _use_current_stream(b.ctx)
    _check(_lib.afd_batch_filter(b.handle, ctypes.c_void_p(k.ctypes.data), _spacing(spacing),
                                 float(dt), int(n_iter), COND[conductance]),
           "afd_batch_filter", b.ctx)


def afd_batch_k(b: Batch):
    import numpy as _np
    out = _np.zeros(len(b.shapes), dtype=_np.float32)
    _use_current_stream(b.ctx)
    _check(_lib.afd_batch_k(b.handle, ctypes.c_void_p(out.ctypes.data)), "afd_batch_k", b.ctx)
    return out


def afd_batch_set_zchunk(b: Batch, zc: int) -> None:
    _use_current_stream(b.ctx)
    _check(_lib.afd_batch_set_zchunk(b.handle, int(zc)), "afd_batch_set_zchunk", b.ctx)


TILES = {"64x32": 0, "wide": 1}


def afd_batch_set_tiles(b: Batch, kind: str) -> None:
    """Tile kind of the batch's passes: '64x32' (4 x 2 voxels per thread) or
    'wide' (per-cube tiles of 8 x 2 voxels per thread, the default)."""
    _use_current_stream(b.ctx)
    _check(_lib.afd_batch_set_tiles(b.handle, TILES[kind]), "afd_batch_set_tiles", b.ctx)


def afd_batch_destroy(b: Batch) -> None:
    b.close()


class Server:
    """An interactive re-filter service over a resident Batch (afd_serve*)."""

    def __init__(self, batch: Batch, mem_bytes: int, max_active: int = 64):
        self.batch = batch
        h = ctypes.c_void_p()
        _check(_lib.afd_serve_create(batch.ctx.handle, batch.handle, int(mem_bytes),
                                     int(max_active), ctypes.byref(h)), "afd_serve_create",
               batch.ctx)
        self.handle = h

    def close(self):
        if self.handle:
            _lib.afd_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afd_serve_create(batch: Batch, mem_bytes: int, max_active: int = 64) -> Server:
    return Server(batch, mem_bytes, max_active)


def afd_serve_submit(srv: Server, cube: int, K: float, dt: float, n_iter: int,
                     conductance: str = "rational") -> int:
    t = ctypes.c_uint64()
    _check(_lib.afd_serve_submit(srv.handle, int(cube), float(K), float(dt), int(n_iter),
                                 COND[conductance], ctypes.byref(t)), "afd_serve_submit",
           srv.batch.ctx)
    return t.value


def afd_serve_step(srv: Server, wait: bool = False):
    """Advance the service; returns (active, queued)."""
    a, q = ctypes.c_int(), ctypes.c_int()
    _use_current_stream(srv.batch.ctx)
    _check(_lib.afd_serve_step(srv.handle, int(bool(wait)), ctypes.byref(a), ctypes.byref(q)),
           "afd_serve_step", srv.batch.ctx)
    return a.value, q.value


def afd_serve_poll(srv: Server, ticket: int):
    """(state, latency seconds): state 0 queued, 1 running, 2 done."""
    st, lat = ctypes.c_int(), ctypes.c_double()
    _check(_lib.afd_serve_poll(srv.handle, int(ticket), ctypes.byref(st), ctypes.byref(lat)),
           "afd_serve_poll", srv.batch.ctx)
    return st.value, lat.value


def afd_serve_times(srv: Server, ticket: int):
    """(submitted, admitted, first round launched, done) host timestamps in
    seconds (-1 for a stage not reached yet)."""
    out = (ctypes.c_double * 4)()
    _check(_lib.afd_serve_times(srv.handle, int(ticket), out), "afd_serve_times",
           srv.batch.ctx)
    return tuple(out)


def afd_serve_result(srv: Server, ticket: int, out: torch.Tensor) -> torch.Tensor:
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    _use_current_stream(srv.batch.ctx, out if out.is_cuda else None)
    _check(_lib.afd_serve_result(srv.handle, int(ticket), ctypes.c_void_p(out.data_ptr())),
           "afd_serve_result", srv.batch.ctx)
    return out


def afd_serve_release(srv: Server, ticket: int) -> None:
    _check(_lib.afd_serve_release(srv.handle, int(ticket)), "afd_serve_release", srv.batch.ctx)


def afd_serve_free_bytes(srv: Server) -> int:
    out = ctypes.c_size_t()
    _check(_lib.afd_serve_free_bytes(srv.handle, ctypes.byref(out)), "afd_serve_free_bytes",
           srv.batch.ctx)
    return out.value


def afd_serve_destroy(srv: Server) -> None:
    srv.close()


NOALLOC_MAX_VOXELS = 8388608


def afd_filter_noalloc(cube_in: torch.Tensor, cube_out: torch.Tensor, K: float, dt: float,
                       n_iter: int, conductance: str = "rational", spacing=None) -> torch.Tensor:
    """Filter without any GPU allocation, for callers that may not allocate
    (no context needed; the library's fixed 32 MiB device scratch is used).

    Runs on the current torch stream of the tensors' device and returns when
    the result is in ``cube_out``.  Cubes above NOALLOC_MAX_VOXELS voxels are
    rejected with AFD_EINVAL.  Calls that overlap on the GPU share the scratch
    and must not run concurrently.
    """
    for t in (cube_in, cube_out):
        if t.dtype != torch.float32 or not t.is_cuda:
            raise ValueError("afd_filter_noalloc takes float32 CUDA tensors")
    if cube_in.shape != cube_out.shape:
        raise ValueError("input and output shapes differ")
    p_in, nx, ny, nz = _cube_args(cube_in)
    p_out, _, _, _ = _cube_args(cube_out)
    with torch.cuda.device(cube_in.device):
        s = torch.cuda.current_stream(cube_in.device).cuda_stream
        status = _lib.afd_filter_noalloc(p_in, p_out, nx, ny, nz, _spacing(spacing), float(K),
                                         float(dt), int(n_iter), COND[conductance],
                                         ctypes.c_void_p(s))
    _check(status, "afd_filter_noalloc", None)
    return cube_out


def afd_selftest_wait(ctx: Context, limit_ns: int) -> None:
    """Launch the bounded-wait diagnostic; the next afd_sync must raise
    AfdError with status AFD_ETIMEOUT."""
    _use_current_stream(ctx)
    _check(_lib.afd_selftest_wait(ctx.handle, int(limit_ns)), "afd_selftest_wait", ctx)


def afd_stats(ctx: Context, cube: torch.Tensor, out4: torch.Tensor) -> torch.Tensor:
    """Asynchronous FP64 stats into a 4-element float64 CUDA tensor:
    sum, sum of squares, negative-half sum of squares, negative count."""
    if out4.dtype != torch.float64 or not out4.is_cuda or out4.numel() < 4:
        raise ValueError("out4 must be a float64 CUDA tensor of 4 elements")
    if cube.dtype != torch.float32 or not cube.is_cuda or not cube.is_contiguous():
        raise ValueError("afd_stats takes a contiguous float32 CUDA tensor")
    _use_current_stream(ctx, cube)
    _check(_lib.afd_stats(ctx.handle, ctypes.c_void_p(cube.data_ptr()), cube.numel(),
                          ctypes.c_void_p(out4.data_ptr())), "afd_stats", ctx)
    return out4


def afd_noise_rms(ctx: Context, cube: torch.Tensor) -> float:
    if cube.dtype != torch.float32 or not cube.is_cuda or not cube.is_contiguous():
        raise ValueError("afd_noise_rms takes a contiguous float32 CUDA tensor")
    _use_current_stream(ctx, cube)
    out = ctypes.c_double()
    _check(_lib.afd_noise_rms(ctx.handle, ctypes.c_void_p(cube.data_ptr()), cube.numel(),
                              ctypes.byref(out)), "afd_noise_rms", ctx)
    return out.value


def afd_sum(ctx: Context, cube: torch.Tensor) -> float:
    if cube.dtype != torch.float32 or not cube.is_cuda or not cube.is_contiguous():
        raise ValueError("afd_sum takes a contiguous float32 CUDA tensor")
    _use_current_stream(ctx, cube)
    out = ctypes.c_double()
    _check(_lib.afd_sum(ctx.handle, ctypes.c_void_p(cube.data_ptr()), cube.numel(),
                        ctypes.byref(out)), "afd_sum", ctx)
    return out.value


def afd_sync(ctx: Context) -> None:
    _check(_lib.afd_sync(ctx.handle), "afd_sync", ctx)


def afd_launch_count(ctx: Context) -> int:
    out = ctypes.c_uint64()
    _check(_lib.afd_launch_count(ctx.handle, ctypes.byref(out)), "afd_launch_count", ctx)
    return out.value


def afd_status_str(status: int) -> str:
    return _lib.afd_status_str(int(status)).decode()
