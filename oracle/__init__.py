"""CPU oracle for the anisotropic-diffusion hot path (arXiv:1609.03782, Sec. 3.3).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the GPU library computes: double precision, single thread,
no blocking or fusion beyond what the paper's definitions state.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_1609_03782_gb300``) and never imports it; the library never imports
this package.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py``
against hand-worked values, closed forms, invariants or library routines.

Contents
--------
pm_filter            per-face Perona-Malik iteration (Sec. 3.3, eq. "perona" and
                     the gradient conductance printed after it), C code in
                     ``afd_oracle.c``
pm_filter_box        the same, evaluated for one sub-box only through the
                     domain of dependence of an explicit n-step stencil
intensity_filter     the paper's intensity-driven update (Sec. 3.3, eq. after
                     "conductivepara")
stats / noise_rms    FP64 sums and the negative-half noise estimate (K is set
                     in units of the noise level, Sec. 3.3)
quantize/dequantize  2-byte storage formats with a power-of-two per-cube scale
f_diagnostic         the smoothing-quality parameter F with its error sigma_F
                     (Sec. 4) and the recovered-signal fraction F_M (Sec. 5)
box_weights /        the box and (rotated) Gaussian kernels of Sec. 3.1 and
gauss_weights        3.2, and smooth, the normalised correlation with them
smooth
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afd_oracle.c")
_LIB = os.path.join(_HERE, "liborcafd.so")
_lock = threading.Lock()
_lib = None

COND_EXPONENTIAL = 0
COND_RATIONAL = 1
_COND = {"exponential": COND_EXPONENTIAL, "rational": COND_RATIONAL}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no FP contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Load an oracle shared object and declare its signatures."""
    lib = ctypes.CDLL(path)
    i64, dbl, c_int = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    vp = ctypes.c_void_p
    lib.orc_pm_filter.argtypes = [vp, i64, i64, i64, dbl, dbl, dbl,
                                  dbl, dbl, c_int, c_int]
    lib.orc_pm_filter.restype = c_int
    lib.orc_intensity_filter.argtypes = [vp, i64, i64, i64, dbl, dbl,
                                         dbl, dbl, dbl, dbl, c_int]
    lib.orc_intensity_filter.restype = c_int
    lib.orc_stats.argtypes = [vp, i64, vp]
    lib.orc_fdiag.argtypes = [vp, vp, vp, i64, i64, i64, vp, dbl, dbl, vp]
    lib.orc_fdiag.restype = ctypes.c_int
    lib.orc_smooth.argtypes = [vp, vp, i64, i64, i64, vp, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int]
    lib.orc_smooth.restype = ctypes.c_int
    lib.orc_stats.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _shape3(a: np.ndarray):
    if a.ndim != 3:
        raise ValueError("cube must be 3-D, shaped (nz, ny, nx)")
    nz, ny, nx = a.shape
    return nx, ny, nz


def pm_filter(cube, K: float, dt: float, n_iter: int,
              conductance: str = "rational", spacing=(1.0, 1.0, 1.0),
              lib=None) -> np.ndarray:
    """n_iter per-face Perona-Malik iterations in FP64; returns a new array.

    ``cube`` is shaped (nz, ny, nx) (x fastest); it is converted to float64.
    ``spacing`` is (hx, hy, hz).  K is in absolute intensity units.  ``lib``
    selects another build of ``afd_oracle.c`` (the mutation tests use it).
    """
    a = np.ascontiguousarray(cube, dtype=np.float64).copy()
    nx, ny, nz = _shape3(a)
    hx, hy, hz = (float(s) for s in spacing)
    rc = (lib or _load()).orc_pm_filter(a.ctypes.data, nx, ny, nz, hx, hy, hz,
                               float(K), float(dt), int(n_iter),
                               _COND[conductance])
    if rc != 0:
        raise ValueError("oracle pm_filter rejected its arguments")
    return a


def pm_filter_box(cube, box, K: float, dt: float, n_iter: int,
                  conductance: str = "rational",
                  spacing=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Oracle result for the sub-box ``box`` = ((z0,z1),(y0,y1),(x0,x1)) only.

    An explicit nearest-neighbour iteration moves information one voxel per
    step, so after n_iter steps a voxel depends only on voxels within n_iter
    of it along each axis.  The box is grown by n_iter on every side (clamped
    to the cube, where the true zero-flux faces then apply), filtered there,
    and the centre cut out.  Within the box the result is the full-cube
    oracle's, operation for operation.
    """
    (z0, z1), (y0, y1), (x0, x1) = box
    nz, ny, nx = cube.shape
    g = int(n_iter)
    gz0, gz1 = max(0, z0 - g), min(nz, z1 + g)
    gy0, gy1 = max(0, y0 - g), min(ny, y1 + g)
    gx0, gx1 = max(0, x0 - g), min(nx, x1 + g)
    sub = cube[gz0:gz1, gy0:gy1, gx0:gx1]
    out = pm_filter(sub, K, dt, n_iter, conductance, spacing)
    return out[z0 - gz0:z1 - gz0, y0 - gy0:y1 - gy0, x0 - gx0:x1 - gx0].copy()


def intensity_filter(cube, K: float, rms: float, tau: float, n_iter: int,
                     C=(5.0, 5.0, 5.0)) -> np.ndarray:
    """The paper's intensity-driven update in FP64 (Sec. 3.3); new array."""
    a = np.ascontiguousarray(cube, dtype=np.float64).copy()
    nx, ny, nz = _shape3(a)
    rc = _load().orc_intensity_filter(a.ctypes.data, nx, ny, nz,
                                      float(C[0]), float(C[1]), float(C[2]),
                                      float(K), float(rms), float(tau),
                                      int(n_iter))
    if rc != 0:
        raise ValueError("oracle intensity_filter rejected its arguments")
    return a


def stats(cube) -> dict:
    """FP64 sums of an FP32 cube: sum, sum of squares, negative half."""
    a = np.ascontiguousarray(cube, dtype=np.float32).reshape(-1)
    out = np.zeros(4, dtype=np.float64)
    _load().orc_stats(a.ctypes.data, a.size, out.ctypes.data)
    return {"sum": out[0], "sumsq": out[1], "negsumsq": out[2],
            "nneg": int(out[3]), "n": int(a.size)}


def noise_rms(cube) -> float:
    """Noise level: rms of the negative voxels, sqrt(sum_{I<0} I^2 / #{I<0}).

    The paper uses the noise level "rms" to set K (Sec. 3.3) and takes it as
    constant over the cube (Sec. 4) without stating the estimator.  Emission
    is positive and the noise symmetric, so the negative half measures the
    noise alone.  Returns 0.0 for a cube with no negative voxel.
    """
    s = stats(cube)
    return math.sqrt(s["negsumsq"] / s["nneg"]) if s["nneg"] else 0.0


def f_diagnostic(orig, filt, model=None, roi=None, rms_o=None, rms_f=None, nsig=3.0,
                 beam=1.0, lib=None) -> dict:
    """The paper's smoothing-quality diagnostic over a ROI box.

    F = |S_of| / |S_oo| (Sec. 4, eqs. "F_equa" and "Sequa"), with masks
    M_i = [I_i >= nsig * rms_i] (eq. "Mfequa", nsig = 3 in the paper) and the
    sums taken over the ORIGINAL intensities.  sigma_F propagates
    sigma_S_oi = sqrt(N_i) rms_i (Sec. 4), with N_i the number of independent
    voxels in mask i: the mask's voxel count divided by `beam`, the number of
    voxels per independent element (1 for uncorrelated noise).  With the
    noiseless model, F_M = |S_mf| / |S_m| (Sec. 5, eq. "sums_equa").
    rms_o / rms_f default to noise_rms of the full cubes (the paper assumes
    the rms constant over the cube).  roi = (x0, x1, y0, y1, z0, z1), None for
    the whole cube.
    """
    Io = np.ascontiguousarray(orig, dtype=np.float32)
    If = np.ascontiguousarray(filt, dtype=np.float32)
    if Io.shape != If.shape or Io.ndim != 3:
        raise ValueError("original and filtered cubes must be 3-D of one shape")
    nz, ny, nx = Io.shape
    Im = None if model is None else np.ascontiguousarray(model, dtype=np.float32)
    if Im is not None and Im.shape != Io.shape:
        raise ValueError("model cube shape differs")
    box = np.array(roi if roi is not None else (0, nx, 0, ny, 0, nz), dtype=np.int64)
    ro = noise_rms(Io) if rms_o is None else float(rms_o)
    rf = noise_rms(If) if rms_f is None else float(rms_f)
    out = np.zeros(6, dtype=np.float64)
    rc = (lib or _load()).orc_fdiag(Io.ctypes.data, If.ctypes.data,
                           None if Im is None else Im.ctypes.data, nx, ny, nz,
                           box.ctypes.data, nsig * ro, nsig * rf, out.ctypes.data)
    if rc != 0:
        raise ValueError("empty or out-of-range ROI")
    s_of, s_oo, s_mf, s_m, n_o, n_f = (float(v) for v in out)
    r = {"S_of": s_of, "S_oo": s_oo, "S_mf": s_mf, "S_m": s_m, "N_o": int(n_o),
         "N_f": int(n_f), "rms_o": ro, "rms_f": rf}
    r["F"] = abs(s_of) / abs(s_oo) if s_oo != 0.0 else math.nan
    sig_of = math.sqrt(n_f / beam) * rf
    sig_oo = math.sqrt(n_o / beam) * ro
    r["sigma_F"] = (math.sqrt(sig_of ** 2 / s_oo ** 2 + s_of ** 2 * sig_oo ** 2 / s_oo ** 4)
                    if s_oo != 0.0 else math.nan)
    r["F_M"] = (abs(s_mf) / abs(s_m) if (Im is not None and s_m != 0.0) else math.nan)
    return r


# --------------------------------------------------------------------------
# Box and Gaussian smoothing (Sec. 3.1, 3.2).  Weight arrays are (nz, ny, nx)
# shaped like the cubes: W[dz + rz, dy + ry, dx + rx].
# --------------------------------------------------------------------------
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))   # FWHM_i = 2 sqrt(2 ln 2) sigma_i


def box_weights(n) -> np.ndarray:
    """The box (mean) filter's kernel: N_x x N_y x N_z ones, sizes odd so the
    window is centred on the voxel (Sec. 3.1; Tab. 1 uses odd sizes)."""
    nx_, ny_, nz_ = (int(v) for v in n)
    if min(nx_, ny_, nz_) < 1 or not (nx_ % 2 and ny_ % 2 and nz_ % 2):
        raise ValueError("box sizes must be odd and positive")
    return np.ones((nz_, ny_, nx_), dtype=np.float64)


def rotation(angles_deg) -> np.ndarray:
    """R = R_z(theta_z) R_y(theta_y) R_x(theta_x), the Euler rotation of the
    Gaussian kernel (Sec. 3.2), angles in degrees, right-handed."""
    ax, ay, az = (math.radians(float(a)) for a in angles_deg)
    cx, sx, cy, sy, cz, sz = (math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay),
                              math.cos(az), math.sin(az))
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def gauss_weights(fwhm, angles_deg=(0.0, 0.0, 0.0), truncate: float = 3.0) -> np.ndarray:
    """The Gaussian kernel of Sec. 3.2: G = exp(-sum_i (x_i)^2 / (2 sigma_i^2))
    with sigma_i = FWHM_i / (2 sqrt(2 ln 2)), rotated by R (K(p) = G(R^T p)),
    sampled at integer offsets and truncated where the ellipsoid's extent
    along each axis passes truncate sigma: r_a = ceil(truncate sqrt(Sigma_aa)),
    Sigma = R diag(sigma^2) R^T.  Unnormalised (smooth() divides by the
    in-cube weight)."""
    sig = np.array([float(f) / FWHM_PER_SIGMA for f in fwhm])
    if np.any(sig <= 0.0):
        raise ValueError("FWHM must be positive")
    R = rotation(angles_deg)
    cov = R @ np.diag(sig ** 2) @ R.T
    r = [int(math.ceil(truncate * math.sqrt(cov[a, a]) - 1e-12)) for a in range(3)]
    dz, dy, dx = np.meshgrid(np.arange(-r[2], r[2] + 1), np.arange(-r[1], r[1] + 1),
                             np.arange(-r[0], r[0] + 1), indexing="ij")
    p = np.stack([dx, dy, dz], axis=-1).astype(np.float64)     # (x, y, z) offsets
    u = p @ R                                                  # R^T p, per offset
    return np.exp(-0.5 * np.sum((u / sig) ** 2, axis=-1))


def smooth(cube, weights, lib=None) -> np.ndarray:
    """Normalised correlation of the cube with the weight array (odd sizes):
    out(p) = sum W(q - p) I(q) / sum W(q - p) over the window inside the cube
    (float64 result)."""
    a = np.ascontiguousarray(cube, dtype=np.float32)
    nx, ny, nz = _shape3(a)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    wz, wy, wx = w.shape
    if not (wz % 2 and wy % 2 and wx % 2):
        raise ValueError("weight array sizes must be odd")
    out = np.empty((nz, ny, nx), dtype=np.float64)
    rc = (lib or _load()).orc_smooth(out.ctypes.data, a.ctypes.data, nx, ny, nz, w.ctypes.data,
                                     wx // 2, wy // 2, wz // 2)
    if rc != 0:
        raise ValueError("oracle smooth rejected its arguments")
    return out


# --------------------------------------------------------------------------
# 2-byte storage (precision line).  The per-cube scale s is a power of two, so
# I/s and q*s are exact; the only rounding is the one into the 2-byte format,
# round-to-nearest-even in every case.
# --------------------------------------------------------------------------
I16_FRAC_BITS = 10   # int16 fixed point: step = s / 2^10, range +-32 s
I16_MAX = 32767


def pow2_scale(sigma: float) -> float:
    """Per-cube scale: the power of two nearest the noise level (log2 rounded
    half up).  A non-positive or non-finite sigma gives 1."""
    if not (sigma > 0.0) or not math.isfinite(sigma):
        return 1.0
    return 2.0 ** math.floor(math.log2(sigma) + 0.5)


def _f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even) by its definition:
    keep the upper 16 bits, rounding on the lower 16; NaN stays NaN."""
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x32)
    r[nan] = ((b[nan] >> 16) | 0x40).astype(np.uint16)
    return r


def quantize(cube, storage: str, scale: float) -> np.ndarray:
    """q = RN(I / scale) in ``storage`` ('f16', 'bf16' or 'i16').

    f16/bf16 return the 2-byte pattern as uint16; i16 returns int16 counts of
    step = scale / 2^10, clamped to +-32767.
    """
    x = np.ascontiguousarray(cube, dtype=np.float32)
    inv = np.float32(1.0 / scale)
    if storage == "f16":
        with np.errstate(over="ignore"):   # out of range rounds to +-inf
            return (x * inv).astype(np.float16).view(np.uint16)
    if storage == "bf16":
        return _f32_to_bf16_bits((x * inv).astype(np.float32))
    if storage == "i16":
        step_inv = np.float32(2.0 ** I16_FRAC_BITS / scale)
        q = np.rint((x * step_inv).astype(np.float64))
        return np.clip(q, -I16_MAX, I16_MAX).astype(np.int16)
    raise ValueError("storage must be 'f16', 'bf16' or 'i16'")


def dequantize(q: np.ndarray, storage: str, scale: float) -> np.ndarray:
    """Inverse of quantize: float32 value = stored value * scale (exact)."""
    if storage == "f16":
        v = q.view(np.float16).astype(np.float32)
        return v * np.float32(scale)
    if storage == "bf16":
        v = (q.astype(np.uint32) << 16).view(np.float32)
        return v * np.float32(scale)
    if storage == "i16":
        return q.astype(np.float32) * np.float32(scale / 2.0 ** I16_FRAC_BITS)
    raise ValueError("storage must be 'f16', 'bf16' or 'i16'")
