"""Seeded synthetic H I cubes (inputs only: nothing here filters anything).

The paper's data cubes (model galaxies built from NGC 3359, NGC 4111, NGC 3379,
WEIN069, NGC 2841; Sec. 2) are not available, so these generators stand in for
them with the same structure: Gaussian noise of rms sigma, galaxies whose
signal-to-noise ratio is ~10 in the inner parts and ~1 in the outer parts
(abstract), and faint tails / filaments at SNR 0.5-1 (Sec. 1).

Every array is float32 shaped (nz, ny, nx): x fastest, z = velocity channel.

Recipe (all random draws from ``numpy.random.Generator(PCG64(seed))``):

* noise   i.i.d. N(0, sigma), sigma = 1.
* disk    inclined rotating exponential disk: surface brightness
          A exp(-R/h_d), h_d = 8 voxels, A = 10 sigma (SNR 1 at R ~ 18 vox);
          sky (x, y) rotated by the position angle and deprojected by the
          inclination to disk-plane radius R and azimuth theta;
          line-of-sight velocity v_sys + v_rot(R) sin(i) cos(theta) with
          v_rot = v_max (2/pi) arctan(R/2), v_max = nz/6 channels;
          Gaussian line profile of sigma_v = 2 channels.
* tail    Gaussian tube (sigma_t = 2 voxels) along a random cubic Bezier curve
          through (x, y, v), amplitude U(0.5, 1) sigma.

The named workloads:

=============  ==============================================================
``cube64``     64^3, one disk (inclination 60 deg), seed 0
``cube512``    512 x 512 x 256, 4 disks (20, 45, 70, 85 deg) + 1 tail, seed 0
``cube2048``   2048 x 2048 x 256, 60 disks + 10 tails, seed 0
``cutouts``    300 cutouts, nx, ny ~ U{32..256}, nz ~ U{32..128}, 1 disk each
``serving``    64 resident cubes: 21 x 128^3, 21 x 256^3, 22 x 512x512x128
``model_b``    104 x 104 x 64 (6.9e5 voxels, the size of the paper's model
               galaxies): one disk of peak SNR 32 + a faint tail (0.75 sigma),
               returned with its noiseless model and the tail's ROI box
=============  ==============================================================
"""
from __future__ import annotations

import math

import numpy as np

SIGMA = 1.0
H_D = 8.0          # disk exponential scale length (voxels)
SIGMA_V = 2.0      # line-profile dispersion (channels)
DISK_PEAK = 10.0   # central SNR
SIGMA_T = 2.0      # tail tube radius (voxels)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def noise(shape, rng: np.random.Generator, sigma: float = SIGMA) -> np.ndarray:
    """i.i.d. Gaussian noise, float32, drawn one z-plane block at a time."""
    out = np.empty(shape, dtype=np.float32)
    nz = shape[0]
    step = max(1, (1 << 24) // max(1, shape[1] * shape[2]))
    for z0 in range(0, nz, step):
        z1 = min(nz, z0 + step)
        out[z0:z1] = rng.standard_normal((z1 - z0,) + tuple(shape[1:]),
                                         dtype=np.float32)
    if sigma != 1.0:
        out *= np.float32(sigma)
    return out


def add_disk(cube: np.ndarray, xc: float, yc: float, incl_deg: float,
             pa_deg: float, v_sys: float, amp: float = DISK_PEAK,
             h_d: float = H_D, sigma_v: float = SIGMA_V,
             v_max: float | None = None) -> None:
    """Add one inclined rotating exponential disk to ``cube`` in place.

    Only the sky box where the surface brightness exceeds 1e-3 sigma is
    touched (R <= h_d ln(amp / 1e-3)).
    """
    nz, ny, nx = cube.shape
    if v_max is None:
        v_max = nz / 6.0
    r_max = h_d * math.log(max(amp, 1e-3) / 1e-3)
    x0, x1 = max(0, int(math.floor(xc - r_max))), min(nx, int(math.ceil(xc + r_max)) + 1)
    y0, y1 = max(0, int(math.floor(yc - r_max))), min(ny, int(math.ceil(yc + r_max)) + 1)
    if x0 >= x1 or y0 >= y1:
        return
    yy, xx = np.meshgrid(np.arange(y0, y1, dtype=np.float64),
                         np.arange(x0, x1, dtype=np.float64), indexing="ij")
    pa, inc = math.radians(pa_deg), math.radians(incl_deg)
    dx, dy = xx - xc, yy - yc
    X = dx * math.cos(pa) + dy * math.sin(pa)          # along the major axis
    Y = (-dx * math.sin(pa) + dy * math.cos(pa)) / max(math.cos(inc), 1e-3)
    R = np.hypot(X, Y)
    cos_t = np.where(R > 0, X / np.where(R > 0, R, 1.0), 0.0)
    v_rot = v_max * (2.0 / math.pi) * np.arctan(R / 2.0)
    v_los = v_sys + v_rot * math.sin(inc) * cos_t
    sb = amp * np.exp(-R / h_d)
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    prof = np.exp(-((z - v_los[None]) ** 2) / (2.0 * sigma_v ** 2))
    cube[:, y0:y1, x0:x1] += (sb[None] * prof).astype(np.float32)


def add_tail(cube: np.ndarray, ctrl: np.ndarray, amp: float,
             sigma_t: float = SIGMA_T) -> None:
    """Add a Gaussian tube of radius sigma_t along the cubic Bezier curve with
    control points ``ctrl`` (4 x 3, columns x, y, v) to ``cube`` in place.

    The curve is sampled every <= 0.25 voxel; the tube's value at a voxel is
    amp * exp(-r^2 / (2 sigma_t^2)) with r the distance to the nearest sample.
    """
    nz, ny, nx = cube.shape
    p = np.asarray(ctrl, dtype=np.float64)
    length = float(np.sum(np.linalg.norm(np.diff(p, axis=0), axis=1)))
    m = max(8, int(math.ceil(length / 0.25)) + 1)
    t = np.linspace(0.0, 1.0, m)[:, None]
    pts = ((1 - t) ** 3 * p[0] + 3 * (1 - t) ** 2 * t * p[1]
           + 3 * (1 - t) * t ** 2 * p[2] + t ** 3 * p[3])
    rad = int(math.ceil(3.5 * sigma_t))
    lo = np.floor(pts.min(axis=0)).astype(int) - rad
    hi = np.ceil(pts.max(axis=0)).astype(int) + rad + 1
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, [nx, ny, nz])
    if np.any(lo >= hi):
        return
    best = np.full((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), np.inf)
    ax = np.arange(-rad, rad + 1)
    for q in pts:
        c = np.round(q).astype(int)
        xs = c[0] + ax
        ys = c[1] + ax
        zs = c[2] + ax
        xs = xs[(xs >= lo[0]) & (xs < hi[0])]
        ys = ys[(ys >= lo[1]) & (ys < hi[1])]
        zs = zs[(zs >= lo[2]) & (zs < hi[2])]
        if xs.size == 0 or ys.size == 0 or zs.size == 0:
            continue
        r2 = ((zs[:, None, None] - q[2]) ** 2 + (ys[None, :, None] - q[1]) ** 2
              + (xs[None, None, :] - q[0]) ** 2)
        sl = (slice(zs[0] - lo[2], zs[-1] - lo[2] + 1),
              slice(ys[0] - lo[1], ys[-1] - lo[1] + 1),
              slice(xs[0] - lo[0], xs[-1] - lo[0] + 1))
        np.minimum(best[sl], r2, out=best[sl])
    val = amp * np.exp(-best / (2.0 * sigma_t ** 2))
    cube[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += val.astype(np.float32)


def _random_disks(cube, rng, count, incls=None):
    nz, ny, nx = cube.shape
    for k in range(count):
        inc = incls[k] if incls is not None else rng.uniform(15.0, 85.0)
        xc = rng.uniform(0.1 * nx, 0.9 * nx)
        yc = rng.uniform(0.1 * ny, 0.9 * ny)
        pa = rng.uniform(0.0, 180.0)
        v_sys = nz / 2.0 + rng.uniform(-0.15, 0.15) * nz
        add_disk(cube, xc, yc, inc, pa, v_sys)


def _random_tails(cube, rng, count):
    nz, ny, nx = cube.shape
    for _ in range(count):
        ctrl = np.stack([rng.uniform(0.05, 0.95, 4) * nx,
                         rng.uniform(0.05, 0.95, 4) * ny,
                         rng.uniform(0.2, 0.8, 4) * nz], axis=1)
        add_tail(cube, ctrl, rng.uniform(0.5, 1.0) * SIGMA)


def galaxy_cube(shape, seed: int, n_disks: int, n_tails: int,
                incls=None) -> np.ndarray:
    """Noise + n_disks random disks + n_tails random tails, float32."""
    rng = rng_for(seed)
    cube = noise(shape, rng)
    _random_disks(cube, rng, n_disks, incls)
    _random_tails(cube, rng, n_tails)
    return cube


def cube64(seed: int = 0) -> np.ndarray:
    """64^3 cube, one disk at inclination 60 deg near the centre."""
    rng = rng_for(seed)
    cube = noise((64, 64, 64), rng)
    add_disk(cube, 32.0 + rng.uniform(-2, 2), 32.0 + rng.uniform(-2, 2),
             60.0, rng.uniform(0.0, 180.0), 32.0)
    return cube


def cube512(seed: int = 0) -> np.ndarray:
    """512 x 512 x 256: four disks (20, 45, 70, 85 deg) and one faint tail."""
    return galaxy_cube((256, 512, 512), seed, 4, 1, incls=[20.0, 45.0, 70.0, 85.0])


def cube2048(seed: int = 0) -> np.ndarray:
    """2048 x 2048 x 256 (4 GiB float32): 60 disks and 10 faint tails."""
    return galaxy_cube((256, 2048, 2048), seed, 60, 10)


def cutout_shapes(seed: int = 0, count: int = 300):
    """(nz, ny, nx) of the uneven cutout batch: nx, ny ~ U{32..256},
    nz ~ U{32..128}."""
    rng = rng_for(seed)
    nx = rng.integers(32, 257, count)
    ny = rng.integers(32, 257, count)
    nz = rng.integers(32, 129, count)
    return [(int(c), int(b), int(a)) for a, b, c in zip(nx, ny, nz)]


def cutout(shape, seed: int) -> np.ndarray:
    """One galaxy cutout: noise plus one centred disk (SNR 10 inner, 1 outer)."""
    rng = rng_for(seed)
    cube = noise(shape, rng)
    nz, ny, nx = shape
    add_disk(cube, nx / 2.0 + rng.uniform(-2, 2), ny / 2.0 + rng.uniform(-2, 2),
             rng.uniform(15.0, 85.0), rng.uniform(0.0, 180.0), nz / 2.0)
    return cube


def cutouts(seed: int = 0, count: int = 300):
    """The uneven batch: list of float32 cubes."""
    return [cutout(s, seed * 100003 + 1 + k)
            for k, s in enumerate(cutout_shapes(seed, count))]


def serving_shapes():
    """Shapes of the 64 resident serving cubes."""
    return ([(128, 128, 128)] * 21 + [(256, 256, 256)] * 21
            + [(128, 512, 512)] * 22)


def serving_cube(k: int, seed: int = 0) -> np.ndarray:
    shape = serving_shapes()[k]
    return galaxy_cube(shape, seed * 1009 + 7 + k, max(1, shape[2] // 128), 1)


def noiseless_disk64() -> np.ndarray:
    """The noiseless model of ``cube64`` (same draws, no noise added)."""
    rng = rng_for(0)
    _ = rng.standard_normal((64, 64, 64), dtype=np.float32)
    cube = np.zeros((64, 64, 64), dtype=np.float32)
    add_disk(cube, 32.0 + rng.uniform(-2, 2), 32.0 + rng.uniform(-2, 2),
             60.0, rng.uniform(0.0, 180.0), 32.0)
    return cube


def model_b(seed: int = 0):
    """A stand-in for the paper's ModelB noise study (Sec. 5): the noiseless
    model (one disk, peak SNR 32, and a faint tail of amplitude 0.75 sigma),
    the same plus unit noise, and the ROI box (x0, x1, y0, y1, z0, z1) around
    the tail.  Returns (cube, model, roi); cube = noise + model in float32."""
    shape = (64, 104, 104)
    nz, ny, nx = shape
    rng = rng_for(seed)
    cube = noise(shape, rng)
    model = np.zeros(shape, dtype=np.float32)
    add_disk(model, 40.0, 52.0, 55.0, rng.uniform(0.0, 180.0), nz / 2.0, amp=32.0)
    ctrl = np.array([[62.0, 20.0, 20.0], [78.0, 40.0, 26.0], [88.0, 66.0, 34.0],
                     [92.0, 90.0, 40.0]])
    add_tail(model, ctrl, 0.75 * SIGMA)
    cube += model
    pad = int(math.ceil(3.5 * SIGMA_T))
    lo = np.maximum(np.floor(ctrl.min(axis=0)).astype(int) - pad, 0)
    hi = np.minimum(np.ceil(ctrl.max(axis=0)).astype(int) + pad + 1, [nx, ny, nz])
    roi = (int(lo[0]), int(hi[0]), int(lo[1]), int(hi[1]), int(lo[2]), int(hi[2]))
    return cube, model, roi



def sha256(cube: np.ndarray) -> str:
    """SHA-256 of a cube's bytes (C order), to identify a generated input."""
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(cube).tobytes()).hexdigest()
