"""GPU parity of the box and Gaussian smoothing filters (Sec. 3.1, 3.2)
against the FP64 oracle (a normalised correlation written as plain loops,
pinned to scipy.ndimage).

Error bound per voxel: the kernels accumulate in float32, the separable one
in three chained sums (x, y, z) of 2r+1 terms each and the direct one in one
chain over all taps, then divide by the in-cube weight.  A chain of m
products and sums with u = 2^-24 errs by at most about (m + 2) u times the
weighted sum of |terms|, so |gpu - oracle| <= (m + 8) u smooth(|I|) with m
the taps summed in sequence.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def gpu_box(afd, ctx, cube, N):
    d = torch.from_numpy(np.ascontiguousarray(cube)).cuda()
    o = torch.full_like(d, float("nan"))
    afd.afd_smooth_box(ctx, d, o, N)
    afd.afd_sync(ctx)
    return o.cpu().numpy()


def gpu_gauss(afd, ctx, cube, fwhm, angles=None):
    d = torch.from_numpy(np.ascontiguousarray(cube)).cuda()
    o = torch.full_like(d, float("nan"))
    afd.afd_smooth_gauss(ctx, d, o, fwhm, angles)
    afd.afd_sync(ctx)
    return o.cpu().numpy()


def assert_close(got, cube, w, chain_taps):
    ref = oracle.smooth(cube, w)
    bound = (chain_taps + 8) * U * oracle.smooth(np.abs(cube), w) + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    assert np.isfinite(got).all()
    assert (err <= bound).all(), (float(err.max()), float((err / bound).max()))


SHAPES = [(1, 1, 1), (3, 2, 5), (7, 9, 13), (20, 17, 70), (33, 40, 129)]


@pytest.mark.parametrize("shape", SHAPES)
# (21, 3, 1): rx = 10, a 12-column x halo (two rounds of halo tasks for the
# loader warp); (49, 1, 1): rx = 24, the largest; (1, 1, 25): rz = 12, the
# largest z window (shared-memory ring)
@pytest.mark.parametrize("N", [(1, 1, 1), (3, 3, 1), (5, 3, 3), (3, 5, 7), (9, 1, 1),
                               (1, 1, 13), (21, 3, 1), (49, 1, 1), (1, 1, 25)])
def test_box_matches_oracle(afd, ctx, shape, N):
    rng = np.random.default_rng(sum(shape) + sum(N))
    cube = (rng.standard_normal(shape) * 2.0 + 0.5).astype(np.float32)
    got = gpu_box(afd, ctx, cube, N)
    if N == (1, 1, 1):
        assert np.array_equal(got, cube)
    assert_close(got, cube, oracle.box_weights(N), sum(N))


@pytest.mark.parametrize("shape", SHAPES[1:])
@pytest.mark.parametrize("fwhm", [(3.0, 3.0, 3.0), (5.0, 3.0, 1.0), (2.0, 2.0, 6.0),
                                  (1.5, 7.0, 2.5)])
def test_gauss_axis_aligned_matches_oracle(afd, ctx, shape, fwhm):
    rng = np.random.default_rng(sum(shape) + int(sum(fwhm) * 10))
    cube = rng.standard_normal(shape).astype(np.float32)
    w = oracle.gauss_weights(fwhm)
    got = gpu_gauss(afd, ctx, cube, fwhm)
    assert_close(got, cube, w, sum(w.shape))
    # zero angles take the same (separable) path
    assert np.array_equal(gpu_gauss(afd, ctx, cube, fwhm, (0.0, 0.0, 0.0)), got)


# (6, 6, 6) rotated has a 17^3 kernel: its ring of 32-row planes does not fit
# in shared memory and the 16-row direct kernel runs instead.
@pytest.mark.parametrize("shape", [(7, 9, 13), (20, 17, 70), (12, 30, 33), (9, 70, 140)])
@pytest.mark.parametrize("fwhm,angles", [((3.0, 5.0, 2.0), (20.0, 30.0, 40.0)),
                                         ((4.0, 2.0, 2.0), (0.0, 0.0, 35.0)),
                                         ((2.0, 2.0, 3.0), (60.0, -10.0, 0.0)),
                                         ((6.0, 6.0, 6.0), (10.0, 20.0, 30.0)),
                                         # x radius 1 (one 4-tap group), 12 and 13 (seven
                                         # groups, the last partial), 7
                                         ((0.7, 3.0, 2.0), (20.0, 0.0, 0.0)),
                                         ((9.0, 1.5, 1.5), (0.0, 0.0, 6.0)),
                                         ((9.5, 2.0, 1.2), (4.0, 3.0, 5.0)),
                                         ((5.0, 1.0, 1.0), (0.0, 0.0, 3.0))])
def test_gauss_rotated_matches_oracle(afd, ctx, shape, fwhm, angles):
    rng = np.random.default_rng(sum(shape) + int(sum(angles)))
    cube = rng.standard_normal(shape).astype(np.float32)
    w = oracle.gauss_weights(fwhm, angles)
    got = gpu_gauss(afd, ctx, cube, fwhm, angles)
    assert_close(got, cube, w, w.size)


@pytest.mark.parametrize("fwhm", [(3.0, 5.0, 2.0), (2.0, 2.0, 3.0)])
def test_gauss_rotated_nan_stays_in_window(afd, ctx, fwhm):
    # a blanked (NaN) voxel reaches exactly the voxels whose window holds it;
    # the x taps that pad a kernel row to a multiple of four take no part
    rng = np.random.default_rng(11)
    cube = rng.standard_normal((10, 40, 90)).astype(np.float32)
    for z, y, x in [(4, 20, 45), (0, 0, 0), (9, 39, 89), (5, 3, 70)]:
        cube[z, y, x] = np.nan
    angles = (25.0, 0.0, 40.0)
    w = oracle.gauss_weights(fwhm, angles)
    got = gpu_gauss(afd, ctx, cube, fwhm, angles)
    ref = oracle.smooth(cube, w)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    fin = ~np.isnan(ref)
    clean = np.where(np.isnan(cube), 0.0, cube)
    bound = (w.size + 8) * U * oracle.smooth(np.abs(clean), w) + 1e-30
    assert (np.abs(got[fin].astype(np.float64) - ref[fin]) <= bound[fin]).all()


@pytest.mark.parametrize("shape", [(9, 20, 64), (70, 33, 132), (5, 3, 4)])
def test_streamed_and_plain_paths_agree(afd, ctx, shape):
    # nx % 4 == 0 runs the TMA-streamed pass; a sliced (unaligned) view of
    # the same data runs the plain-load pass: the same floats either way
    rng = np.random.default_rng(sum(shape))
    cube = rng.standard_normal(shape).astype(np.float32)
    d = torch.from_numpy(cube).cuda()
    big = torch.zeros(cube.size + 1, device="cuda")
    big[1:] = d.reshape(-1)
    shifted = big[1:].view(shape)                      # 4-byte offset: not 16-byte aligned
    for fn, arg in ((afd.afd_smooth_box, (3, 5, 3)), (afd.afd_smooth_gauss, (3.0, 2.0, 4.0))):
        a = torch.empty_like(d)
        fn(ctx, d, a, arg)
        b = torch.empty_like(d)
        fn(ctx, shifted, b, arg)
        afd.afd_sync(ctx)
        assert torch.equal(a, b)


def test_constants_and_errors(afd, ctx):
    k = np.full((9, 10, 11), 1.75, dtype=np.float32)
    for got in (gpu_box(afd, ctx, k, (5, 3, 3)), gpu_gauss(afd, ctx, k, (3.0, 4.0, 2.0)),
                gpu_gauss(afd, ctx, k, (3.0, 4.0, 2.0), (10.0, 20.0, 30.0))):
        assert np.abs(got - 1.75).max() <= 4 * U * 1.75 * 64
    d = torch.zeros((4, 5, 6), device="cuda")
    o = torch.zeros_like(d)
    for bad in [(2, 1, 1), (1, 1, 0), (51, 1, 1), (1, 1, 27)]:
        with pytest.raises(afd.AfdError):
            afd.afd_smooth_box(ctx, d, o, bad)
    with pytest.raises(afd.AfdError):
        afd.afd_smooth_box(ctx, d, d, (3, 3, 3))              # in place
    for fw in [(0.0, 1.0, 1.0), (1.0, float("nan"), 1.0), (30.0, 1.0, 1.0)]:
        with pytest.raises(afd.AfdError):
            afd.afd_smooth_gauss(ctx, d, o, fw)


def crop_check(got, cube, w, boxes, chain_taps):
    """Oracle on the box grown by the kernel radius: every voxel of the box
    sees its whole in-cube window, so its value is exact there."""
    rz, ry, rx = (s // 2 for s in w.shape)
    nz, ny, nx = cube.shape
    for (z0, z1), (y0, y1), (x0, x1) in boxes:
        a = (max(z0 - rz, 0), max(y0 - ry, 0), max(x0 - rx, 0))
        b = (min(z1 + rz, nz), min(y1 + ry, ny), min(x1 + rx, nx))
        sub = np.ascontiguousarray(cube[a[0]:b[0], a[1]:b[1], a[2]:b[2]])
        sl = (slice(z0 - a[0], z1 - a[0]), slice(y0 - a[1], y1 - a[1]),
              slice(x0 - a[2], x1 - a[2]))
        ref = oracle.smooth(sub, w)[sl]
        bound = (chain_taps + 8) * U * oracle.smooth(np.abs(sub), w)[sl] + 1e-30
        err = np.abs(got[z0:z1, y0:y1, x0:x1].astype(np.float64) - ref)
        assert (err <= bound).all(), (float(err.max()), (z0, y0, x0))


def test_full_size_cube512(afd, ctx):
    cube = synth.cube512()
    boxes = [((0, 6), (0, 8), (0, 12)), ((250, 256), (500, 512), (496, 512)),
             ((120, 130), (250, 262), (250, 266)), ((60, 64), (0, 512), (300, 304))]
    w = oracle.box_weights((5, 5, 3))
    crop_check(gpu_box(afd, ctx, cube, (5, 5, 3)), cube, w, boxes, 13)
    w = oracle.gauss_weights((3.0, 3.0, 3.0))
    crop_check(gpu_gauss(afd, ctx, cube, (3.0, 3.0, 3.0)), cube, w, boxes, sum(w.shape))
    w = oracle.gauss_weights((3.0, 5.0, 2.0), (20.0, 30.0, 40.0))
    crop_check(gpu_gauss(afd, ctx, cube, (3.0, 5.0, 2.0), (20.0, 30.0, 40.0)), cube, w,
               boxes[:2], w.size)
