"""GPU parity for the paper's own intensity-driven filter (Sec. 3.3, the
update after eq. "conductivepara") against the FP64 oracle, whose pins are in
test_oracle_pins.py.  Tolerance: min(1e-5 n, 1e-4) sigma, as for the
per-face filter; all kernels bit-identical."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tol(n):
    return min(1e-5 * max(n, 1), 1e-4)


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def run(afd, ctx, cube, K, rms, tau, n, C, kernel="auto"):
    afd.afd_set_kernel(ctx, kernel)
    src = torch.from_numpy(np.ascontiguousarray(cube, dtype=np.float32)).cuda()
    out = torch.empty_like(src)
    afd.afd_filter_intensity(ctx, src, out, K, rms, tau, n, C)
    afd.afd_sync(ctx)
    afd.afd_set_kernel(ctx, "auto")
    return out.cpu().numpy()


def test_paper_defaults_cube64(afd, ctx):
    # K = 1.5, tau = 0.0325, n = 20, C = 5 (the paper's defaults)
    cube = synth.cube64()
    src = torch.from_numpy(cube).cuda()
    rms = afd.afd_noise_rms(ctx, src)
    ref = oracle.intensity_filter(cube, 1.5, rms, 0.0325, 20, (5.0, 5.0, 5.0))
    for kernel in ("simple", "stream"):
        got = run(afd, ctx, cube, 1.5, rms, 0.0325, 20, (5.0, 5.0, 5.0), kernel)
        assert np.abs(got - ref).max() <= tol(20), kernel
    # not conservative (the paper notes the flux scale is not kept)
    assert abs(float(ref.sum()) - float(cube.astype(np.float64).sum())) > 1.0


@pytest.mark.parametrize("shape", [(1, 1, 4), (5, 17, 33), (9, 35, 132), (37, 19, 68)])
def test_ragged_and_kernels_identical(afd, ctx, shape):
    rng = np.random.default_rng(sum(shape))
    cube = (rng.standard_normal(shape) * 2).astype(np.float32)
    C = (5.0, 2.0, 1.0)
    ref = oracle.intensity_filter(cube, 1.2, 1.0, 0.05, 7, C)
    a = run(afd, ctx, cube, 1.2, 1.0, 0.05, 7, C, "simple")
    assert np.abs(a - ref).max() <= tol(7)
    if shape[2] % 4 == 0:
        b = run(afd, ctx, cube, 1.2, 1.0, 0.05, 7, C, "stream")
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_heat_limit_and_identity(afd, ctx):
    cube = synth.cube64()[:20, :24, :32].copy()
    ref = oracle.intensity_filter(cube, math.inf, 1.0, 0.01, 6, (5.0, 2.0, 1.0))
    got = run(afd, ctx, cube, math.inf, 1.0, 0.01, 6, (5.0, 2.0, 1.0))
    assert np.abs(got - ref).max() <= tol(6)
    for K, rms, n in ((0.0, 1.0, 5), (1.5, 0.0, 5), (1.5, 1.0, 0)):
        assert np.array_equal(run(afd, ctx, cube, K, rms, 0.0325, n, (5, 5, 5)), cube)
    with pytest.raises(afd.AfdError):
        run(afd, ctx, cube, 1.5, 1.0, 0.0, 3, (5, 5, 5))
