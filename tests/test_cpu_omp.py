"""The multithreaded FP32 CPU build (cpu_omp), the host baseline of the
benchmark, against the FP64 oracle: the same method in float32, so within
the float32 tolerance of the GPU path (1e-5 sigma per iteration, at most
1e-4 sigma), on every thread count, bit-identical across thread counts."""
import math

import numpy as np
import pytest

import cpu_omp
import oracle
import synth


def tol(n):
    return min(1e-5 * max(n, 1), 1e-4)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_cube64_exponential(threads):
    c = synth.cube64()
    ref = oracle.pm_filter(c, 1.5, 1 / 16, 10, "exponential")
    got = cpu_omp.filter(c, 1.5, 1 / 16, 10, "exponential", threads=threads)
    assert np.abs(got - ref).max() <= tol(10)


@pytest.mark.parametrize("shape", [(7, 13, 11), (1, 9, 5), (20, 1, 1), (33, 17, 5)])
@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_ragged_anisotropic(shape, cond):
    rng = np.random.default_rng(3)
    c = rng.standard_normal(shape).astype(np.float32) * 2.0
    sp = (1.0, 1.5, 0.75)
    ref = oracle.pm_filter(c, 1.1, 0.1, 12, cond, spacing=sp)
    got1 = cpu_omp.filter(c, 1.1, 0.1, 12, cond, spacing=sp, threads=1)
    got5 = cpu_omp.filter(c, 1.1, 0.1, 12, cond, spacing=sp, threads=5)
    assert np.array_equal(got1, got5)          # thread split changes no rounding
    assert np.abs(got1 - ref).max() <= tol(12) * max(1.0, float(np.abs(c).max()) / 4)


def test_headline_subcube_50_iterations():
    c = synth.cube512()[:24, :64, :96].copy()
    K = float(np.float32(oracle.noise_rms(c)))
    ref = oracle.pm_filter(c, K, 1 / 8, 50, "rational")
    got = cpu_omp.filter(c, K, 1 / 8, 50, "rational")
    assert np.abs(got - ref).max() <= tol(50)
    # the voxel sum is conserved (zero-flux faces)
    assert abs(float(got.astype(np.float64).sum()) - float(c.astype(np.float64).sum())) <= \
        1e-6 * float(np.abs(c.astype(np.float64)).sum())


def test_identities_and_heat_limit():
    c = synth.cube64()[:16, :16, :16].copy()
    assert np.array_equal(cpu_omp.filter(c, 0.0, 0.1, 5), c)          # K = 0
    assert np.array_equal(cpu_omp.filter(c, 1.0, 0.1, 0), c)          # n = 0
    const = np.full((6, 7, 8), 3.25, np.float32)
    assert np.array_equal(cpu_omp.filter(const, 1.0, 0.1, 9), const)  # fixed point
    ref = oracle.pm_filter(c, math.inf, 0.1, 6, "rational")
    assert np.abs(cpu_omp.filter(c, math.inf, 0.1, 6) - ref).max() <= tol(6) * 10


def test_argument_errors():
    c = np.zeros((2, 2, 2), np.float32)
    with pytest.raises(ValueError):
        cpu_omp.filter(c, -1.0, 0.1, 1)
    with pytest.raises(ValueError):
        cpu_omp.filter(c, 1.0, 0.0, 1)
    with pytest.raises(ValueError):
        cpu_omp.filter(c, 1.0, 0.1, -1)
    with pytest.raises(ValueError):
        cpu_omp.filter_inplace(c.astype(np.float64), 1.0, 0.1, 1)


def test_stream_copy_and_threads():
    assert cpu_omp.max_threads() >= 1
    assert cpu_omp.stream_copy_gbs(1 << 24, 2) > 0.0
    assert isinstance(cpu_omp.cpu_model(), str)
