"""Property-based checks of the oracle (hypothesis, CPU only): random tiny
cubes, K, dt, spacing and iteration counts against the exact rational
brute force written face by face (rational g), and invariants that hold for
any parameters (constants kept, sum conserved, n = 0 the identity).
Skipped where hypothesis is not installed."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_pins import frac_pm_facewise

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

dyadic = st.integers(-64, 64).map(lambda v: v / 16.0)        # exact in binary


@settings(max_examples=40, deadline=None)
@given(nz=st.integers(1, 3), ny=st.integers(1, 3), nx=st.integers(1, 4),
       seed=st.integers(0, 10 ** 6), K=st.sampled_from([0.25, 0.5, 1.0, 1.5, 3.0]),
       dt=st.sampled_from([1 / 16, 1 / 8, 0.1]), n=st.integers(0, 3),
       h=st.tuples(st.sampled_from([0.5, 1.0, 2.0]), st.sampled_from([0.5, 1.0, 2.0]),
                   st.sampled_from([0.5, 1.0, 2.0])))
def test_oracle_equals_exact_rational(nz, ny, nx, seed, K, dt, n, h):
    rng = np.random.default_rng(seed)
    cube = rng.integers(-64, 65, size=(nz, ny, nx)) / 16.0
    exact = frac_pm_facewise(cube.tolist(), K, dt, n, h)
    got = oracle.pm_filter(cube, K, dt, n, "rational", spacing=h)
    scale = max(1.0, float(np.abs(cube).max()))
    for (x, y, z), v in exact.items():
        assert abs(got[z, y, x] - float(v)) <= 1e-13 * scale


@settings(max_examples=40, deadline=None)
@given(nz=st.integers(1, 5), ny=st.integers(1, 5), nx=st.integers(1, 6),
       seed=st.integers(0, 10 ** 6), K=st.floats(0.1, 10.0), dt=st.floats(0.01, 0.16),
       n=st.integers(0, 6), cond=st.sampled_from(["rational", "exponential"]),
       c=dyadic)
def test_oracle_invariants(nz, ny, nx, seed, K, dt, n, cond, c):
    rng = np.random.default_rng(seed)
    cube = rng.standard_normal((nz, ny, nx))
    out = oracle.pm_filter(cube, K, dt, n, cond)
    # conservation of the sum (per-face fluxes cancel in pairs)
    assert abs(out.sum() - cube.sum()) <= 1e-12 * max(1.0, np.abs(cube).sum())
    # inside the stability bound dt * 12 <= 1 (unit spacing), no new extrema
    if dt * 12 <= 1.0:
        assert out.max() <= cube.max() + 1e-12 and out.min() >= cube.min() - 1e-12
    # a constant cube is kept exactly; n = 0 is the identity
    k = np.full((nz, ny, nx), c)
    assert np.array_equal(oracle.pm_filter(k, K, dt, n, cond), k)
    assert np.array_equal(oracle.pm_filter(cube, K, dt, 0, cond), cube)
