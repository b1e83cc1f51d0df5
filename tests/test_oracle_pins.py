"""Pins for the CPU oracle: every check here is fixed by the paper or by
mathematics, never by the oracle itself.

The filter is the per-face Perona-Malik iteration (arXiv:1609.03782, Sec. 3.3,
eq. "perona" with the gradient conductance printed after it):
    I'[p] = I[p] + dt * sum_faces g(d; K) d / h_a,   d = (I[q] - I[p]) / h_a,
zero flux through the cube's faces, synchronous update, exactly n steps.

Pins, and the mistakes each one catches:
  * hand-worked 4^3 impulse values (rational and exponential g, anisotropic
    spacing, iterations 1 and 2): wrong g, wrong dt or spacing factor,
    Gauss-Seidel instead of Jacobi, off-by-one iteration count;
  * exact rational brute force, written face-centrically (each face flux
    added to one voxel and subtracted from the other): index or stride
    mistakes, boundary handling, a dropped face;
  * K = +inf is the discrete heat equation, diagonalised by the DCT-II
    (scipy): wrong sign, wrong weights, wrong boundary;
  * invariants: constants fixed, sum conserved, maximum principle,
    translation, odd symmetry and power-of-two scale equivariance, axis
    flips and transposition, 1-D cubes along every axis agree, n = 0 and
    K = 0 are the identity, spacing equivalence.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth

try:
    import scipy.fft as sfft
except ImportError:  # pragma: no cover
    sfft = None


def impulse(n=4, at=(1, 1, 1), dtype=np.float64):
    c = np.zeros((n, n, n), dtype=dtype)
    x, y, z = at
    c[z, y, x] = 1.0
    return c


# ---------------------------------------------------------------- hand-worked
def test_p1_rational_impulse_two_iterations():
    # 4^3 zeros, I(1,1,1)=1, unit spacing, g = 1/(1+d^2) (K=1), dt = 1/8.
    # Iteration 1: centre: six faces with d=-1, g=1/2 -> acc=-3 -> 1-3/8 = 5/8;
    # each face neighbour: one face with d=+1 -> 1/8 * 1/2 = 1/16.
    r1 = oracle.pm_filter(impulse(), 1.0, 0.125, 1, "rational")
    assert r1[1, 1, 1] == 5 / 8
    for (x, y, z) in [(0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)]:
        assert r1[z, y, x] == 1 / 16
    assert np.count_nonzero(r1) == 7
    # Iteration 2 (worked with fractions by hand):
    #  centre: d = 1/16-5/8 = -9/16, g = 256/337, g d = -144/337, six of them,
    #          5/8 - (1/8)(864/337) = 821/2696;
    #  (0,1,1): +144/337 from the centre, four zero neighbours with
    #          d=-1/16, g=256/257, g d=-16/257: 1/16 + 18/337 - 8/257
    #          = 117489/1385744;
    #  (2,1,1): one more zero neighbour: 1/16 + 18/337 - 10/257 = 106705/1385744;
    #  (2,2,1), (0,0,1): two neighbours at 1/16 -> (1/8)(32/257) = 4/257;
    #  (3,1,1): one neighbour at 1/16 -> 2/257.
    r2 = oracle.pm_filter(impulse(), 1.0, 0.125, 2, "rational")
    exp = {(1, 1, 1): Fr(821, 2696), (0, 1, 1): Fr(117489, 1385744),
           (2, 1, 1): Fr(106705, 1385744), (2, 2, 1): Fr(4, 257),
           (0, 0, 1): Fr(4, 257), (3, 1, 1): Fr(2, 257)}
    for (x, y, z), v in exp.items():
        assert r2[z, y, x] == pytest.approx(float(v), rel=1e-15, abs=0)
    assert math.fsum(r2.ravel()) == pytest.approx(1.0, abs=1e-15)


def test_p1_exponential_impulse():
    # g = exp(-d^2): centre 1 - (6/8) e^-1, each neighbour (1/8) e^-1.
    r = oracle.pm_filter(impulse(), 1.0, 0.125, 1, "exponential")
    assert r[1, 1, 1] == pytest.approx(1 - 0.75 * math.exp(-1), rel=1e-15)
    assert r[1, 1, 2] == pytest.approx(0.125 * math.exp(-1), rel=1e-15)
    assert r[1, 1, 0] == pytest.approx(0.125 * math.exp(-1), rel=1e-15)


def test_p1_corner_impulse():
    # Corner (0,0,0): three faces only; 1 - (3/8)(1/2) = 13/16; neighbours 1/16.
    r = oracle.pm_filter(impulse(at=(0, 0, 0)), 1.0, 0.125, 1, "rational")
    assert r[0, 0, 0] == 0.8125
    assert r[0, 0, 1] == r[0, 1, 0] == r[1, 0, 0] == 0.0625
    assert np.count_nonzero(r) == 4


def test_p1_anisotropic_spacing():
    # hx = 2: x faces have d = -1/2, g = 1/(1+1/4) = 4/5, flux g d/h = -1/5;
    # y, z faces flux -1/2 each; acc = -2/5 - 2 = -12/5 -> 1 - 3/10 = 7/10;
    # x neighbour (1/8)(1/5) = 1/40, y/z neighbour (1/8)(1/2) = 1/16.
    r = oracle.pm_filter(impulse(), 1.0, 0.125, 1, "rational", spacing=(2.0, 1.0, 1.0))
    assert r[1, 1, 1] == pytest.approx(0.7, rel=1e-15)
    assert r[1, 1, 0 + 2] == pytest.approx(1 / 40, rel=1e-15)
    assert r[1, 1, 0] == pytest.approx(1 / 40, rel=1e-15)
    assert r[1, 2, 1] == pytest.approx(1 / 16, rel=1e-15)
    assert r[2, 1, 1] == pytest.approx(1 / 16, rel=1e-15)


# ------------------------------------------------------- exact brute force
def frac_pm_facewise(cube, K, dt, n_iter, h=(1, 1, 1)):
    """Exact rational PM, rational g, written face by face: every interior
    face between p and q = p + e_a carries F = g(d) d / h_a with
    d = (I[q]-I[p])/h_a, added to p and subtracted from q."""
    nz, ny, nx = len(cube), len(cube[0]), len(cube[0][0])
    I = {(x, y, z): Fr(cube[z][y][x]) for z in range(nz) for y in range(ny) for x in range(nx)}
    K = Fr(K)
    dims = (nx, ny, nz)
    for _ in range(n_iter):
        delta = {p: Fr(0) for p in I}
        for a in range(3):
            ha = Fr(h[a])
            for p in I:
                if p[a] + 1 >= dims[a]:
                    continue
                q = list(p)
                q[a] += 1
                q = tuple(q)
                d = (I[q] - I[p]) / ha
                g = Fr(0) if K == 0 else 1 / (1 + (d / K) ** 2)
                F = g * d / ha
                delta[p] += F
                delta[q] -= F
        I = {p: I[p] + Fr(dt) * delta[p] for p in I}
    return I


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (1, 2, 3), (3, 2, 1), (2, 3, 5), (4, 4, 4)])
def test_p2_exact_rational_bruteforce(shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape))
    # dyadic inputs so that the float64 cube holds them exactly
    vals = rng.integers(-64, 65, size=shape) / 16.0
    h = (1.0, 0.5, 2.0)
    exact = frac_pm_facewise(vals.tolist(), 1.5, 0.0625, 3, h)
    got = oracle.pm_filter(vals, 1.5, 0.0625, 3, "rational", spacing=h)
    scale = max(1.0, np.abs(vals).max())
    for (x, y, z), v in exact.items():
        assert abs(got[z, y, x] - float(v)) <= 1e-14 * scale


# ------------------------------------------------ heat equation, closed form
def heat_closed_form(I0, dt, n, h):
    """K = +inf: I_n = IDCT( DCT(I0) * (1 - sum_a 4 dt/h_a^2 sin^2(pi k_a/(2 n_a)))^n ).
    Zero-flux (mirror) boundaries are diagonalised by the type-II DCT."""
    nz, ny, nx = I0.shape
    lam = np.zeros(I0.shape)
    for axis, (na, ha) in zip((2, 1, 0), ((nx, h[0]), (ny, h[1]), (nz, h[2]))):
        k = np.arange(na)
        s = 4.0 * dt / ha ** 2 * np.sin(np.pi * k / (2 * na)) ** 2
        shape = [1, 1, 1]
        shape[axis] = na
        lam = lam + s.reshape(shape)
    c = sfft.dctn(I0, type=2, norm="ortho")
    return sfft.idctn(c * (1.0 - lam) ** n, type=2, norm="ortho")


@pytest.mark.skipif(sfft is None, reason="scipy missing")
@pytest.mark.parametrize("cond", ["rational", "exponential"])
@pytest.mark.parametrize("shape,h,dt,n", [((7, 5, 6), (1, 1, 1), 1 / 8, 9),
                                          ((3, 9, 4), (0.5, 1.0, 2.0), 1 / 64, 5),
                                          ((1, 1, 17), (1, 1, 1), 0.25, 12)])
def test_p3_heat_equation_limit(cond, shape, h, dt, n):
    rng = np.random.default_rng(3)
    I0 = rng.standard_normal(shape)
    got = oracle.pm_filter(I0, math.inf, dt, n, cond, spacing=h)
    ref = heat_closed_form(I0, dt, n, h)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(I0).max()


# ------------------------------------------------------------- invariants
def rand_cube(shape=(6, 7, 5), seed=1):
    return np.random.default_rng(seed).standard_normal(shape) * 2.0


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i1_constant_fixed_point(cond):
    c = np.full((5, 6, 7), 3.25)
    assert np.array_equal(oracle.pm_filter(c, 1.0, 0.125, 7, cond), c)


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i2_sum_conserved(cond):
    c = synth.cube64()
    r = oracle.pm_filter(c[:20, :24, :28], 1.5, 1 / 16, 10, cond)
    s0 = math.fsum(c[:20, :24, :28].astype(np.float64).ravel())
    s1 = math.fsum(r.ravel())
    assert abs(s1 - s0) <= 1e-13 * np.abs(c[:20, :24, :28]).sum()


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i3_max_principle(cond):
    c = rand_cube((9, 8, 7))
    h = (1.0, 2.0, 0.5)
    dt = 1.0 / sum(2.0 / x ** 2 for x in h)        # dt * sum 2/h^2 = 1
    r = oracle.pm_filter(c, 0.7, dt, 20, cond, spacing=h)
    assert r.max() <= c.max() + 1e-12 and r.min() >= c.min() - 1e-12
    # and the bound is sharp in the other direction: beyond it the impulse
    # overshoots below zero for the heat limit
    r = oracle.pm_filter(impulse(), math.inf, 0.25, 1, cond)
    assert r.min() < 0


def test_i4_k_zero_identity():
    c = rand_cube()
    for cond in ("rational", "exponential"):
        assert np.array_equal(oracle.pm_filter(c, 0.0, 0.125, 5, cond), c)


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i5_translation(cond):
    c = rand_cube()
    a = oracle.pm_filter(c + 5.0, 1.0, 0.125, 6, cond)
    b = oracle.pm_filter(c, 1.0, 0.125, 6, cond) + 5.0
    assert np.abs(a - b).max() <= 1e-12


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i6_odd_and_scale(cond):
    c = rand_cube()
    f = oracle.pm_filter(c, 1.3, 0.1, 6, cond)
    assert np.array_equal(oracle.pm_filter(-c, 1.3, 0.1, 6, cond), -f)
    assert np.array_equal(oracle.pm_filter(c * 8.0, 1.3 * 8.0, 0.1, 6, cond), f * 8.0)


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i7_flips_and_transpose(cond):
    c = rand_cube((5, 6, 6))
    f = oracle.pm_filter(c, 1.1, 0.1, 5, cond)
    for ax in range(3):
        g = oracle.pm_filter(np.flip(c, ax), 1.1, 0.1, 5, cond)
        assert np.abs(np.flip(g, ax) - f).max() <= 1e-13
    g = oracle.pm_filter(np.transpose(c, (0, 2, 1)), 1.1, 0.1, 5, cond)
    assert np.abs(np.transpose(g, (0, 2, 1)) - f).max() <= 1e-13


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_i8_degenerate(cond):
    c = rand_cube()
    assert np.array_equal(oracle.pm_filter(c, 1.0, 0.1, 0, cond), c)
    one = np.full((1, 1, 1), 2.5)
    assert np.array_equal(oracle.pm_filter(one, 1.0, 0.1, 9, cond), one)
    # a 1-D line gives the same numbers along each axis
    line = np.random.default_rng(5).standard_normal(11)
    rx = oracle.pm_filter(line.reshape(1, 1, 11), 0.8, 0.2, 7, cond).ravel()
    ry = oracle.pm_filter(line.reshape(1, 11, 1), 0.8, 0.2, 7, cond).ravel()
    rz = oracle.pm_filter(line.reshape(11, 1, 1), 0.8, 0.2, 7, cond).ravel()
    assert np.array_equal(rx, ry) and np.array_equal(rx, rz)


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_spacing_equivalence(cond):
    # isotropic spacing h: d/h/K = d/(K h) and the flux carries dt/h^2, so
    # f(I; h, K, dt) = f(I; 1, K h, dt / h^2)
    c = rand_cube()
    a = oracle.pm_filter(c, 1.2, 0.5, 5, cond, spacing=(2.0, 2.0, 2.0))
    b = oracle.pm_filter(c, 2.4, 0.125, 5, cond)
    assert np.abs(a - b).max() <= 1e-13


def test_box_matches_full_cube():
    c = synth.cube64()[:30, :40, :36]
    full = oracle.pm_filter(c, 1.5, 1 / 16, 6, "exponential")
    for box in [((0, 5), (0, 7), (0, 9)), ((10, 20), (12, 30), (5, 36)), ((25, 30), (33, 40), (30, 36))]:
        sub = oracle.pm_filter_box(c, box, 1.5, 1 / 16, 6, "exponential")
        (z0, z1), (y0, y1), (x0, x1) = box
        assert np.array_equal(sub, full[z0:z1, y0:y1, x0:x1])


# ------------------------------------------------------- intensity form
def test_intensity_form_pins():
    # constant cube: every second difference is zero
    c = np.full((4, 5, 6), 1.75)
    assert np.array_equal(oracle.intensity_filter(c, 1.5, 1.0, 0.0325, 5), c)
    # hand-worked: impulse at the centre of 4^3, C = 5, tau = 1/32, K=1, rms=1:
    # centre Dx=Dy=Dz=-2, lap = 5*(-6) = -30, S = 1/(1+1) = 1/2:
    # 1 + (1/32)(-30)(1/2) = 17/32; a neighbour: lap = 5 * 1, S = 1 -> 5/32.
    r = oracle.intensity_filter(impulse(), 1.0, 1.0, 1 / 32, 1, C=(5, 5, 5))
    assert r[1, 1, 1] == 17 / 32 and r[1, 1, 2] == 5 / 32
    # not conservative (the conductance is per voxel, Sec. 3.3): 17/32 + 30/32 != 1
    assert abs(r.sum() - 1.0) > 0.1
    # K -> inf: the heat equation with weights tau*C_a
    rng = np.random.default_rng(9)
    I0 = rng.standard_normal((5, 6, 7))
    got = oracle.intensity_filter(I0, math.inf, 1.0, 0.01, 6, C=(5.0, 2.0, 1.0))
    # weights tau*C_a play the role of dt/h_a^2
    h = tuple(1.0 / math.sqrt(0.01 * Ca) for Ca in (5.0, 2.0, 1.0))
    ref = heat_closed_form(I0, 1.0, 6, h)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(I0).max()


# ------------------------------------------------------- sums, noise, formats
def test_stats_and_noise_rms():
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(100_003) * 3.0).astype(np.float32)
    s = oracle.stats(x)
    xd = x.astype(np.float64)
    assert s["sum"] == pytest.approx(math.fsum(xd), rel=1e-12, abs=1e-9)
    assert s["sumsq"] == pytest.approx(math.fsum(xd * xd), rel=1e-12)
    neg = xd[xd < 0]
    assert s["nneg"] == neg.size
    assert s["negsumsq"] == pytest.approx(math.fsum(neg * neg), rel=1e-12)
    # symmetric +-a data: the negative half gives exactly a
    sym = np.array([2.0, -2.0, 2.0, -2.0, 2.0], dtype=np.float32)
    assert oracle.noise_rms(sym) == 2.0
    # emission is positive: adding it leaves the estimate near sigma = 3
    assert abs(oracle.noise_rms(x) - 3.0) < 0.03
    y = x.copy()
    y[:1000] += 50.0
    assert abs(oracle.noise_rms(y) - 3.0) < 0.03
    assert oracle.noise_rms(np.ones(10, np.float32)) == 0.0


def test_storage_formats():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(50_000) * 4.0).astype(np.float32)
    x[:6] = [0.0, -0.0, 1e-30, 65504.0, 3.0e4, -7.5]
    for s in (1.0, 0.5, 4.0):
        q16 = oracle.quantize(x, "f16", s)
        ref = torch.from_numpy(x / np.float32(s)).to(torch.float16).numpy().view(np.uint16)
        assert np.array_equal(q16, ref)
        qb = oracle.quantize(x, "bf16", s)
        refb = torch.from_numpy(x / np.float32(s)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        assert np.array_equal(qb, refb)
        # dequantize is exact: the stored value times a power of two
        assert np.array_equal(oracle.dequantize(q16, "f16", s),
                              q16.view(np.float16).astype(np.float32) * np.float32(s))
    # bf16 ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    t = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], dtype=np.float32)
    back = oracle.dequantize(oracle.quantize(t, "bf16", 1.0), "bf16", 1.0)
    assert back.tolist() == [1.0, 1 + 2 ** -6]
    # int16 fixed point: step s/1024, ties to even, clamped
    s = 2.0
    v = np.array([0.0, 1 / 512, 1.5 / 512, 2.5 / 512, 100.0, -100.0], dtype=np.float32)
    q = oracle.quantize(v, "i16", s)
    assert q.tolist() == [0, 1, 2, 2, 32767, -32767]
    big = (rng.uniform(-60, 60, 1000)).astype(np.float32)
    err = np.abs(oracle.dequantize(oracle.quantize(big, "i16", s), "i16", s) - big)
    assert err.max() <= s / 2048 + 1e-7
    assert oracle.pow2_scale(1.0) == 1.0 and oracle.pow2_scale(0.7) == 0.5
    assert oracle.pow2_scale(0.75) == 1.0 and oracle.pow2_scale(3.0) == 4.0

# ------------------------------------------------------- F diagnostics
def fdiag_hand_cubes():
    """2x2x2 hand example; rms 1, so both thresholds are 3.  Voxels exactly at
    3 belong to the masks (eq. "Mfequa": I >= 3 rms)."""
    Io = np.array([4, 1, 3, 0, -1, 2, 5, 0.5], np.float32).reshape(2, 2, 2)
    If = np.array([2, 3.5, 1, 3, 0, 0, 6, 3], np.float32).reshape(2, 2, 2)
    Im = np.array([3, 0, 2, 1, 0, 0, 4, 1], np.float32).reshape(2, 2, 2)
    return Io, If, Im


def test_f_diagnostic_hand_values():
    Io, If, Im = fdiag_hand_cubes()
    r = oracle.f_diagnostic(Io, If, Im, rms_o=1.0, rms_f=1.0)
    # M_o = {4, 3, 5}: S_oo = 12, N_o = 3.  M_f = {3.5, 3, 6, 3} at voxels
    # 1, 3, 6, 7: S_of = I_o there = 1 + 0 + 5 + 0.5 = 6.5 (Sec. 4: the sums
    # take the original intensities), N_f = 4.
    assert (r["S_oo"], r["N_o"], r["S_of"], r["N_f"]) == (12.0, 3, 6.5, 4)
    assert r["F"] == 6.5 / 12.0
    # sigma_F^2 = sigma_of^2 / S_oo^2 + S_of^2 sigma_oo^2 / S_oo^4 with
    # sigma_of = sqrt(4) * 1, sigma_oo = sqrt(3) * 1
    assert r["sigma_F"] == pytest.approx(math.sqrt(4 / 144 + 6.5 ** 2 * 3 / 12 ** 4), rel=1e-15)
    # F_M: S_m = 11, S_mf = I_m at 1, 3, 6, 7 = 0 + 1 + 4 + 1 = 6
    assert (r["S_m"], r["S_mf"], r["F_M"]) == (11.0, 6.0, 6.0 / 11.0)
    # independent voxels: a beam of 4 voxels divides N_i by 4, sigma_F by 2
    r4 = oracle.f_diagnostic(Io, If, Im, rms_o=1.0, rms_f=1.0, beam=4.0)
    assert r4["sigma_F"] == pytest.approx(r["sigma_F"] / 2, rel=1e-15)
    # another threshold multiple: at 2 rms, M_o = {4, 3, 2, 5} and M_f gains
    # voxel 0 (I_f = 2, I_o = 4)
    r2 = oracle.f_diagnostic(Io, If, rms_o=1.0, rms_f=1.0, nsig=2.0)
    assert (r2["S_oo"], r2["N_o"], r2["S_of"], r2["N_f"]) == (14.0, 4, 10.5, 5)


def test_f_diagnostic_invariants():
    rng = np.random.default_rng(21)
    Io = (rng.standard_normal((9, 11, 13)) * 1.3).astype(np.float32)
    Io[3:6, 4:8, 5:9] += 6.0
    If = (Io + rng.standard_normal(Io.shape).astype(np.float32) * 0.3).astype(np.float32)
    Im = np.clip(Io, 0, None).astype(np.float32)
    # unfiltered: F = 1 exactly and both error terms are equal
    r = oracle.f_diagnostic(Io, Io)
    assert r["F"] == 1.0 and r["N_f"] == r["N_o"]
    assert r["sigma_F"] == pytest.approx(math.sqrt(2 * r["N_o"]) * r["rms_o"] / abs(r["S_oo"]),
                                         rel=1e-14)
    # default rms: the noise estimate of each full cube
    r = oracle.f_diagnostic(Io, If, Im)
    assert r["rms_o"] == oracle.noise_rms(Io) and r["rms_f"] == oracle.noise_rms(If)
    # power-of-two scaling of every cube (and so of the rms) changes nothing
    r8 = oracle.f_diagnostic(Io * 8, If * 8, Im * 8)
    for key in ("F", "sigma_F", "F_M", "N_o", "N_f"):
        assert r8[key] == r[key], key
    # a ROI equals the same diagnostic on the cropped cubes with the same rms
    roi = (2, 10, 1, 9, 3, 7)
    a = oracle.f_diagnostic(Io, If, Im, roi=roi, rms_o=r["rms_o"], rms_f=r["rms_f"])
    crop = lambda c: np.ascontiguousarray(c[3:7, 1:9, 2:10])
    b = oracle.f_diagnostic(crop(Io), crop(If), crop(Im), rms_o=r["rms_o"], rms_f=r["rms_f"])
    assert a == b
    # brute force in plain numpy on the whole cube
    mo, mf = Io >= 3 * r["rms_o"], If >= 3 * r["rms_f"]
    d = Io.astype(np.float64)
    assert r["S_oo"] == pytest.approx(math.fsum(d[mo]), rel=1e-13)
    assert r["S_of"] == pytest.approx(math.fsum(d[mf]), rel=1e-13)
    assert (r["N_o"], r["N_f"]) == (int(mo.sum()), int(mf.sum()))
    with pytest.raises(ValueError):
        oracle.f_diagnostic(Io, If, roi=(0, 0, 0, 1, 0, 1))


# ------------------------------------------------------- box / Gaussian smoothing
def smooth_library(cube, w):
    """The same normalised correlation through scipy.ndimage: zero-padded
    correlation divided by the zero-padded correlation of ones."""
    nd = pytest.importorskip("scipy.ndimage")
    c = np.asarray(cube, dtype=np.float64)
    return nd.correlate(c, w, mode="constant") / nd.correlate(np.ones_like(c), w, mode="constant")


def test_box_hand_values():
    c = np.arange(4 * 5 * 6, dtype=np.float32).reshape(4, 5, 6)   # value = x + 6y + 30z
    r = oracle.smooth(c, oracle.box_weights((3, 3, 3)))
    # interior: the mean of a linear field over a centred window is its centre value
    assert r[2, 2, 2] == c[2, 2, 2]
    # corner (0,0,0): the mean over the 2x2x2 in-cube block = 0.5 + 3 + 15
    assert r[0, 0, 0] == pytest.approx(18.5, abs=1e-12)
    # a 1x1x1 box is the identity; a 1-D box averages along its axis only
    assert np.array_equal(oracle.smooth(c, oracle.box_weights((1, 1, 1))), c)
    r = oracle.smooth(c, oracle.box_weights((5, 1, 1)))
    assert r[1, 1, 0] == pytest.approx((c[1, 1, 0] + c[1, 1, 1] + c[1, 1, 2]) / 3, abs=1e-12)
    with pytest.raises(ValueError):
        oracle.box_weights((2, 3, 3))


def test_gauss_kernel_definition():
    # FWHM: the profile falls to one half at FWHM / 2 (FWHM = 2 sqrt(2 ln 2) sigma)
    w = oracle.gauss_weights((2.0, 2.0, 2.0))
    rz, ry, rx = (s // 2 for s in w.shape)
    assert w[rz, ry, rx] == 1.0
    assert w[rz, ry, rx + 1] == pytest.approx(0.5, abs=1e-15)
    # truncation at 3 sigma: sigma = 2 / 2.3548 = 0.849 -> r = ceil(2.548) = 3
    assert w.shape == (7, 7, 7)
    # axis-aligned: the outer product of three 1-D Gaussians
    w = oracle.gauss_weights((3.0, 5.0, 1.5))
    sig = np.array([3.0, 5.0, 1.5]) / oracle.FWHM_PER_SIGMA
    g = [np.exp(-0.5 * (np.arange(-(n // 2), n // 2 + 1) / s) ** 2)
         for n, s in zip(w.shape[::-1], sig)]
    assert np.allclose(w, g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :],
                       rtol=1e-14, atol=0)
    # rotation by 90 degrees about z swaps the x and y widths
    a = oracle.gauss_weights((3.0, 5.0, 2.0), (0.0, 0.0, 90.0))
    b = oracle.gauss_weights((5.0, 3.0, 2.0))
    assert a.shape == b.shape and np.allclose(a, b, rtol=1e-12, atol=1e-15)
    # R = Rz Ry Rx: a rotation about z maps x to (cos, sin, 0)
    R = oracle.rotation((0.0, 0.0, 30.0))
    assert np.allclose(R @ [1, 0, 0], [math.cos(math.radians(30)), math.sin(math.radians(30)), 0])
    assert np.allclose(oracle.rotation((10, 20, 30)) @ oracle.rotation((10, 20, 30)).T, np.eye(3))


def test_smooth_against_library_and_invariants():
    rng = np.random.default_rng(31)
    c = rng.standard_normal((9, 10, 12)).astype(np.float32)
    for w in (oracle.box_weights((3, 5, 1)), oracle.gauss_weights((3.0, 2.0, 1.0)),
              oracle.gauss_weights((4.0, 2.0, 3.0), (20.0, -35.0, 60.0))):
        assert np.allclose(oracle.smooth(c, w), smooth_library(c, w), rtol=0, atol=1e-13)
    # constants stay constant (renormalised at the faces)
    k = np.full((5, 6, 7), 2.5, dtype=np.float32)
    assert np.allclose(oracle.smooth(k, oracle.gauss_weights((3.0, 3.0, 3.0), (10, 20, 30))),
                       2.5, rtol=0, atol=1e-14)
    # a symmetric kernel commutes with flipping the cube
    w = oracle.gauss_weights((3.0, 2.0, 2.0))
    assert np.allclose(oracle.smooth(c[:, :, ::-1], w), oracle.smooth(c, w)[:, :, ::-1],
                       rtol=0, atol=1e-13)
