"""GPU parity for the precision line: 2-byte storage and temporal blocking.

* afd_quantize / afd_dequantize are bit-exact against the oracle's
  definitions (round to nearest even into float16 / bfloat16 / int16 counts,
  exact power-of-two scaling).
* afd_filter_ex with float32 storage is bit-identical to afd_filter_out for
  every depth T: T fused iterations per pass change no rounding.
* afd_filter_ex with 2-byte storage is bit-identical, code for code, to the
  composition of its passes: dequantise (oracle) -> T float32 iterations
  (afd_filter_out) -> quantise (oracle).
* Against the FP64 oracle on the float32 input, the error is bounded by the
  storage rounding: at most half a unit in the last place of the largest
  stored value per pass, plus the float32 tolerance; the error norms of
  every format are checked against that bound.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
NPDT = {"f16": np.uint16, "bf16": np.uint16, "i16": np.int16}


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def to_bits(t, storage):
    """Storage tensor -> numpy array of its 16-bit codes."""
    return t.cpu().view(torch.int16).numpy().view(NPDT[storage])


def from_bits(q, storage):
    return torch.from_numpy(np.ascontiguousarray(q).view(np.int16)).view(TDT[storage]).cuda()


def pass_depths(n, T):
    d = [T] * (n // T)
    left = n - T * (n // T)
    for s in (4, 2, 1):
        while s <= T and left >= s:
            d.append(s)
            left -= s
    return d


@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
@pytest.mark.parametrize("scale", [1.0, 0.5, 4.0])
def test_quantize_dequantize_bit_exact(afd, ctx, storage, scale):
    rng = np.random.default_rng(21)
    x = (rng.standard_normal(100_003) * 6).astype(np.float32)
    x[:8] = [0.0, -0.0, 1e-30, 7e4, -7e4, 1 + 2 ** -11, 100.0, -33.0 * scale]
    t = torch.from_numpy(x).cuda()
    q = torch.empty(x.size, dtype=TDT[storage], device="cuda")
    afd.afd_quantize(ctx, t, q, storage, scale)
    afd.afd_sync(ctx)
    ref = oracle.quantize(x, storage, scale)
    assert np.array_equal(to_bits(q, storage), ref.view(NPDT[storage]))
    back = torch.empty_like(t)
    afd.afd_dequantize(ctx, q, back, storage, scale)
    afd.afd_sync(ctx)
    bref = oracle.dequantize(ref, storage, scale)
    assert np.array_equal(back.cpu().numpy().view(np.uint32), bref.view(np.uint32))
    # an input that is not 16-byte aligned takes the scalar path
    q2 = torch.empty(x.size - 1, dtype=TDT[storage], device="cuda")
    afd.afd_quantize(ctx, t[1:], q2, storage, scale)
    afd.afd_sync(ctx)
    assert np.array_equal(to_bits(q2, storage), ref[1:].view(NPDT[storage]))


def test_bad_scale_rejected(afd, ctx):
    t = torch.zeros(16, device="cuda")
    q = torch.empty(16, dtype=torch.float16, device="cuda")
    for s in (0.0, -1.0, 3.0, float("inf"), float("nan")):
        with pytest.raises(afd.AfdError) as ei:
            afd.afd_quantize(ctx, t, q, "f16", s)
        assert ei.value.status == afd.AFD_EINVAL


SHAPES = [(1, 1, 8), (5, 17, 32), (37, 45, 136), (70, 33, 64), (9, 20, 200), (3, 40, 1000)]


@pytest.mark.parametrize("T", [1, 2, 4, 8])
@pytest.mark.parametrize("shape", SHAPES)
def test_f32_blocked_bit_identical_to_plain(afd, ctx, T, shape):
    rng = np.random.default_rng(sum(shape) + T)
    cube = (rng.standard_normal(shape) * 2).astype(np.float32)
    src = torch.from_numpy(cube).cuda()
    for cond, n in (("rational", 7), ("exponential", 2 * T + 1)):
        ref = torch.empty_like(src)
        afd.afd_filter_out(ctx, src, ref, 1.2, 0.1, n, cond, (1.0, 1.25, 0.8))
        got = torch.full_like(src, float("nan"))
        afd.afd_filter_ex(ctx, src, got, "f32", 1.0, 1.2, 0.1, n, cond, (1.0, 1.25, 0.8), T)
        afd.afd_sync(ctx)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32)), \
            (cond, n)


def test_f32_blocked_zchunks_and_fallback(afd, ctx):
    cube = synth.cube512()[:100, :70, :72].copy()
    src = torch.from_numpy(cube).cuda()
    ref = torch.empty_like(src)
    afd.afd_filter_out(ctx, src, ref, 1.0, 1 / 8, 8, "rational")
    for zc in (1, 3, 16):
        afd.afd_set_stream_zchunk(ctx, zc)
        got = torch.empty_like(src)
        afd.afd_filter_ex(ctx, src, got, "f32", 1.0, 1.0, 1 / 8, 8, "rational", None, 4)
        afd.afd_sync(ctx)
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), zc
    afd.afd_set_stream_zchunk(ctx, 0)
    # nx % 4 != 0: passes go through float32 scratch, same bits
    odd = torch.from_numpy(cube[:, :, :71].copy()).cuda()
    r2 = torch.empty_like(odd)
    afd.afd_filter_out(ctx, odd, r2, 1.0, 1 / 8, 6, "rational")
    g2 = torch.empty_like(odd)
    afd.afd_filter_ex(ctx, odd, g2, "f32", 1.0, 1.0, 1 / 8, 6, "rational", None, 4)
    afd.afd_sync(ctx)
    assert torch.equal(g2.view(torch.int32), r2.view(torch.int32))
    # in place
    inp = src.clone()
    afd.afd_filter_ex(ctx, inp, inp, "f32", 1.0, 1.0, 1 / 8, 8, "rational", None, 2)
    afd.afd_sync(ctx)
    assert torch.equal(inp.view(torch.int32), ref.view(torch.int32))


def lp_reference(afd, ctx, q0, storage, scale, K, dt, n, cond, T, spacing=None):
    """Passes composed from their definition: oracle dequantise, float32
    iterations on the GPU, oracle quantise."""
    q = q0
    for d in pass_depths(n, T):
        v = torch.from_numpy(oracle.dequantize(q, storage, scale)).cuda()
        o = torch.empty_like(v)
        afd.afd_filter_out(ctx, v, o, K, dt, d, cond, spacing)
        afd.afd_sync(ctx)
        q = oracle.quantize(o.cpu().numpy(), storage, scale)
    return q


@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
@pytest.mark.parametrize("T", [1, 2, 4, 8])
def test_2byte_passes_bit_exact(afd, ctx, storage, T):
    cube = synth.cube512()[:40, :72, :136].copy()
    scale = oracle.pow2_scale(1.0)
    q0 = oracle.quantize(cube, storage, scale)
    n = 2 * T + 3 if T < 8 else 11
    ref = lp_reference(afd, ctx, q0, storage, scale, 1.0, 1 / 8, n, "rational", T)
    src = from_bits(q0, storage)
    got = torch.empty_like(src)
    afd.afd_filter_ex(ctx, src, got, storage, scale, 1.0, 1 / 8, n, "rational", None, T)
    afd.afd_sync(ctx)
    g = to_bits(got, storage)
    assert np.array_equal(g, ref.view(NPDT[storage])), int((g != ref.view(NPDT[storage])).sum())


@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
def test_2byte_odd_width_fallback_bit_exact(afd, ctx, storage):
    cube = synth.cube64()[:20, :30, :44].copy()   # 44 * 2 bytes is not a multiple of 16
    q0 = oracle.quantize(cube, storage, 1.0)
    ref = lp_reference(afd, ctx, q0, storage, 1.0, 1.5, 1 / 16, 6, "exponential", 4)
    src = from_bits(q0, storage)
    got = torch.empty_like(src)
    afd.afd_filter_ex(ctx, src, got, storage, 1.0, 1.5, 1 / 16, 6, "exponential", None, 4)
    afd.afd_sync(ctx)
    assert np.array_equal(to_bits(got, storage), ref.view(NPDT[storage]))


def rounding_bounds(storage, cond, dt, n, T, vmax, scale, sigma=1.0):
    """(max-norm bound, faint-band rms bound) on the error of a 2-byte run of
    n iterations at depth T against the FP64 oracle on the float32 input:
    every rounding into the storage format (the initial one and one per pass)
    adds at most half an ulp of the largest value, amplified by the scheme's
    Lipschitz constant L per later iteration; the float32 arithmetic adds its
    own 1e-4 sigma.  In the faint band (|I| < 3 sigma) the rms stays within
    one faint half-ulp per rounding."""
    L = lipschitz(cond, dt)
    done, amp = 0, L ** n          # the initial rounding, before any iteration
    for d in pass_depths(n, T):
        done += d
        amp += L ** (n - done)     # the rounding at the end of this pass
    rounds = len(pass_depths(n, T)) + 1
    return (amp * half_ulp(storage, vmax, scale) + 1e-4 * sigma,
            rounds * half_ulp(storage, 3 * sigma, scale) + 1e-4 * sigma)


def half_ulp(storage, vmax, scale):
    if storage == "i16":
        return scale / 2048.0
    mant = 10 if storage == "f16" else 7
    e = math.floor(math.log2(vmax / scale))
    return scale * 2.0 ** (e - mant) / 2.0


def lipschitz(cond, dt):
    """Per-iteration infinity-norm Lipschitz bound of the explicit scheme with
    unit spacing: a perturbation e changes by e_p (1 - dt sum phi') +
    dt sum phi' e_q, phi(d) = g(d) d, so |e'| <= (1 + 12 dt m) |e| with
    m = max(-phi'): 2 exp(-3/2) for g = exp(-(d/K)^2) (at d^2 = 1.5 K^2) and
    1/8 for g = 1/(1+(d/K)^2) (at d^2 = 3 K^2).  Above 1 where differences
    exceed K/sqrt(2) (exponential) or K (rational): backward diffusion."""
    m = 2.0 * math.exp(-1.5) if cond == "exponential" else 0.125
    return 1.0 + 12.0 * dt * m


@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
@pytest.mark.parametrize("T", [1, 2, 4, 8])
def test_error_vs_fp64_oracle(afd, ctx, storage, T):
    """cube64 (exponential, K = 1.5, dt = 1/16, 10 iterations) against the
    FP64 oracle on the float32 input.  Every rounding into the storage format
    (the initial one and one per pass) adds at most half an ulp of the
    largest value, and each is amplified by at most L per later iteration
    (lipschitz above); the float32 arithmetic adds its own 1e-4 sigma.  The
    rms in the faint band (|I| < 3 sigma) stays within the faint values' own
    half-ulp per rounding."""
    cube = synth.cube64()
    sigma = 1.0
    scale = oracle.pow2_scale(oracle.noise_rms(cube))
    n, dt = 10, 1 / 16
    ref = oracle.pm_filter(cube, 1.5 * sigma, dt, n, "exponential")
    src = torch.empty(cube.shape, dtype=TDT[storage], device="cuda")
    afd.afd_quantize(ctx, torch.from_numpy(cube).cuda(), src, storage, scale)
    got = torch.empty_like(src)
    afd.afd_filter_ex(ctx, src, got, storage, scale, 1.5 * sigma, dt, n, "exponential", None, T)
    out = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    afd.afd_dequantize(ctx, got, out, storage, scale)
    afd.afd_sync(ctx)
    err = np.abs(out.cpu().numpy() - ref)
    L = lipschitz("exponential", dt)
    done, amp = 0, L ** n          # the initial rounding, before any iteration
    for d in pass_depths(n, T):
        done += d
        amp += L ** (n - done)     # the rounding at the end of this pass
    h = half_ulp(storage, float(np.abs(cube).max()), scale)
    bound = amp * h + 1e-4 * sigma
    assert err.max() <= bound, (err.max(), bound)
    faint = np.abs(ref) < 3 * sigma
    rounds = len(pass_depths(n, T)) + 1
    faint_rms = float(np.sqrt(np.mean(err[faint] ** 2)))
    assert faint_rms <= rounds * half_ulp(storage, 3 * sigma, scale) + 1e-4 * sigma, faint_rms
