"""afd_filter_ex's passes of depth 2, 4 and 8 three ways, bit for bit, for
every storage format: chains of T one-iteration launches with float32
intermediate cubes (the default for widths that are a multiple of 8; the
ends on pm_wide.cu's storage <-> float32 kernels), chains of T/2 launches of
the two-iteration kernel (pm_wide2.cu, afd_set_kernel 'two_stage'), and the
general temporally blocked kernel (afd_set_kernel 'stream').  All compute
dequantise -> T canonical float32 iterations -> quantise, so any difference
is a staging, halo, boundary, hand-over or chaining mistake.  With float32
storage a pass also equals single-iteration passes.  Shapes cover
single planes, rows and columns, widths and heights at and around the
128 x 28 tile, iteration counts with a remainder (shallower passes at the
end), both conductances with anisotropic spacing, int16 with a non-unit
scale, in place and out of place, and forced z-chunks."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
RAW = {"f32": (torch.int32, np.int32), "f16": (torch.int16, np.uint16),
       "bf16": (torch.int16, np.uint16), "i16": (torch.int16, np.int16)}
SCALE = {"f32": 1.0, "f16": 1.0, "bf16": 1.0, "i16": 0.25}


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def stored(cube, storage):
    """The cube in its storage format, on the device."""
    if storage == "f32":
        return torch.from_numpy(cube).cuda()
    q = oracle.quantize(cube, storage, SCALE[storage])
    return torch.from_numpy(np.ascontiguousarray(q).view(np.int16)).view(TDT[storage]).cuda()


def run(afd, ctx, src, storage, K, dt, n, cond, sp, kernel, t_block=2, zc=0, inplace=False):
    afd.afd_set_kernel(ctx, kernel)
    afd.afd_set_stream_zchunk(ctx, zc)
    try:
        x = src.clone()
        out = x if inplace else torch.empty_like(x)
        afd.afd_filter_ex(ctx, x, out, storage, SCALE[storage], K, dt, n, cond, sp, t_block)
        afd.afd_sync(ctx)
    finally:
        afd.afd_set_kernel(ctx, "auto")
        afd.afd_set_stream_zchunk(ctx, 0)
    tdt, ndt = RAW[storage]
    return out.view(tdt).cpu().numpy().view(ndt)


def cube(shape, seed):
    rng = np.random.default_rng(seed)
    c = (rng.standard_normal(shape) * 2.0).astype(np.float32)
    c[tuple(s // 2 for s in shape)] = 9.0          # a bright voxel: large differences
    return c


SHAPES = [(1, 1, 8), (3, 2, 16), (2, 1, 136), (5, 33, 136), (17, 27, 128), (4, 28, 128),
          (6, 29, 256), (40, 72, 264), (9, 57, 520), (4, 40, 8), (7, 23, 128)]
CASES = (("rational", None, 1.0, 1 / 8), ("exponential", (1.0, 1.5, 0.75), 1.3, 0.1))


@pytest.mark.parametrize("T", [2, 4, 8])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "i16"])
def test_depth_equals_blocked_kernel(afd, ctx, shape, storage, T):
    src = stored(cube(shape, sum(shape) + len(storage) + T), storage)
    for cond, sp, K, dt in CASES:
        for n in (T, 2 * T - 1):
            b = run(afd, ctx, src, storage, K, dt, n, cond, sp, "stream", t_block=T)
            for kern in ("auto", "two_stage"):
                a = run(afd, ctx, src, storage, K, dt, n, cond, sp, kern, t_block=T)
                assert np.array_equal(a, b), (kern, cond, n, int((a != b).sum()))


@pytest.mark.parametrize("T", [2, 4, 8])
@pytest.mark.parametrize("shape", [(3, 2, 16), (17, 23, 128), (40, 72, 264)])
def test_float32_depth_equals_single_passes(afd, ctx, shape, T):
    src = stored(cube(shape, 3 * sum(shape)), "f32")
    for cond, sp, K, dt in CASES:
        b = run(afd, ctx, src, "f32", K, dt, 2 * T, cond, sp, "stream", t_block=1)
        for kern in ("auto", "two_stage"):
            a = run(afd, ctx, src, "f32", K, dt, 2 * T, cond, sp, kern, t_block=T)
            assert np.array_equal(a, b), (kern, cond, T)


@pytest.mark.parametrize("T", [2, 4])
@pytest.mark.parametrize("zc", [1, 3, 7])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_depth_zchunks_and_in_place(afd, ctx, zc, storage, T):
    src = stored(cube((23, 45, 200), zc), storage)
    ref = run(afd, ctx, src, storage, 1.0, 1 / 8, 2 * T, "rational", None, "stream", t_block=T)
    for kern in ("auto", "two_stage"):
        got = run(afd, ctx, src, storage, 1.0, 1 / 8, 2 * T, "rational", None, kern,
                  t_block=T, zc=zc)
        assert np.array_equal(got, ref), kern
        got = run(afd, ctx, src, storage, 1.0, 1 / 8, 2 * T, "rational", None, kern,
                  t_block=T, zc=zc, inplace=True)
        assert np.array_equal(got, ref), kern


@pytest.mark.parametrize("T", [2, 4, 8])
def test_depth_against_oracle(afd, ctx, T):
    c = cube((20, 37, 136), 5)
    ref = oracle.pm_filter(c, 1.0, 0.125, 10, "rational")
    for kern in ("auto", "two_stage"):
        got = run(afd, ctx, stored(c, "f32"), "f32", 1.0, 0.125, 10, "rational", None, kern,
                  t_block=T)
        # float32 rounding of 10 iterations over values up to 9 (the bright voxel)
        assert np.abs(got.view(np.float32) - ref).max() <= 4e-4, kern


def test_tuner_picks_a_route_at_the_minimum_depth(afd, ctx):
    """tune.Tuner.tune_filter_ex with min_depth 4 on a real cube: it times
    depths 4 and 8 over both routes, leaves its choice applied, and the
    tuned call gives the general kernel's bits."""
    from paper_1609_03782_gb300 import tune
    src = stored(cube((24, 64, 128), 11), "f16")
    out = torch.empty_like(src)
    t = tune.Tuner(cache_path=None, reps=1)
    try:
        T = t.tune_filter_ex(afd, ctx, src, out, "f16", 1.0, 1.0, 1 / 8, 8, "rational",
                             zchunks=(0,), min_depth=4)
        assert T in (4, 8)
        afd.afd_filter_ex(ctx, src, out, "f16", 1.0, 1.0, 1 / 8, 8, "rational", None, T)
        afd.afd_sync(ctx)
        got = out.view(torch.int16).cpu().numpy().view(np.uint16)
    finally:
        afd.afd_set_kernel(ctx, "auto")
        afd.afd_set_stream_zchunk(ctx, 0)
    ref = run(afd, ctx, src, "f16", 1.0, 1 / 8, 8, "rational", None, "stream", t_block=T)
    assert np.array_equal(got, ref)
