"""The 8 x 2-voxel depth-1 pass for 2-byte storage (pm_wide.cu) against the
4 x 2-voxel streaming kernel (pm_stream.cu), bit for bit: both compute the
canonical per-face arithmetic, so any difference is a mapping, halo or
boundary mistake.  Shapes cover single planes, rows and columns, widths
that are not a multiple of the 128-wide tile, heights that are not a
multiple of the 32-row tile, odd z-chunks, anisotropic spacing, both
conductances, every 2-byte format, and the in-place form."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
NPDT = {"f16": np.uint16, "bf16": np.uint16, "i16": np.int16}


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def run(afd, ctx, q, storage, scale, K, dt, n, cond, sp, kernel, zc=0, inplace=False):
    afd.afd_set_kernel(ctx, kernel)
    afd.afd_set_stream_zchunk(ctx, zc)
    src = torch.from_numpy(np.ascontiguousarray(q).view(np.int16)).view(TDT[storage]).cuda()
    out = src if inplace else torch.empty_like(src)
    afd.afd_filter_ex(ctx, src, out, storage, scale, K, dt, n, cond, sp, 1)
    afd.afd_sync(ctx)
    afd.afd_set_kernel(ctx, "auto")
    afd.afd_set_stream_zchunk(ctx, 0)
    return out.cpu().view(torch.int16).numpy().view(NPDT[storage])


SHAPES = [(1, 1, 8), (3, 2, 8), (2, 1, 136), (5, 33, 136), (17, 31, 128), (2, 65, 256),
          (33, 40, 24), (40, 72, 264), (9, 3, 392)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
def test_wide_equals_streaming_kernel(afd, ctx, shape, storage):
    rng = np.random.default_rng(list(TDT).index(storage) * 1000 + sum(shape))
    cube = (rng.standard_normal(shape) * 2.0).astype(np.float32)
    cube[tuple(s // 2 for s in shape)] = 9.0          # a bright voxel: large differences
    scale = 1.0
    q = oracle.quantize(cube, storage, scale)
    for cond, sp, K, dt in (("rational", None, 1.0, 1 / 8),
                            ("exponential", (1.0, 1.5, 0.75), 1.3, 0.1)):
        a = run(afd, ctx, q, storage, scale, K, dt, 3, cond, sp, "auto")
        b = run(afd, ctx, q, storage, scale, K, dt, 3, cond, sp, "stream")
        assert np.array_equal(a, b), (cond, int((a != b).sum()))


@pytest.mark.parametrize("zc", [1, 3, 7])
def test_wide_zchunks_and_in_place(afd, ctx, zc):
    rng = np.random.default_rng(zc)
    cube = (rng.standard_normal((23, 45, 200)) * 2.0).astype(np.float32)
    q = oracle.quantize(cube, "f16", 1.0)
    ref = run(afd, ctx, q, "f16", 1.0, 1.0, 1 / 8, 4, "rational", None, "stream")
    got = run(afd, ctx, q, "f16", 1.0, 1.0, 1 / 8, 4, "rational", None, "auto", zc=zc)
    assert np.array_equal(got, ref)
    got = run(afd, ctx, q, "f16", 1.0, 1.0, 1 / 8, 4, "rational", None, "auto", zc=zc,
              inplace=True)
    assert np.array_equal(got, ref)
