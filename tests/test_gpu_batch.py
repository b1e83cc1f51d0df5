"""GPU parity for the batching line: many uneven cubes filtered together.

Every cube's result must be bit-identical to the single-cube entry point
with the same K (the batched kernel runs the same per-voxel code); the K
each cube gets from its GPU noise estimate must match the FP64 oracle's
estimate; a sample of cubes is checked against the FP64 oracle itself.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f32": torch.float32, "f16": torch.float16}


def tol(n):
    return min(1e-5 * n, 1e-4)


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def shapes(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append((int(rng.integers(3, 40)), int(rng.integers(5, 90)), int(rng.integers(5, 150))))
    out[0] = (1, 1, 1)
    out[1] = (40, 70, 129)   # several tiles, odd width
    return out


@pytest.mark.parametrize("tiles", ["wide", "64x32"])
def test_batch_fp32_matches_alone_and_oracle(afd, ctx, tiles):
    shp = shapes(14, 3)
    cubes = [synth.cutout(s, 50 + i) for i, s in enumerate(shp)]
    b = afd.afd_batch_create(ctx, shp, "f32")
    afd.afd_batch_set_tiles(b, tiles)
    try:
        for i, c in enumerate(cubes):
            afd.afd_batch_set(b, i, torch.from_numpy(c).cuda())
        K = [-1.5] * len(shp)
        K[3] = 2.25                       # one absolute K
        afd.afd_batch_filter(b, K, 1 / 8, 20, "rational")
        Kused = afd.afd_batch_k(b)
        for i, c in enumerate(cubes):
            got = afd.afd_batch_get(b, i, torch.empty(shp[i], device="cuda")).cpu().numpy()
            if i == 3:
                assert Kused[i] == np.float32(2.25)
            else:
                sig = oracle.noise_rms(c)
                assert abs(Kused[i] / 1.5 - sig) <= 1e-6 * max(sig, 1e-30), (i, Kused[i], sig)
            src = torch.from_numpy(c).cuda()
            ref = torch.empty_like(src)
            afd.afd_filter_out(ctx, src, ref, float(Kused[i]), 1 / 8, 20, "rational")
            afd.afd_sync(ctx)
            assert np.array_equal(got.view(np.uint32), ref.cpu().numpy().view(np.uint32)), i
            if i < 4:
                o = oracle.pm_filter(c, float(Kused[i]), 1 / 8, 20, "rational")
                assert np.abs(got - o).max() <= tol(20), i
        # replay of the captured graph, then a retuned z-chunk: same bits
        first = afd.afd_batch_get(b, 1, torch.empty(shp[1], device="cuda")).clone()
        afd.afd_batch_filter(b, K, 1 / 8, 20, "rational")
        again = afd.afd_batch_get(b, 1, torch.empty(shp[1], device="cuda"))
        afd.afd_sync(ctx)
        assert torch.equal(first.view(torch.int32), again.view(torch.int32))
        afd.afd_batch_set_zchunk(b, 5)
        afd.afd_batch_filter(b, K, 1 / 8, 20, "rational")
        tuned = afd.afd_batch_get(b, 1, torch.empty(shp[1], device="cuda"))
        afd.afd_sync(ctx)
        assert torch.equal(first.view(torch.int32), tuned.view(torch.int32))
    finally:
        b.close()


@pytest.mark.parametrize("tiles", ["wide", "64x32"])
@pytest.mark.parametrize("storage", ["f16", "bf16", "i16"])
@pytest.mark.parametrize("cond", ["exponential", "rational"])
def test_batch_2byte_matches_alone(afd, ctx, cond, storage, tiles):
    shp = [(24, 40, 64), (17, 33, 77), (30, 64, 200), (5, 9, 11), (9, 150, 33), (3, 2, 260)]
    cubes = [synth.cutout(s, 7 + i) for i, s in enumerate(shp)]
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}[storage]
    b = afd.afd_batch_create(ctx, shp, storage, 1.0)
    afd.afd_batch_set_tiles(b, tiles)
    try:
        qs = []
        for i, c in enumerate(cubes):
            q = torch.empty(shp[i], dtype=tdt, device="cuda")
            afd.afd_quantize(ctx, torch.from_numpy(c).cuda(), q, storage, 1.0)
            qs.append(q)
            afd.afd_batch_set(b, i, q)
        afd.afd_batch_filter(b, [-1.5] * len(shp), 1 / 16, 7, cond, (1.0, 1.0, 0.5))
        Kused = afd.afd_batch_k(b)
        for i in range(len(shp)):
            got = afd.afd_batch_get(b, i, torch.empty(shp[i], dtype=tdt, device="cuda"))
            ref = torch.empty_like(qs[i])
            afd.afd_filter_ex(ctx, qs[i], ref, storage, 1.0, float(Kused[i]), 1 / 16, 7, cond,
                              (1.0, 1.0, 0.5), 1)
            afd.afd_sync(ctx)
            assert torch.equal(got.view(torch.int16), ref.view(torch.int16)), i
    finally:
        b.close()


@pytest.mark.parametrize("tiles", ["wide", "64x32"])
def test_batch_heat_equation_limit(afd, ctx, tiles):
    # K = +inf on every cube: the linear flux (g = 1), the discrete heat
    # equation; each cube equal to the single-cube filter with K = +inf
    shp = [(12, 30, 45), (20, 70, 129), (4, 5, 3)]
    cubes = [synth.cutout(s, 31 + i) for i, s in enumerate(shp)]
    b = afd.afd_batch_create(ctx, shp, "f32")
    afd.afd_batch_set_tiles(b, tiles)
    try:
        for i, c in enumerate(cubes):
            afd.afd_batch_set(b, i, torch.from_numpy(c).cuda())
        afd.afd_batch_filter(b, [float("inf")] * len(shp), 0.1, 6, "rational")
        for i, c in enumerate(cubes):
            got = afd.afd_batch_get(b, i, torch.empty(shp[i], device="cuda"))
            src = torch.from_numpy(c).cuda()
            ref = torch.empty_like(src)
            afd.afd_filter_out(ctx, src, ref, float("inf"), 0.1, 6, "rational")
            afd.afd_sync(ctx)
            assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), i
        o = oracle.pm_filter(cubes[1], float("inf"), 0.1, 6, "rational")
        assert np.abs(afd.afd_batch_get(b, 1, torch.empty(shp[1], device="cuda")).cpu().numpy()
                      - o).max() <= tol(6) * 10
    finally:
        b.close()


def test_batch_tile_kind_switch_keeps_bits(afd, ctx):
    # the same batch filtered under both tile kinds, switching back and forth
    shp = shapes(9, 11)
    cubes = [synth.cutout(s, 90 + i) for i, s in enumerate(shp)]
    b = afd.afd_batch_create(ctx, shp, "f32")
    try:
        for i, c in enumerate(cubes):
            afd.afd_batch_set(b, i, torch.from_numpy(c).cuda())
        res = {}
        for kind in ("wide", "64x32", "wide"):
            afd.afd_batch_set_tiles(b, kind)
            afd.afd_batch_filter(b, [-1.5] * len(shp), 1 / 8, 9, "rational")
            res.setdefault(kind, []).append(
                [afd.afd_batch_get(b, i, torch.empty(shp[i], device="cuda")).clone()
                 for i in range(len(shp))])
        afd.afd_sync(ctx)
        for i in range(len(shp)):
            a = res["wide"][0][i].view(torch.int32)
            assert torch.equal(a, res["64x32"][0][i].view(torch.int32)), i
            assert torch.equal(a, res["wide"][1][i].view(torch.int32)), i
        with pytest.raises(KeyError):
            afd.afd_batch_set_tiles(b, "square")
    finally:
        b.close()


def test_batch_argument_errors(afd, ctx):
    b = afd.afd_batch_create(ctx, [(4, 4, 4), (3, 5, 7)], "f32")
    try:
        for K in ([0.0, 1.0], [float("nan"), 1.0], [float("inf"), 1.0]):
            with pytest.raises(afd.AfdError) as ei:
                afd.afd_batch_filter(b, K, 0.1, 2, "rational")
            assert ei.value.status == afd.AFD_EINVAL
        with pytest.raises(ValueError):
            afd.afd_batch_set(b, 0, torch.zeros((4, 4, 5), device="cuda"))
    finally:
        b.close()
