"""afd_filter_slabs: a host cube through the device in z-slabs with halo
planes, in rounds of up to `halo` iterations.  Every result is bit-identical
to afd_filter on the whole cube in device memory (the same kernels on the
same neighbourhoods), across slab sizes, halos, iteration counts that halo
does not divide, one-slab and one-plane slabs; plus the FP64 oracle on a
small cube, the argument checks, and the 2048 x 2048 x 256 cube (4 GiB)
through 32-plane slabs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def whole(afd, ctx, cube, K, dt, n, cond, sp=None):
    d = torch.from_numpy(cube).cuda()
    afd.afd_filter(ctx, d, K, dt, n, cond, sp)
    afd.afd_sync(ctx)
    return d.cpu()


def slabbed(afd, ctx, cube, K, dt, n, cond, slab_nz, halo, sp=None):
    h_in = torch.from_numpy(cube).pin_memory()
    h_out = torch.full(cube.shape, float("nan")).pin_memory()
    h_tmp = torch.full(cube.shape, float("nan")).pin_memory()
    afd.afd_filter_slabs(ctx, h_in, h_out, K, dt, n, cond, sp, slab_nz, halo, h_tmp)
    assert torch.equal(h_in, torch.from_numpy(cube))       # input untouched
    return h_out


@pytest.mark.parametrize("shape,slab_nz,halo,n", [
    ((40, 33, 68), 8, 3, 10),      # rounds 3, 3, 3, 1
    ((40, 33, 68), 8, 8, 8),       # halo = slab, one round
    ((29, 17, 36), 5, 2, 7),       # ragged last slab, odd rounds
    ((29, 17, 36), 64, 4, 9),      # one slab: the whole cube
    ((12, 20, 24), 1, 3, 6),       # one-plane slabs
    ((9, 35, 132), 4, 20, 6),      # halo > n: one round, halo n
])
@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_slabs_equal_whole_cube(afd, ctx, shape, slab_nz, halo, n, cond):
    cube = synth.cutout(shape, sum(shape) + n)
    sp = (1.0, 1.5, 0.75)
    ref = whole(afd, ctx, cube, 1.2, 0.1, n, cond, sp)
    got = slabbed(afd, ctx, cube, 1.2, 0.1, n, cond, slab_nz, halo, sp)
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))


def test_slabs_against_oracle(afd, ctx):
    cube = synth.cutout((30, 40, 64), 11)
    got = slabbed(afd, ctx, cube, 1.0, 0.125, 12, "rational", 7, 5).numpy()
    ref = oracle.pm_filter(cube, 1.0, 0.125, 12, "rational")
    scale = float(np.abs(cube).max())
    assert np.abs(got - ref).max() <= 1e-5 * scale


def test_identities_and_argument_checks(afd, ctx):
    cube = synth.cutout((10, 12, 16), 3)
    for K, n in ((1.0, 0), (0.0, 5)):                      # n = 0 and K = 0: the input
        got = slabbed(afd, ctx, cube, K, 0.1, n, "rational", 3, 2)
        assert torch.equal(got, torch.from_numpy(cube))
    h = torch.from_numpy(cube)
    o = torch.empty_like(h)
    with pytest.raises(afd.AfdError):
        afd.afd_filter_slabs(ctx, h, h, 1.0, 0.1, 3, "rational")        # out == in
    with pytest.raises(afd.AfdError):
        afd.afd_filter_slabs(ctx, h, o, 1.0, 0.1, 9, "rational", None, 4, 2)  # rounds > 1, no tmp
    with pytest.raises(afd.AfdError):
        afd.afd_filter_slabs(ctx, h, o, 1.0, 0.1, 3, "rational", None, 0, 2)  # slab_nz < 1
    with pytest.raises(afd.AfdError):
        afd.afd_filter_slabs(ctx, h, o, 1.0, 0.1, 3, "rational", None, 4, 0)  # halo < 1
    got = afd.afd_filter_slabs(ctx, h, o, 1.0, 0.1, 2, "rational", None, 4, 2)  # one round
    assert torch.equal(got.view(torch.int32),
                       whole(afd, ctx, cube, 1.0, 0.1, 2, "rational").view(torch.int32))


def test_cube2048_through_slabs(afd, ctx):
    cube = synth.cube2048()
    d = torch.from_numpy(cube).cuda()
    sigma = afd.afd_noise_rms(ctx, d)
    K = float(np.float32(sigma))
    afd.afd_filter(ctx, d, K, 0.125, 30, "rational")
    afd.afd_sync(ctx)
    ref = d.cpu()
    del d
    got = slabbed(afd, ctx, cube, K, 0.125, 30, "rational", 32, 8)
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))


def test_slab_decomposition_gpu_step_single_rank(afd, ctx):
    # slabs.filter_slab with the library's step on a CUDA slab, one rank (no
    # neighbours: rounds of `halo` iterations, no exchange): the rounds equal
    # one afd_filter call bit for bit
    from paper_1609_03782_gb300 import slabs
    cube = synth.cutout((20, 24, 32), 9)
    own = torch.from_numpy(cube).cuda()
    got = slabs.filter_slab(own, 0, 20, 20, 11, 4, slabs.gpu_step(ctx, 1.1, 0.1))
    afd.afd_sync(ctx)
    ref = whole(afd, ctx, cube, 1.1, 0.1, 11, "rational")
    assert torch.equal(got.cpu().view(torch.int32), ref.view(torch.int32))


# the paper's intensity-driven form through the same slabs
@pytest.mark.parametrize("shape,slab_nz,halo,n", [
    ((40, 33, 68), 8, 3, 10),
    ((29, 17, 36), 5, 2, 7),
    ((12, 20, 24), 1, 3, 6),
    ((9, 35, 132), 4, 20, 6),
    ((64, 24, 40), 16, 20, 20),    # the paper's n = 20 in one round
])
def test_intensity_slabs_equal_whole_cube(afd, ctx, shape, slab_nz, halo, n):
    cube = synth.cutout(shape, 3 * sum(shape) + n)
    C, K, tau = (5.0, 4.0, 3.0), 1.5, 0.0325
    d = torch.from_numpy(cube).cuda()
    rms = afd.afd_noise_rms(ctx, d)
    o = torch.empty_like(d)
    afd.afd_filter_intensity(ctx, d, o, K, rms, tau, n, C)
    afd.afd_sync(ctx)
    ref = o.cpu()
    h_in = torch.from_numpy(cube).pin_memory()
    h_out = torch.full(cube.shape, float("nan")).pin_memory()
    h_tmp = torch.full(cube.shape, float("nan")).pin_memory()
    afd.afd_filter_intensity_slabs(ctx, h_in, h_out, K, rms, tau, n, C, slab_nz, halo, h_tmp)
    assert torch.equal(h_in, torch.from_numpy(cube))
    assert torch.equal(h_out.view(torch.int32), ref.view(torch.int32))


def test_intensity_slabs_identities_and_argument_checks(afd, ctx):
    cube = synth.cutout((10, 12, 16), 5)
    h_in = torch.from_numpy(cube)
    h_out = torch.empty_like(h_in)
    for K, rms, n in ((0.0, 1.0, 5), (1.5, 0.0, 5), (1.5, 1.0, 0)):   # S = 0 or no iterations
        afd.afd_filter_intensity_slabs(ctx, h_in, h_out, K, rms, 0.0325, n, (5.0, 5.0, 5.0), 4, 2,
                                       torch.empty_like(h_in))
        assert torch.equal(h_out, h_in)
    bad = [dict(tau=0.0), dict(tau=-1.0), dict(K=-1.0), dict(C=(1.0, -1.0, 1.0)),
           dict(slab_nz=0), dict(halo=0)]
    for b in bad:
        kw = dict(K=1.5, rms=1.0, tau=0.0325, n_iter=3, C=(5.0, 5.0, 5.0), slab_nz=4, halo=2)
        kw.update(b)
        with pytest.raises(afd.AfdError):
            afd.afd_filter_intensity_slabs(ctx, h_in, h_out, host_tmp=torch.empty_like(h_in),
                                           **kw)
    with pytest.raises(afd.AfdError):           # the result may not overwrite the input
        afd.afd_filter_intensity_slabs(ctx, h_in, h_in, 1.5, 1.0, 0.0325, 3)
    with pytest.raises(afd.AfdError):           # several rounds need host_tmp
        afd.afd_filter_intensity_slabs(ctx, h_in, h_out, 1.5, 1.0, 0.0325, 5, slab_nz=4, halo=2)
