"""GPU parity: the CUDA filter, called through the C ABI, against the FP64 oracle.

Tolerance (FP32 path): max |GPU - oracle| <= min(1e-5 * n_iter, 1e-4) * sigma,
sigma = 1 the generator's noise rms: 1e-5 sigma per iteration, never more than
1e-4 sigma after any number of iterations (50 at the full-size workload).
Every kernel variant must give bit-identical results (one canonical
per-voxel expression order).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA = 1.0


def tol(n_iter):
    return min(1e-5 * max(n_iter, 1), 1e-4) * SIGMA


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def run(afd, ctx, cube_np, K, dt, n, cond, spacing=None, kernel="auto", zc=0):
    afd.afd_set_kernel(ctx, kernel)
    afd.afd_set_stream_zchunk(ctx, zc)
    t = torch.from_numpy(np.ascontiguousarray(cube_np, dtype=np.float32)).cuda()
    afd.afd_filter(ctx, t, K, dt, n, cond, spacing)
    afd.afd_sync(ctx)
    out = t.cpu().numpy()
    afd.afd_set_kernel(ctx, "auto")
    afd.afd_set_stream_zchunk(ctx, 0)
    return out


def test_cube64_exponential_matches_oracle(afd, ctx):
    # 64^3, one disk, exponential g, K = 1.5 sigma, dt = 1/16, 10 iterations
    cube = synth.cube64()
    K = 1.5 * SIGMA
    ref = oracle.pm_filter(cube, K, 1 / 16, 10, "exponential")
    for kernel in ("simple", "stream"):
        got = run(afd, ctx, cube, K, 1 / 16, 10, "exponential", kernel=kernel)
        err = np.abs(got - ref).max()
        assert err <= tol(10), (kernel, err)
    a = run(afd, ctx, cube, K, 1 / 16, 10, "exponential", kernel="simple")
    b = run(afd, ctx, cube, K, 1 / 16, 10, "exponential", kernel="stream")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_single_iteration_error(afd, ctx, cond):
    cube = synth.cube64()
    ref = oracle.pm_filter(cube, 1.0, 1 / 8, 1, cond)
    got = run(afd, ctx, cube, 1.0, 1 / 8, 1, cond)
    assert np.abs(got - ref).max() <= tol(1)


SHAPES = [  # (nz, ny, nx): several tiles and a ragged tail on every axis
    (1, 1, 1), (1, 1, 4), (3, 1, 8), (2, 3, 5), (5, 17, 33), (9, 35, 132), (37, 19, 68),
    (12, 16, 64), (17, 40, 196),
    # last tile column 28 and 32 wide (the 8-quad mapping), last tile row 6 and 13 high
    (6, 70, 92), (5, 45, 160),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cond", ["rational", "exponential"])
def test_ragged_shapes_all_kernels(afd, ctx, shape, cond):
    rng = np.random.default_rng(sum(shape))
    cube = (rng.standard_normal(shape) * 2.0).astype(np.float32)
    n = 7
    ref = oracle.pm_filter(cube, 1.3, 0.1, n, cond, spacing=(1.0, 1.5, 0.75))
    sp = (1.0, 1.5, 0.75)
    a = run(afd, ctx, cube, 1.3, 0.1, n, cond, sp, kernel="simple")
    assert np.abs(a - ref).max() <= tol(n)
    if shape[2] % 4 == 0:
        for zc in (0, 1, 3, 5, 8):  # uneven chunk lengths where zc does not divide nz
            b = run(afd, ctx, cube, 1.3, 0.1, n, cond, sp, kernel="stream", zc=zc)
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), zc


def test_heat_limit_and_identities(afd, ctx):
    cube = synth.cube64()[:20, :24, :32].copy()
    # K = +inf: the discrete heat equation (oracle pinned to the DCT closed form)
    ref = oracle.pm_filter(cube, math.inf, 1 / 8, 6, "rational", spacing=(1.0, 2.0, 1.0))
    got = run(afd, ctx, cube, math.inf, 1 / 8, 6, "rational", spacing=(1.0, 2.0, 1.0))
    assert np.abs(got - ref).max() <= tol(6)
    # K = 0 and n = 0: identity, bit for bit
    assert np.array_equal(run(afd, ctx, cube, 0.0, 0.1, 5, "rational"), cube)
    assert np.array_equal(run(afd, ctx, cube, 1.0, 0.1, 0, "rational"), cube)
    # a constant cube is a fixed point, bit for bit
    c = np.full((9, 10, 12), 2.75, np.float32)
    for kernel in ("simple", "stream"):
        assert np.array_equal(run(afd, ctx, c, 1.0, 0.125, 4, "exponential", kernel=kernel), c)


def test_odd_iteration_count(afd, ctx):
    cube = synth.cube64()[:16, :16, :64].copy()
    ref = oracle.pm_filter(cube, 1.5, 1 / 16, 3, "exponential")
    for kernel in ("simple", "stream"):
        got = run(afd, ctx, cube, 1.5, 1 / 16, 3, "exponential", kernel=kernel)
        assert np.abs(got - ref).max() <= tol(3)


def test_stats_and_noise_rms(afd, ctx):
    cube = synth.cube512()[:96].copy()   # 512 x 512 x 96, ragged n % 16 handled too
    flat = np.concatenate([cube.ravel(), np.float32([-1.5, 2.0, -0.25])])
    t = torch.from_numpy(flat).cuda()
    out4 = torch.zeros(4, dtype=torch.float64, device="cuda")
    afd.afd_stats(ctx, t, out4)
    afd.afd_sync(ctx)
    g = out4.cpu().numpy()
    s = oracle.stats(flat)
    u = 2.0 ** -24
    absum = float(np.abs(flat.astype(np.float64)).sum())
    # float32 pairwise partials of 16: <= 4 ulp of the chunk's |sum|; squares +1 ulp
    assert abs(g[0] - s["sum"]) <= 5 * u * absum
    assert abs(g[1] - s["sumsq"]) <= 6 * u * s["sumsq"]
    assert abs(g[2] - s["negsumsq"]) <= 6 * u * s["negsumsq"]
    assert g[3] == s["nneg"]
    sig = afd.afd_noise_rms(ctx, t)
    assert abs(sig - math.sqrt(s["negsumsq"] / s["nneg"])) <= 4 * u * sig
    assert abs(sig - 1.0) < 0.01    # the generator's sigma
    assert afd.afd_sum(ctx, t) == g[0]
    # deterministic
    afd.afd_stats(ctx, t, out4)
    assert np.array_equal(out4.cpu().numpy(), g)


def test_full_size_cube512_sampled(afd, ctx):
    """512 x 512 x 256, rational g, K = 1.0 sigma from the GPU noise estimate,
    dt = 1/8, 50 iterations, launched as the benchmark launches it; sampled
    boxes (corners, faces, disks, interior) against the oracle through the
    50-voxel domain of dependence."""
    cube = synth.cube512()
    t = torch.from_numpy(cube).cuda()
    sig = afd.afd_noise_rms(ctx, t)
    sig_o = oracle.noise_rms(cube)
    assert abs(sig - sig_o) <= 1e-6 * sig_o
    K = float(np.float32(1.0 * sig))
    s0 = afd.afd_sum(ctx, t)
    afd.afd_filter(ctx, t, K, 1 / 8, 50, "rational")
    afd.afd_sync(ctx)
    s1 = afd.afd_sum(ctx, t)
    assert abs(s1 - s0) <= 1e-6 * float(np.abs(cube).sum())   # conservation
    got = t.cpu().numpy()
    assert np.isfinite(got).all()
    boxes = [((0, 6), (0, 6), (0, 8)),            # corner
             ((250, 256), (506, 512), (500, 512)),  # opposite corner
             ((125, 131), (200, 206), (0, 8)),      # x = 0 face
             ((126, 132), (254, 260), (252, 260))]  # interior
    # and one box on the brightest voxel (a disk centre)
    z, y, x = np.unravel_index(int(np.argmax(cube)), cube.shape)
    boxes.append(((max(0, z - 3), min(256, z + 3)), (max(0, y - 3), min(512, y + 3)),
                  (max(0, x - 4), min(512, x + 4))))
    worst = 0.0
    for box in boxes:
        ref = oracle.pm_filter_box(cube, box, K, 1 / 8, 50, "rational")
        (z0, z1), (y0, y1), (x0, x1) = box
        worst = max(worst, float(np.abs(got[z0:z1, y0:y1, x0:x1] - ref).max()))
    assert worst <= tol(50), worst


def test_determinism_and_host_entry(afd, ctx):
    cube = synth.cube64()
    a = run(afd, ctx, cube, 1.5, 1 / 16, 10, "exponential")
    b = run(afd, ctx, cube, 1.5, 1 / 16, 10, "exponential")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    h = torch.from_numpy(cube.copy()).pin_memory()
    ho = torch.empty_like(h).pin_memory()
    afd.afd_filter_host(ctx, h, ho, 1.5, 1 / 16, 10, "exponential")
    assert np.array_equal(ho.numpy().view(np.uint32), a.view(np.uint32))
    assert np.array_equal(h.numpy(), cube)          # input untouched
    afd.afd_filter_host(ctx, h, h, 1.5, 1 / 16, 10, "exponential")   # in == out
    assert np.array_equal(h.numpy().view(np.uint32), a.view(np.uint32))


@pytest.mark.parametrize("shape,cond,k,n", [((24, 40, 64), "rational", 1.0, 7),
                                             ((16, 33, 96), "exponential", 1.5, 4),
                                             ((10, 12, 30), "rational", 2.0, 3)])  # nx % 4 != 0
def test_filter_rel_equals_host_K(afd, ctx, shape, cond, k, n):
    # K relative to the noise rms, computed on the device: the same K and the
    # same result, bit for bit, as afd_filter_out with K from afd_noise_rms
    cube = synth.cutout(shape, 400 + n)
    src = torch.from_numpy(cube).cuda()
    sig = afd.afd_noise_rms(ctx, src)
    K = float(np.float32(np.float32(k) * sig))
    ref = torch.empty_like(src)
    afd.afd_filter_out(ctx, src, ref, K, 1 / 8, n, cond, (1.0, 1.25, 0.8))
    got = torch.full_like(src, float("nan"))
    K_dev = torch.zeros(1, dtype=torch.float32, device="cuda")
    afd.afd_filter_rel(ctx, src, got, k, 1 / 8, n, cond, (1.0, 1.25, 0.8), K_out=K_dev)
    afd.afd_sync(ctx)
    assert float(K_dev.item()) == K
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))


def test_filter_rel_without_noise_is_identity(afd, ctx):
    cube = np.abs(synth.cutout((8, 16, 32), 7)) + 1.0      # no negative voxel: rms 0
    src = torch.from_numpy(cube).cuda()
    got = torch.empty_like(src)
    K_dev = torch.full((1,), -1.0, device="cuda")
    afd.afd_filter_rel(ctx, src, got, 1.5, 1 / 8, 5, "rational", K_out=K_dev)
    afd.afd_sync(ctx)
    assert float(K_dev.item()) == 0.0
    assert torch.equal(got, src)
    with pytest.raises(afd.AfdError):
        afd.afd_filter_rel(ctx, src, got, 0.0, 1 / 8, 5, "rational")


def test_host_async_sequence(afd, ctx):
    # several cubes in flight through the two staging slots, with different
    # shapes (a slot grows while the other is busy; a slot takes a small cube
    # and then a larger one within its capacity, whose copy in must not touch
    # the small cube's result still being copied out), parameters and buffer
    # kinds; each result equals the same filter on the device, bit for bit
    jobs = [((24, 40, 64), 1.3, 1 / 8, 7, "rational", True),
            ((16, 33, 96), 0.8, 1 / 16, 4, "exponential", True),
            ((40, 64, 128), 2.0, 1 / 8, 3, "rational", False),
            ((24, 40, 64), 1.1, 0.1, 1, "exponential", True),
            ((9, 20, 36), 1.5, 1 / 8, 5, "rational", True),
            ((8, 16, 32), 1.2, 1 / 8, 2, "rational", True),
            ((20, 40, 64), 0.9, 1 / 8, 6, "exponential", True)]
    hosts, refs = [], []
    for i, (shape, K, dt, n, cond, pinned) in enumerate(jobs):
        cube = synth.cutout(shape, 300 + i)
        refs.append(run(afd, ctx, cube, K, dt, n, cond))
        h_in = torch.from_numpy(cube.copy())
        h_out = torch.full(shape, float("nan"))
        if pinned:
            h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
        hosts.append((h_in, h_out))
    for (h_in, h_out), (shape, K, dt, n, cond, _) in zip(hosts, jobs):
        afd.afd_filter_host_async(ctx, h_in, h_out, K, dt, n, cond)
    afd.afd_sync(ctx)
    for i, ((h_in, h_out), ref) in enumerate(zip(hosts, refs)):
        assert np.array_equal(h_out.numpy().view(np.uint32), ref.view(np.uint32)), i


@pytest.mark.parametrize("n", [0, 1, 2, 5])
def test_out_of_place(afd, ctx, n):
    cube = synth.cube64()[:24].copy()
    ref = run(afd, ctx, cube, 1.0, 1 / 8, n, "rational")
    for kernel in ("simple", "stream"):
        afd.afd_set_kernel(ctx, kernel)
        src = torch.from_numpy(cube).cuda()
        dst = torch.full_like(src, float("nan"))
        afd.afd_filter_out(ctx, src, dst, 1.0, 1 / 8, n, "rational")
        afd.afd_sync(ctx)
        assert np.array_equal(src.cpu().numpy(), cube)
        assert np.array_equal(dst.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    afd.afd_set_kernel(ctx, "auto")


def test_bounded_wait_reports_timeout(afd, ctx):
    """A wait that can never complete gives up after its limit; afd_sync
    reports AFD_ETIMEOUT and the context keeps working."""
    afd.afd_selftest_wait(ctx, 50_000_000)   # 50 ms
    with pytest.raises(afd.AfdError) as ei:
        afd.afd_sync(ctx)
    assert ei.value.status == afd.AFD_ETIMEOUT
    afd.afd_sync(ctx)                        # error word cleared
    cube = synth.cube64()[:8].copy()
    got = run(afd, ctx, cube, 1.5, 1 / 16, 2, "exponential")
    ref = oracle.pm_filter(cube, 1.5, 1 / 16, 2, "exponential")
    assert np.abs(got - ref).max() <= tol(2)


def test_argument_errors(afd, ctx):
    t = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    bad = [dict(K=float("nan")), dict(K=-1.0), dict(dt=0.0), dict(dt=float("inf")),
           dict(n_iter=-1), dict(spacing=(1.0, 0.0, 1.0)), dict(spacing=(1.0, float("nan"), 1.0))]
    for kw in bad:
        args = dict(K=1.0, dt=0.1, n_iter=2, spacing=None)
        args.update(kw)
        with pytest.raises(afd.AfdError) as ei:
            afd.afd_filter(ctx, t, args["K"], args["dt"], args["n_iter"], "rational",
                           args["spacing"])
        assert ei.value.status == afd.AFD_EINVAL, kw
    # the streaming kernel refuses layouts it cannot stage
    afd.afd_set_kernel(ctx, "stream")
    odd = torch.zeros((4, 4, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(afd.AfdError) as ei:
        afd.afd_filter(ctx, odd, 1.0, 0.1, 1, "rational")
    assert ei.value.status == afd.AFD_EINVAL
    afd.afd_set_kernel(ctx, "auto")
    afd.afd_sync(ctx)


def test_injected_allocation_failure():
    """AFD_FAULT=alloc:2 fails the scratch allocation (host-side injection):
    afd_filter returns AFD_ENOMEM and the next call works."""
    code = r"""
import torch, numpy as np
from paper_1609_03782_gb300 import afd
c = afd.afd_create(0)
t = torch.ones((8, 8, 8), device="cuda")
try:
    afd.afd_filter(c, t, 1.0, 0.1, 2, "rational")
    print("NOERROR")
except afd.AfdError as e:
    print("STATUS", e.status)
afd.afd_filter(c, t, 1.0, 0.1, 2, "rational")
afd.afd_sync(c)
print("RECOVERED", float(t.sum()))
"""
    env = dict(os.environ, AFD_FAULT="alloc:2")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         timeout=300)
    assert "STATUS 2" in res.stdout, res.stdout + res.stderr
    assert "RECOVERED 512.0" in res.stdout, res.stdout + res.stderr
