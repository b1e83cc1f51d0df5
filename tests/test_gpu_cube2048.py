"""Full-size parity of the 2048 x 2048 x 256 cube (60 disks + 10 tails, 4 GiB
in float32): float32, and stored in float16 / bfloat16 / int16 with a
power-of-two scale, temporal depths 1 (the streaming pass), 2, 4 and 8, 30
rational iterations
(K = 1.0 sigma, dt = 1/8).

The FP64 oracle runs on one 256 x 256 x 256 subcube (the whole z range):
after n iterations a voxel depends only on voxels within n steps, so the
oracle on the subcube grown by n = 30 voxels in x and y is exact on the
subcube itself.

Bounds (the same reasoning as test_gpu_precision.py): float32 within
1e-4 sigma; a 2-byte run within the Lipschitz-amplified sum of its
roundings (max norm), and its faint-band (|I| < 3 sigma) rms within one
faint half-ulp per rounding.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_precision import half_ulp, lipschitz, pass_depths

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_IT, DT, COND = 30, 1.0 / 8, "rational"
SUB = (slice(0, 256), slice(896, 1152), slice(896, 1152))   # z, y, x


@pytest.fixture(scope="module")
def setup(afd):
    ctx = afd.afd_create(0)
    cube = synth.cube2048()
    d_in = torch.from_numpy(cube).cuda()
    sigma = afd.afd_noise_rms(ctx, d_in)
    K = float(np.float32(1.0 * sigma))
    grown = np.ascontiguousarray(cube[:, 896 - N_IT:1152 + N_IT, 896 - N_IT:1152 + N_IT])
    ref = oracle.pm_filter(grown, K, DT, N_IT, COND)[:, N_IT:-N_IT, N_IT:-N_IT]
    yield ctx, cube, d_in, sigma, K, ref
    ctx.close()


def test_float32(afd, setup):
    ctx, cube, d_in, sigma, K, ref = setup
    out = torch.empty_like(d_in)
    afd.afd_filter_out(ctx, d_in, out, K, DT, N_IT, COND)
    afd.afd_sync(ctx)
    got = out[SUB].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-4 * sigma


@pytest.mark.parametrize("storage,T", [("f16", 1), ("f16", 2), ("f16", 4), ("f16", 8),
                                       ("bf16", 1), ("bf16", 2), ("bf16", 4), ("bf16", 8),
                                       ("i16", 1), ("i16", 4)])
def test_two_byte_storage(afd, setup, storage, T):
    ctx, cube, d_in, sigma, K, ref = setup
    dt_ = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}[storage]
    scale = oracle.pow2_scale(sigma)
    q = torch.empty(cube.shape, dtype=dt_, device="cuda")
    afd.afd_quantize(ctx, d_in, q, storage, scale)
    r = torch.empty_like(q)
    afd.afd_filter_ex(ctx, q, r, storage, scale, K, DT, N_IT, COND, None, T)
    back = torch.empty(cube.shape, dtype=torch.float32, device="cuda")
    afd.afd_dequantize(ctx, r, back, storage, scale)
    afd.afd_sync(ctx)
    got = back[SUB].cpu().numpy()
    del q, r, back
    err = np.abs(got - ref)
    L = lipschitz(COND, DT)
    done, amp = 0, L ** N_IT
    for d in pass_depths(N_IT, T):
        done += d
        amp += L ** (N_IT - done)
    h = half_ulp(storage, float(np.abs(cube).max()), scale)
    assert err.max() <= amp * h + 1e-4 * sigma, (err.max(), amp * h)
    faint = np.abs(ref) < 3 * sigma
    rounds = len(pass_depths(N_IT, T)) + 1
    faint_rms = float(np.sqrt(np.mean(err[faint] ** 2)))
    assert faint_rms <= rounds * half_ulp(storage, 3 * sigma, scale) + 1e-4 * sigma, faint_rms
