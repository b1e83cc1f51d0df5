"""Seeded random parameter draws against the FP64 oracle (GPU).

Shapes from 1 to 70 voxels per axis (widths that are and are not multiples
of 4, so both kernel families run), K, dt, spacing, conductance and the
iteration count drawn from a fixed seed.  Both kernels must match the oracle
within the float32 tolerance and each other bit for bit."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def cases(count=24, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = int(rng.integers(1, 18)) * 4 if i % 2 == 0 else int(rng.integers(1, 71))
        shape = (int(rng.integers(1, 40)), int(rng.integers(1, 71)), nx)
        out.append(dict(shape=shape, K=float(rng.uniform(0.3, 3.0)),
                        dt=float(rng.uniform(0.02, 0.16)), n=int(rng.integers(1, 13)),
                        cond=str(rng.choice(["rational", "exponential"])),
                        spacing=tuple(float(v) for v in rng.uniform(0.7, 2.0, 3)),
                        seed=int(rng.integers(0, 10 ** 6))))
    return out


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", cases(), ids=lambda c: "x".join(map(str, c["shape"])))
def test_random_case(afd, ctx, case):
    rng = np.random.default_rng(case["seed"])
    cube = (rng.standard_normal(case["shape"]) * 2.0).astype(np.float32)
    ref = oracle.pm_filter(cube, case["K"], case["dt"], case["n"], case["cond"],
                           spacing=case["spacing"])
    outs = []
    for kernel in ("auto", "simple"):
        afd.afd_set_kernel(ctx, kernel)
        t = torch.from_numpy(cube).cuda()
        afd.afd_filter(ctx, t, case["K"], case["dt"], case["n"], case["cond"], case["spacing"])
        afd.afd_sync(ctx)
        outs.append(t.cpu().numpy())
    afd.afd_set_kernel(ctx, "auto")
    scale = max(1.0, float(np.abs(cube).max()))
    tol = min(1e-5 * case["n"], 1e-4) * scale
    assert np.abs(outs[0] - ref).max() <= tol
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


def ex_cases(count=16, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = int(rng.integers(1, 20)) * 8 if i % 4 else int(rng.integers(1, 17)) * 4
        shape = (int(rng.integers(1, 30)), int(rng.integers(1, 60)), nx)
        out.append(dict(shape=shape, storage=str(rng.choice(["f32", "f16", "bf16", "i16"])),
                        scale=float(2.0 ** int(rng.integers(-1, 2))),
                        T=int(rng.choice([1, 2, 4, 8])), n=int(rng.integers(1, 18)),
                        K=float(rng.uniform(0.3, 3.0)), dt=float(rng.uniform(0.02, 0.16)),
                        cond=str(rng.choice(["rational", "exponential"])),
                        spacing=tuple(float(v) for v in rng.uniform(0.7, 2.0, 3)),
                        seed=int(rng.integers(0, 10 ** 6))))
    return out


def depth_schedule(n, T):
    """afd_filter_ex's passes: n // T of depth T, then the rest as depths 4, 2, 1
    (each at most T)."""
    passes = [T] * (n // T)
    left = n - T * (n // T)
    for d in (4, 2, 1):
        while d <= T and left >= d:
            passes.append(d)
            left -= d
    return passes


TDT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
RAW = {"f32": torch.int32, "f16": torch.int16, "bf16": torch.int16, "i16": torch.int16}


@pytest.mark.parametrize("case", ex_cases(), ids=lambda c: "%s_T%d_n%d_%s" % (
    c["storage"], c["T"], c["n"], "x".join(map(str, c["shape"]))))
def test_random_storage_depth_case(afd, ctx, case):
    """afd_filter_ex under its three routes, bit for bit, and against its
    definition composed from other entry points: for every pass of depth d,
    dequantise (afd_dequantize), d float32 iterations (afd_filter_out),
    quantise (afd_quantize)."""
    st, scale, T, n = case["storage"], case["scale"], case["T"], case["n"]
    rng = np.random.default_rng(case["seed"])
    cube = torch.from_numpy((rng.standard_normal(case["shape"]) * 2.0).astype(np.float32)).cuda()
    args = (case["K"], case["dt"])
    if st == "f32":
        q = cube.clone()
    else:
        q = torch.empty(case["shape"], dtype=TDT[st], device="cuda")
        afd.afd_quantize(ctx, cube, q, st, scale)
    outs = []
    for kern in ("auto", "two_stage", "stream"):
        afd.afd_set_kernel(ctx, kern)
        o = torch.empty_like(q)
        afd.afd_filter_ex(ctx, q, o, st, scale, *args, n, case["cond"], case["spacing"], T)
        afd.afd_sync(ctx)
        outs.append(o.view(RAW[st]).cpu())
    afd.afd_set_kernel(ctx, "auto")
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    # the definition, pass by pass
    ref = q.clone()
    x = torch.empty(case["shape"], dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for d in depth_schedule(n, T):
        if st == "f32":
            x.copy_(ref)
        else:
            afd.afd_dequantize(ctx, ref, x, st, scale)
        afd.afd_filter_out(ctx, x, y, *args, d, case["cond"], case["spacing"])
        if st == "f32":
            ref.copy_(y)
        else:
            afd.afd_quantize(ctx, y, ref, st, scale)
    afd.afd_sync(ctx)
    assert torch.equal(outs[0], ref.view(RAW[st]).cpu())
