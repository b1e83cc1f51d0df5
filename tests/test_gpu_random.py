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
