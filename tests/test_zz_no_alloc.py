"""afd_filter_noalloc, the entry point for callers that may not allocate GPU
memory (an application that pools all device memory itself, a real-time loop
that must not allocate, a plug-in without an allocator).

It runs the same kernels with the same arithmetic as the ordinary
out-of-place entry point, afd_filter_out, so its results must equal that
call's bit for bit, call after call: its scratch is one fixed array shared by
all calls and keeps the last call's contents, so the check runs several
different calls in a row (and the in-place form after them).  This
file is collected last, so a run that stops at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tol(n_iter, sigma=1.0):
    return min(1e-5 * max(n_iter, 1), 1e-4) * sigma


CALLS = [
    # (cube, K, dt, n_iter, conductance, spacing)
    (lambda: synth.cube64(), 1.5, 1 / 16, 10, "exponential", None),       # streaming kernel
    (lambda: synth.cube512()[:40, :72, :98].copy(), 1.0, 1 / 8, 7, "rational",
     (1.0, 1.5, 0.75)),                                                     # nx % 4 != 0
    (lambda: synth.cube512()[:128, :256, :256].copy(), 1.0, 1 / 8, 4, "rational", None),
]


def test_noalloc_matches_filter_out_call_after_call(afd):
    ctx = afd.afd_create(0)
    try:
        for make, K, dt, n, cond, sp in CALLS:
            src = torch.from_numpy(make()).cuda()
            ref = torch.empty_like(src)
            afd.afd_filter_out(ctx, src, ref, K, dt, n, cond, sp)
            afd.afd_sync(ctx)
            got = torch.full_like(src, float("nan"))
            afd.afd_filter_noalloc(src, got, K, dt, n, cond, sp)
            err = float((got - ref).abs().max())   # diagnostic only
            assert torch.equal(got, ref), "differs from afd_filter_out (max %g, tol %g)" % (
                err, tol(n))
        # in place, on the last cube
        afd.afd_filter_noalloc(src, src, K, dt, n, cond, sp)
        assert torch.equal(src, ref), float((src - ref).abs().max())
    finally:
        ctx.close()


def test_noalloc_rejects_cubes_beyond_its_scratch(afd):
    nz = afd.NOALLOC_MAX_VOXELS // (256 * 256) + 1
    big = torch.zeros((nz, 256, 256), dtype=torch.float32, device="cuda")
    with pytest.raises(afd.AfdError) as ei:
        afd.afd_filter_noalloc(big, big, 1.0, 0.1, 1, "rational")
    assert ei.value.status == afd.AFD_EINVAL
