"""GPU parity of the F / F_M diagnostics (Sec. 4, eqs. F_equa, Sequa,
Mfequa; Sec. 5, eq. sums_equa) against the FP64 oracle.

Mask decisions are integers: with the same rms on both sides the counts
N_o, N_f must match exactly (the library rounds each threshold up to the
next float, which decides every float voxel as the exact comparison does).
The sums are float32 partial sums of four values added to float-float
accumulators: each term is rounded at most three times in float32, so
|S_gpu - S_oracle| <= 4 u sum |terms| with u = 2^-24.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


def check(got, ref, io, im, roi):
    assert got["N_o"] == ref["N_o"] and got["N_f"] == ref["N_f"]
    x0, x1, y0, y1, z0, z1 = roi
    a_o = float(np.abs(io[z0:z1, y0:y1, x0:x1].astype(np.float64)).sum())
    for key in ("S_of", "S_oo"):
        assert abs(got[key] - ref[key]) <= 4 * U * a_o + 1e-300, key
    if im is not None:
        a_m = float(np.abs(im[z0:z1, y0:y1, x0:x1].astype(np.float64)).sum())
        for key in ("S_mf", "S_m"):
            assert abs(got[key] - ref[key]) <= 4 * U * a_m + 1e-300, key
        assert got["F_M"] == pytest.approx(ref["F_M"], rel=1e-5, nan_ok=True)
    else:
        assert math.isnan(got["F_M"])
    assert got["F"] == pytest.approx(ref["F"], rel=1e-5, nan_ok=True)  # NaN: S_oo = 0
    assert got["sigma_F"] == pytest.approx(ref["sigma_F"], rel=1e-5, nan_ok=True)


def test_model_b_after_intensity_filter(afd, ctx):
    cube, model, roi = synth.model_b()
    d_o = torch.from_numpy(cube).cuda()
    d_m = torch.from_numpy(model).cuda()
    d_f = torch.empty_like(d_o)
    rms = afd.afd_noise_rms(ctx, d_o)
    afd.afd_filter_intensity(ctx, d_o, d_f, 1.0, rms, 0.0325, 20, (4.0, 5.0, 4.0))
    afd.afd_sync(ctx)
    filt = d_f.cpu().numpy()
    rms_o, rms_f = oracle.noise_rms(cube), oracle.noise_rms(filt)
    for box in (roi, (0, 104, 0, 104, 0, 64), (3, 4, 50, 51, 30, 31), (1, 26, 7, 9, 0, 64),
                (5, 101, 2, 103, 1, 63)):
        got = afd.afd_f_diagnostic(ctx, d_o, d_f, d_m, roi=box, rms_o=rms_o, rms_f=rms_f)
        ref = oracle.f_diagnostic(cube, filt, model, roi=box, rms_o=rms_o, rms_f=rms_f)
        check(got, ref, cube, model, box)
    # without the model; another threshold and beam
    got = afd.afd_f_diagnostic(ctx, d_o, d_f, roi=roi, rms_o=rms_o, rms_f=rms_f, nsig=2.5,
                               beam=3.0)
    ref = oracle.f_diagnostic(cube, filt, roi=roi, rms_o=rms_o, rms_f=rms_f, nsig=2.5, beam=3.0)
    check(got, ref, cube, None, roi)
    # estimated noise levels: the GPU estimate against the FP64 one
    got = afd.afd_f_diagnostic(ctx, d_o, d_f, d_m, roi=roi)
    assert got["rms_o"] == pytest.approx(rms_o, rel=1e-6)
    assert got["rms_f"] == pytest.approx(rms_f, rel=1e-6)
    ref = oracle.f_diagnostic(cube, filt, model, roi=roi)
    assert got["F"] == pytest.approx(ref["F"], rel=1e-3)


def test_thresholds_are_exact(afd, ctx):
    # rms 1: threshold 3 exactly; rms 0.1: 3 * 0.1 = 0.30000000000000004 in
    # double, above float32(0.3) = 0.300000011920928955..., which is in
    below3 = np.nextafter(np.float32(3.0), np.float32(0.0))
    io = np.zeros((3, 5, 37), np.float32)
    io[0, 0, :6] = [3.0, below3, 3.5, -3.0, 2.0, 3.0]
    iff = np.zeros_like(io)
    iff[1, 2, 30:36] = [np.float32(0.3), np.nextafter(np.float32(0.3), np.float32(0)), 0.31,
                        0.29, 1.0, np.float32(0.3)]
    d_o, d_f = torch.from_numpy(io).cuda(), torch.from_numpy(iff).cuda()
    got = afd.afd_f_diagnostic(ctx, d_o, d_f, rms_o=1.0, rms_f=0.1)
    ref = oracle.f_diagnostic(io, iff, rms_o=1.0, rms_f=0.1)
    assert (got["N_o"], got["N_f"]) == (ref["N_o"], ref["N_f"]) == (3, 4)
    assert got["S_oo"] == ref["S_oo"] == 9.5


def test_bad_arguments(afd, ctx):
    a = torch.zeros((4, 5, 6), device="cuda")
    for kw in (dict(roi=(0, 0, 0, 5, 0, 4)), dict(roi=(0, 7, 0, 5, 0, 4)),
               dict(roi=(-1, 6, 0, 5, 0, 4)), dict(nsig=0.0), dict(beam=0.5),
               dict(rms_o=float("nan"))):
        with pytest.raises(afd.AfdError):
            afd.afd_f_diagnostic(ctx, a, a, rms_o=kw.pop("rms_o", 1.0), rms_f=1.0, **kw)


def test_full_size_cube512(afd, ctx):
    """The benchmark's cube after 50 rational iterations: the whole cube and a
    ragged ROI, every voxel summed by the oracle."""
    cube = synth.cube512()
    d_o = torch.from_numpy(cube).cuda()
    d_f = torch.empty_like(d_o)
    afd.afd_filter_rel(ctx, d_o, d_f, 1.0, 1 / 8, 50, "rational")
    afd.afd_sync(ctx)
    filt = d_f.cpu().numpy()
    rms_o, rms_f = oracle.noise_rms(cube), oracle.noise_rms(filt)
    for box in ((0, 512, 0, 512, 0, 256), (37, 499, 11, 301, 5, 250)):
        got = afd.afd_f_diagnostic(ctx, d_o, d_f, roi=box, rms_o=rms_o, rms_f=rms_f)
        ref = oracle.f_diagnostic(cube, filt, roi=box, rms_o=rms_o, rms_f=rms_f)
        check(got, ref, cube, None, box)
