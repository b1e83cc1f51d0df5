"""Full-size parity of the batching and serving workloads.

* 300 galaxy cutouts (nx, ny ~ U{32..256}, nz ~ U{32..128}, one disk each,
  seed 0), K_i = 1.5 sigma_i from the GPU noise estimate, 20 rational
  iterations, float32 and float16-stored, in one graph launch: every cube is
  bit-identical to the same filter on that cube alone (compared on the
  device), its K matches the FP64 noise estimate, and ten cubes are checked
  against the FP64 oracle.
* 64 resident float16 cubes (21 x 128^3, 21 x 256^3, 22 x 512x512x128): a mix
  of re-filter requests, some submitted while others run, each bit-identical
  to the same request run alone.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = 1.0 / 8


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_300_cutouts(afd, ctx, storage):
    shapes = synth.cutout_shapes(0, 300)
    cubes = synth.cutouts(0, 300)
    tdt = torch.float32 if storage == "f32" else torch.float16
    b = afd.afd_batch_create(ctx, shapes, storage, 1.0)
    try:
        dev = []
        for i, c in enumerate(cubes):
            t = torch.from_numpy(c).cuda()
            if storage == "f16":
                q = torch.empty(c.shape, dtype=torch.float16, device="cuda")
                afd.afd_quantize(ctx, t, q, "f16", 1.0)
                t = q
            afd.afd_batch_set(b, i, t)
            dev.append(t)
        afd.afd_batch_filter(b, [-1.5] * len(shapes), DT, 20, "rational")
        Kused = afd.afd_batch_k(b)
        mism = []
        for i in range(len(shapes)):
            got = afd.afd_batch_get(b, i, torch.empty(shapes[i], dtype=tdt, device="cuda"))
            ref = torch.empty_like(dev[i])
            if storage == "f32":
                afd.afd_filter_out(ctx, dev[i], ref, float(Kused[i]), DT, 20, "rational")
            else:
                afd.afd_filter_ex(ctx, dev[i], ref, "f16", 1.0, float(Kused[i]), DT, 20,
                                  "rational", None, 1)
            same = torch.equal(got.view(torch.int16 if storage == "f16" else torch.int32),
                               ref.view(torch.int16 if storage == "f16" else torch.int32))
            if not same:
                mism.append(i)
        afd.afd_sync(ctx)
        assert not mism, mism
        if storage == "f32":
            # K from the GPU noise estimate against the FP64 one, every cube
            for i in range(0, 300, 7):
                sig = oracle.noise_rms(cubes[i])
                assert abs(Kused[i] / 1.5 - sig) <= 1e-6 * sig, i
            # ten cubes against the FP64 oracle (the smallest of ten strata)
            order = np.argsort([a * bb * cc for a, bb, cc in shapes])
            for i in order[::30][:10]:
                got = afd.afd_batch_get(b, int(i), torch.empty(shapes[i], device="cuda"))
                o = oracle.pm_filter(cubes[i], float(Kused[i]), DT, 20, "rational")
                assert np.abs(got.cpu().numpy() - o).max() <= 1e-4, int(i)
    finally:
        b.close()


def test_serving_64_resident(afd, ctx):
    shapes = synth.serving_shapes()
    b = afd.afd_batch_create(ctx, shapes, "f16", 1.0)
    srv = None
    try:
        qs, sig = [], []
        for i, s in enumerate(shapes):
            t = torch.from_numpy(synth.serving_cube(i)).cuda()
            sig.append(afd.afd_noise_rms(ctx, t))
            q = torch.empty(s, dtype=torch.float16, device="cuda")
            afd.afd_quantize(ctx, t, q, "f16", 1.0)
            afd.afd_batch_set(b, i, q)
            qs.append(q)
            del t
        srv = afd.afd_serve_create(b, 16 << 30, 128)
        rng = np.random.default_rng(5)
        reqs = [(int(rng.integers(0, 64)), float(rng.uniform(0.5, 3.0)), int(rng.integers(1, 51)))
                for _ in range(24)]
        tickets = []
        for k, (c, ks, n) in enumerate(reqs):
            tickets.append(afd.afd_serve_submit(srv, c, ks * sig[c], DT, n, "rational"))
            if k % 5 == 4:
                for _ in range(3):          # rounds run while later requests arrive
                    afd.afd_serve_step(srv)
        for _ in range(100000):
            afd.afd_serve_step(srv, wait=True)
            if all(afd.afd_serve_poll(srv, t)[0] == 2 for t in tickets):
                break
        for t, (c, ks, n) in zip(tickets, reqs):
            assert afd.afd_serve_poll(srv, t)[0] == 2
            got = afd.afd_serve_result(srv, t, torch.empty_like(qs[c]))
            ref = torch.empty_like(qs[c])
            afd.afd_filter_ex(ctx, qs[c], ref, "f16", 1.0, ks * sig[c], DT, n, "rational",
                              None, 1)
            afd.afd_sync(ctx)
            assert torch.equal(got.view(torch.int16), ref.view(torch.int16)), (t, c, n)
            afd.afd_serve_release(srv, t)
    finally:
        if srv is not None:
            srv.close()
        b.close()
