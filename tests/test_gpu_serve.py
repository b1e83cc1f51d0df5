"""GPU tests of the re-filter service (continuous batching at iteration
granularity over resident cubes).

* Requests with different cubes, K, dt, iteration counts and conductances,
  some submitted while others are already running, each give the result the
  same request gives alone (afd_filter_ex, depth 1, on that cube): bit for
  bit, so mixing changes nothing.
* Admission is by memory: with a budget for one request's result + scratch,
  the next request waits in the queue until the first is released.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(afd):
    c = afd.afd_create(0)
    yield c
    c.close()


SHAPES = [(16, 40, 64), (9, 30, 45), (24, 64, 130), (5, 8, 8), (12, 33, 77)]


@pytest.fixture(scope="module", params=["wide", "64x32"])
def resident(afd, ctx, request):
    cubes = []
    b = afd.afd_batch_create(ctx, SHAPES, "f16", 1.0)
    afd.afd_batch_set_tiles(b, request.param)   # the service runs the batch's tile kind
    for i, s in enumerate(SHAPES):
        q = torch.empty(s, dtype=torch.float16, device="cuda")
        afd.afd_quantize(ctx, torch.from_numpy(synth.cutout(s, 90 + i)).cuda(), q, "f16", 1.0)
        afd.afd_batch_set(b, i, q)
        cubes.append(q)
    afd.afd_sync(ctx)
    yield b, cubes
    b.close()


def alone(afd, ctx, q, K, dt, n, cond):
    out = torch.empty_like(q)
    afd.afd_filter_ex(ctx, q, out, "f16", 1.0, K, dt, n, cond, None, 1)
    afd.afd_sync(ctx)
    return out


def drain(afd, srv, tickets, max_steps=100000):
    for _ in range(max_steps):
        afd.afd_serve_step(srv, wait=True)
        if all(afd.afd_serve_poll(srv, t)[0] == 2 for t in tickets):
            return
    raise AssertionError("service did not finish")


def test_mix_equals_alone(afd, ctx, resident):
    b, cubes = resident
    srv = afd.afd_serve_create(b, 1 << 30, 16)
    try:
        reqs = [(0, 1.3, 0.125, 5, "rational"), (2, 0.9, 0.0625, 9, "exponential"),
                (1, 2.0, 0.125, 1, "rational"), (4, 1.1, 0.1, 7, "exponential"),
                (0, 0.7, 0.125, 3, "exponential")]
        late = [(3, 1.5, 0.125, 4, "rational"), (2, 1.0, 0.125, 2, "rational"),
                (4, float("inf"), 0.125, 3, "rational")]
        tickets = [afd.afd_serve_submit(srv, *r) for r in reqs]
        for _ in range(3):            # some rounds run before the late arrivals
            afd.afd_serve_step(srv)
        tickets += [afd.afd_serve_submit(srv, *r) for r in late]
        drain(afd, srv, tickets)
        for t, (c, K, dt, n, cond) in zip(tickets, reqs + late):
            state, lat = afd.afd_serve_poll(srv, t)
            assert state == 2 and lat > 0
            got = afd.afd_serve_result(srv, t, torch.empty_like(cubes[c]))
            ref = alone(afd, ctx, cubes[c], K, dt, n, cond)
            assert torch.equal(got.view(torch.int16), ref.view(torch.int16)), (t, c, K, n, cond)
            afd.afd_serve_release(srv, t)
    finally:
        srv.close()


def test_admission_by_memory(afd, ctx, resident):
    b, cubes = resident
    # room for exactly one request on cube 2 (result + scratch, padded rows)
    px = (130 + 7) // 8 * 8
    one = 2 * ((px * 64 * 24 * 2 + 255) // 256 * 256)
    srv = afd.afd_serve_create(b, one, 8)
    try:
        t1 = afd.afd_serve_submit(srv, 2, 1.0, 0.125, 3, "rational")
        t2 = afd.afd_serve_submit(srv, 2, 1.2, 0.125, 2, "rational")
        active, queued = afd.afd_serve_step(srv)
        assert (active, queued) == (1, 1)
        assert afd.afd_serve_free_bytes(srv) == 0
        drain(afd, srv, [t1])
        active, queued = afd.afd_serve_step(srv)
        assert afd.afd_serve_poll(srv, t2)[0] == 0 and queued == 1   # still waiting
        with pytest.raises(afd.AfdError) as ei:
            afd.afd_serve_release(srv, t2)                           # not done
        assert ei.value.status == afd.AFD_EBUSY
        afd.afd_serve_release(srv, t1)
        assert afd.afd_serve_free_bytes(srv) == one
        drain(afd, srv, [t2])
        got = afd.afd_serve_result(srv, t2, torch.empty_like(cubes[2]))
        ref = alone(afd, ctx, cubes[2], 1.2, 0.125, 2, "rational")
        assert torch.equal(got.view(torch.int16), ref.view(torch.int16))
        afd.afd_serve_release(srv, t2)
        # a request that could never fit is refused at once
        small = afd.afd_serve_create(b, 1024, 2)
        try:
            with pytest.raises(afd.AfdError) as ei:
                afd.afd_serve_submit(small, 0, 1.0, 0.1, 1, "rational")
            assert ei.value.status == afd.AFD_ENOMEM
        finally:
            small.close()
        for bad in [dict(cube=9), dict(K=0.0), dict(n=0)]:
            a = dict(cube=0, K=1.0, n=2)
            a.update(bad)
            with pytest.raises(afd.AfdError) as ei:
                afd.afd_serve_submit(srv, a["cube"], a["K"], 0.1, a["n"], "rational")
            assert ei.value.status == afd.AFD_EINVAL
    finally:
        srv.close()


def test_request_timestamps_are_ordered(afd, ctx, resident):
    b, cubes = resident
    srv = afd.afd_serve_create(b, 1 << 30, 8)
    try:
        t = afd.afd_serve_submit(srv, 2, 1.0, 0.125, 9, "rational")
        sub, adm, first, done = afd.afd_serve_times(srv, t)
        assert sub > 0 and adm == -1.0 and first == -1.0 and done == -1.0
        drain(afd, srv, [t])
        sub, adm, first, done = afd.afd_serve_times(srv, t)
        assert 0 < sub <= adm <= first <= done, (sub, adm, first, done)
        st, lat = afd.afd_serve_poll(srv, t)
        assert st == 2 and abs(lat - (done - sub)) < 1e-9
        afd.afd_serve_release(srv, t)
        with pytest.raises(afd.AfdError):
            afd.afd_serve_times(srv, t)          # released: unknown ticket
    finally:
        srv.close()
