"""The z-slab decomposition with halo exchange (slabs.py) on gloo ranks on
the CPU.  The compute step is the FP64 oracle (the slab path's arithmetic is
the library's kernels on a GPU; here only the plane bookkeeping and the
exchange are under test).  The whole cube filtered by the oracle in one
piece is the reference: an explicit nearest-neighbour iteration moves
information one plane per iteration, so every rank's planes must equal it
bit for bit (FP64, the same operations in the same order)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1609_03782_gb300 import slabs

K, DT, COND, SP = 1.1, 0.12, "rational", (1.0, 1.5, 0.75)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _cube(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) * 2.0).astype(np.float32)


def oracle_step(buf: torch.Tensor, its: int) -> None:
    """The oracle as a slab step: its iterations on the slab, zero-flux faces."""
    buf.copy_(torch.from_numpy(oracle.pm_filter(buf.numpy(), K, DT, its, COND, spacing=SP)))


def _worker(rank, world, port, shape, seed, n_iter, halo, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cube = _cube(shape, seed)
        nz = shape[0]
        z0, z1 = slabs.slab_bounds(nz, world, rank)
        own = torch.from_numpy(cube[z0:z1].astype(np.float64))
        res = slabs.filter_slab(own, z0, z1, nz, n_iter, halo, oracle_step)
        out.put((rank, z0, z1, res.numpy()))
    finally:
        dist.destroy_process_group()


def _run(world, shape, seed, n_iter, halo):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shape, seed, n_iter, halo, q))
             for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([part for _, _, _, part in parts])
    assert [(z0, z1) for _, z0, z1, _ in parts] == \
        [slabs.slab_bounds(shape[0], world, r) for r in range(world)]
    return got


@pytest.mark.parametrize("world,shape,n_iter,halo", [
    (2, (12, 9, 10), 7, 3),    # rounds of 3, 3, 1
    (3, (17, 6, 8), 9, 4),     # uneven slabs (6, 6, 5), rounds of 4, 4, 1
    (2, (8, 5, 7), 4, 4),      # one round, halo = the slab
    (4, (9, 5, 6), 5, 1),      # four ranks, one ghost plane per round, slabs of 3, 2, 2, 2
])
def test_slab_ranks_equal_the_whole_cube(world, shape, n_iter, halo):
    got = _run(world, shape, 5, n_iter, halo)
    ref = oracle.pm_filter(_cube(shape, 5), K, DT, n_iter, COND, spacing=SP)
    assert np.array_equal(got, ref)


def _worker_bad_halo(rank, world, port, shape, halo, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz = shape[0]
        z0, z1 = slabs.slab_bounds(nz, world, rank)
        own = torch.zeros((z1 - z0,) + tuple(shape[1:]), dtype=torch.float64)
        try:
            slabs.filter_slab(own, z0, z1, nz, 6, halo, oracle_step)
            out.put((rank, z1 - z0, "returned"))
        except ValueError as e:
            out.put((rank, z1 - z0, "ValueError: %s" % e))
    finally:
        dist.destroy_process_group()


def test_uneven_slabs_reject_a_halo_on_every_rank():
    # nz = 9 over 2 ranks gives slabs of 5 and 4 planes.  halo = 5 fits the
    # first rank's slab but not the second's: both ranks must raise (and
    # neither may wait for the other in an exchange).
    world, shape = 2, (9, 4, 6)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_bad_halo, args=(r, world, port, shape, 5, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5, 4]
    assert all(r[2].startswith("ValueError") and "smallest slab" in r[2] for r in res), res


def test_too_few_ghosts_would_differ():
    # the check above has teeth: with halo planes but more iterations than
    # ghosts per round, the slab edges see the artificial faces
    cube = _cube((12, 9, 10), 5).astype(np.float64)
    ref = oracle.pm_filter(cube, K, DT, 4, COND, spacing=SP)
    lo = oracle.pm_filter(cube[:6 + 2], K, DT, 4, COND, spacing=SP)[:6]
    assert not np.array_equal(lo, ref[:6])
    lo = oracle.pm_filter(cube[:6 + 4], K, DT, 4, COND, spacing=SP)[:6]
    assert np.array_equal(lo, ref[:6])


def test_slab_bounds_cover_the_cube():
    for nz, world in [(10, 3), (7, 7), (256, 8), (5, 2)]:
        b = [slabs.slab_bounds(nz, world, r) for r in range(world)]
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
        assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 1
    with pytest.raises(ValueError):
        slabs.slab_bounds(3, 4, 0)


def test_single_rank_and_argument_checks():
    cube = _cube((6, 4, 5), 2).astype(np.float64)
    own = torch.from_numpy(cube.copy())
    got = slabs.filter_slab(own, 0, 6, 6, 5, 2, oracle_step)  # no neighbours: no exchange
    assert np.array_equal(got.numpy(), oracle.pm_filter(cube, K, DT, 5, COND, spacing=SP))
    assert torch.equal(slabs.filter_slab(own, 0, 6, 6, 0, 9, oracle_step), own)  # n = 0
    with pytest.raises(ValueError):
        slabs.filter_slab(own, 0, 6, 6, 5, 7, oracle_step)   # halo > slab
    with pytest.raises(ValueError):
        slabs.filter_slab(own, 1, 6, 6, 5, 2, oracle_step)   # wrong plane count
