"""One cube over several ranks: a z-slab decomposition with halo exchange.

An explicit nearest-neighbour iteration (Sec. 3.3) moves information one
plane per iteration.  A rank that owns planes [z0, z1) and holds `its` more
planes of each neighbour can therefore run `its` iterations on its own.  Its
own planes are then the whole cube's after those iterations, while the ghost
planes are spoiled (the rank treats the slab's ends as faces).  Each round:
1. exchange `its` edge planes with each neighbour (point-to-point send and
   receive into the rank's own buffer);
2. run `its` iterations;
3. repeat until n_iter iterations are done.
The cube's own z faces are the true zero-flux faces and get no ghosts.

The compute is a callable ``step(buf, its)`` that filters the contiguous
(planes, ny, nx) tensor ``buf`` in place with zero-flux faces:
``gpu_step`` runs the library's kernels on a CUDA tensor (NCCL moves the
planes); tests pass a CPU stand-in (gloo moves the planes).  Nothing here
does arithmetic on the data.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def slab_bounds(nz: int, world: int, rank: int):
    """Planes [z0, z1) of rank `rank` when nz planes are split as evenly as
    possible over `world` ranks (the first nz % world ranks get one more)."""
    if not (0 <= rank < world) or nz < world:
        raise ValueError("need 0 <= rank < world <= nz")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def filter_slab(own: torch.Tensor, z0: int, z1: int, nz: int, n_iter: int, halo: int, step,
                group=None) -> torch.Tensor:
    """n_iter iterations of the whole cube, computed by the ranks of `group`
    (default: the world), each owning planes [z0, z1) of the cube in the
    same order as the ranks.  own: this rank's (z1 - z0, ny, nx) planes.
    halo: iterations per round, at most the smallest slab of the group (a
    neighbour's ghost planes are its edge planes).  Returns this rank's
    planes after n_iter iterations (a new tensor, on own's device, in own's
    dtype).

    Every rank of the group must call this with the same nz, n_iter and halo.
    Argument errors are raised on every rank alike, before any exchange.
    """
    S = z1 - z0
    # Every rank must reach the same verdict before any exchange: a rank that
    # raised alone would leave its neighbours waiting in their sends and
    # receives.  So each rank checks its own arguments, and one small MIN
    # reduction over the group (this call's only collective, once per call,
    # not on the data path) gives every rank the group's smallest slab and
    # whether all ranks' own checks passed.
    local_ok = own.dim() == 3 and own.shape[0] == S and 0 <= z0 < z1 <= nz
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        v = torch.tensor([S if local_ok else 0, 1 if local_ok else 0, halo, -halo, n_iter,
                          -n_iter], dtype=torch.int64, device=own.device)
        dist.all_reduce(v, op=dist.ReduceOp.MIN, group=group)
        min_slab, all_ok = int(v[0]), bool(v[1])
        same = int(v[2]) == -int(v[3]) == halo and int(v[4]) == -int(v[5]) == n_iter
    else:
        min_slab, all_ok, same = S, local_ok, True
    if not all_ok:
        raise ValueError("own must hold planes [z0, z1) of the cube (on every rank)")
    if not same:
        raise ValueError("every rank must pass the same halo and n_iter")
    if n_iter < 0:
        raise ValueError("n_iter must be >= 0")
    if halo < 1 or (n_iter > 0 and halo > min_slab):
        raise ValueError("halo must be >= 1 and at most the smallest slab's planes (%d)"
                         % min_slab)
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    below, above = z0 > 0, z1 < nz       # neighbours: rank - 1 and rank + 1
    buf = own.new_zeros((S + 2 * halo,) + tuple(own.shape[1:]))
    buf[halo:halo + S] = own
    done = 0
    while done < n_iter:
        its = min(halo, n_iter - done)
        ops = []
        if below:
            ops.append(dist.P2POp(dist.isend, buf[halo:halo + its].contiguous(),
                                  _peer(rank - 1, group), group))
            ops.append(dist.P2POp(dist.irecv, buf[halo - its:halo], _peer(rank - 1, group),
                                  group))
        if above:
            ops.append(dist.P2POp(dist.isend, buf[halo + S - its:halo + S].contiguous(),
                                  _peer(rank + 1, group), group))
            ops.append(dist.P2POp(dist.irecv, buf[halo + S:halo + S + its],
                                  _peer(rank + 1, group), group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        lo = halo - (its if below else 0)
        hi = halo + S + (its if above else 0)
        step(buf[lo:hi], its)
        done += its
    return buf[halo:halo + S].clone()


def _peer(group_rank: int, group):
    """The global rank of `group_rank` in `group` (the world: itself)."""
    if group is None:
        return group_rank
    return dist.get_global_rank(group, group_rank)


def gpu_step(ctx, K: float, dt: float, conductance: str = "rational", spacing=None):
    """The library's filter as a slab step: afd_filter in place on a float32
    CUDA slab (stream-ordered on the current stream)."""
    from . import afd

    def step(buf: torch.Tensor, its: int) -> None:
        afd.afd_filter(ctx, buf, K, dt, its, conductance, spacing)

    return step
