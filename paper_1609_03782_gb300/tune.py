"""Autotuner for the launch parameters that do not change results.

Three knobs are tuned by timing, never by changing arithmetic (every kernel
variant is bit-identical):

* the z-chunk of the streaming kernels (planes per tile), for a single cube
  (``afd_set_stream_zchunk``) or a resident batch (``afd_batch_set_zchunk``);
* the tile shape of a resident batch (``afd_batch_set_tiles``): 64 x 32
  tiles of 4 x 2 voxels per thread, or per-cube tiles of 8 x 2 voxels per
  thread (tile columns of at most 128 voxels, as tall as the threads cover);
* the temporal-blocking depth of ``afd_filter_ex`` (1, 2, 4 or 8; at least
  a caller's minimum, which bounds the roundings to 2-byte storage) and the
  route its deeper passes take (``afd_set_kernel``: chains of one-iteration
  launches or of the two-stage kernel).

Results are cached in a JSON file keyed by what the choice depends on: the
cube shape rounded to powers of two (or the batch's voxel count and cube
count), the storage format, the conductance and the iteration count.
``timer`` is injectable so that the host logic can be tested without a GPU.
"""
from __future__ import annotations

import json
import math
import os
import threading

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "afd_tune.json")
ZCHUNKS = (0, 8, 16, 32, 64)
DEPTHS = (1, 2, 4, 8)
# afd_filter_ex's routes for passes of depth 2 or more (afd_set_kernel names)
ROUTES = ("auto", "two_stage")
TILES = ("wide", "64x32")
BATCH_ZCHUNKS = (64, 32, 16)


def _bucket(v: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, int(v))))))


def shape_key(kind: str, shape, storage: str, cond: str, n_iter: int) -> str:
    nz, ny, nx = (int(v) for v in shape)
    return "%s|%dx%dx%d|%s|%s|n%d" % (kind, _bucket(nx), _bucket(ny), _bucket(nz), storage,
                                      cond, n_iter)


def batch_key(shapes, storage: str, cond: str, n_iter: int) -> str:
    vox = sum(int(a) * int(b) * int(c) for a, b, c in shapes)
    return "batch|%d cubes|%d vox|%s|%s|n%d" % (_bucket(len(shapes)), _bucket(vox), storage,
                                                 cond, n_iter)


class Tuner:
    """Times candidates, keeps the fastest, remembers it."""

    def __init__(self, cache_path: str | None = DEFAULT_CACHE, timer=None, reps: int = 3):
        self.cache_path = cache_path
        self.reps = reps
        self.timer = timer or _cuda_timer
        self._lock = threading.Lock()
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as fh:
                    self.cache = json.load(fh)
            except (OSError, ValueError):
                self.cache = {}

    def _save(self):
        if not self.cache_path:
            return
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(self.cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def pick(self, key: str, candidates, run):
        """Return the candidate with the smallest time of run(candidate);
        cached per key.  `run` executes one call with that candidate."""
        candidates = [tuple(c) if isinstance(c, list) else c for c in candidates]
        with self._lock:
            if key in self.cache:
                ch = self.cache[key]["choice"]
                ch = tuple(ch) if isinstance(ch, list) else ch
                if ch in candidates:
                    return ch
        times = {}
        for c in candidates:
            times[c] = self.timer(lambda: run(c), self.reps)
        best = min(times, key=lambda c: times[c])
        with self._lock:
            self.cache[key] = {"choice": best, "ms": {str(c): t for c, t in times.items()}}
            self._save()
        return best

    # -- the library's knobs ------------------------------------------------
    def tune_batch(self, afd, batch, K, dt, n_iter, conductance="rational", spacing=None,
                   candidates=None):
        """Choose and apply the batch's (tile kind, z-chunk); returns it."""
        key = batch_key(batch.shapes, batch.storage, conductance, n_iter)
        if candidates is None:
            candidates = [(t, z) for t in TILES for z in BATCH_ZCHUNKS]

        def apply(c):
            afd.afd_batch_set_tiles(batch, c[0])
            afd.afd_batch_set_zchunk(batch, c[1])

        def run(c):
            apply(c)
            afd.afd_batch_filter(batch, K, dt, n_iter, conductance, spacing)

        best = self.pick(key, candidates, run)
        apply(best)
        return best

    def tune_filter_ex(self, afd, ctx, src, dst, storage, scale, K, dt, n_iter,
                       conductance="rational", spacing=None, depths=DEPTHS,
                       zchunks=(0, 16, 32), routes=ROUTES, min_depth=1):
        """Choose (t_block, z-chunk, route) for afd_filter_ex on this shape:
        the fastest with t_block >= min_depth.  A caller that wants at most
        n_iter / d roundings to the storage format (the error of 2-byte
        storage grows with them) sets min_depth = d.  `routes` are
        afd_set_kernel names tried for passes of depth 2 or more (one-
        iteration chains, two-stage chains); depth 1 takes the first.  The
        z-chunk and route are left applied to the context; t_block is
        returned."""
        key = "%s|min depth %d" % (shape_key("filter_ex", src.shape, storage, conductance,
                                             n_iter), min_depth)
        cands = [(t, z, r) for t in depths if t >= min_depth for z in zchunks
                 for r in (routes if t >= 2 else routes[:1])]
        if not cands:
            raise ValueError("no depth in %r is at least %d" % (tuple(depths), min_depth))

        def apply(c):
            afd.afd_set_stream_zchunk(ctx, c[1])
            afd.afd_set_kernel(ctx, c[2])

        def run(c):
            apply(c)
            afd.afd_filter_ex(ctx, src, dst, storage, scale, K, dt, n_iter, conductance,
                              spacing, c[0])

        best = self.pick(key, cands, run)
        apply(best)
        return best[0]


def _cuda_timer(fn, reps):
    import torch
    fn()  # warm-up (and graph capture, first-use set-up)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps
