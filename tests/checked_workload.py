"""A battery of small filter calls for the bounds-checked debug build.

Run as a script with the library chosen by AFD_LIB (the release libafd.so or
the checked libafd_check.so): every kernel family on ragged shapes, odd
widths, unaligned buffers and several z-chunks.  Saves each step's result and,
for the checked build, the bounds-check record after the step, to the .npz
file named on the command line.  test_gpu_checked.py compares the two builds.
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1609_03782_gb300 import afd  # noqa: E402


def main(path):
    ctx = afd.afd_create(0)
    res, checks = {}, {}

    def step(name, tensor):
        afd.afd_sync(ctx)
        res[name] = tensor.detach().cpu().contiguous().view(torch.uint8).numpy().copy()
        checks[name] = np.array(afd.afd_check_violations(ctx), dtype=np.int64)

    rng = np.random.default_rng(7)
    cube = lambda s: torch.from_numpy((rng.standard_normal(s) * 2.0).astype(np.float32)).cuda()

    # plain float32 filter: streaming (nx % 4 == 0) and one-voxel kernels, z-chunks
    for shape in [(9, 35, 132), (37, 19, 68), (12, 16, 64), (17, 40, 196), (5, 17, 33)]:
        src = cube(shape)
        for cond in ("rational", "exponential"):
            for kernel, zc in (("auto", 0), ("auto", 3), ("simple", 0)):
                afd.afd_set_kernel(ctx, kernel)
                afd.afd_set_stream_zchunk(ctx, zc)
                t = src.clone()
                afd.afd_filter(ctx, t, 1.3, 0.1, 5, cond, (1.0, 1.5, 0.75))
                step("pm_%s_%s_%s_%d" % (shape, cond, kernel, zc), t)
        afd.afd_set_kernel(ctx, "auto")
        afd.afd_set_stream_zchunk(ctx, 0)
    # device-relative K, intensity form
    src = torch.from_numpy(synth.cutout((24, 40, 64), 3)).cuda()
    out = torch.empty_like(src)
    afd.afd_filter_rel(ctx, src, out, 1.0, 0.125, 6, "rational")
    step("rel", out)
    afd.afd_filter_intensity(ctx, src, out, 1.5, 1.0, 0.0325, 5, (5.0, 4.0, 3.0))
    step("intensity", out)
    # 2-byte storage and temporal blocking
    for shape in [(17, 40, 196), (12, 16, 64), (9, 37, 264)]:
        src = cube(shape)
        for st, dt_ in (("f16", torch.float16), ("bf16", torch.bfloat16), ("i16", torch.int16)):
            q = torch.empty(shape, dtype=dt_, device="cuda")
            afd.afd_quantize(ctx, src, q, st, 1.0)
            for T in (1, 2, 4):
                r = torch.empty_like(q)
                afd.afd_filter_ex(ctx, q, r, st, 1.0, 1.1, 0.1, 6, "exponential", None, T)
                step("ex_%s_%s_%d" % (shape, st, T), r)
            # the deep passes' other route: chains of the two-stage kernel
            afd.afd_set_kernel(ctx, "two_stage")
            r = torch.empty_like(q)
            afd.afd_filter_ex(ctx, q, r, st, 1.0, 1.1, 0.1, 6, "exponential", None, 4)
            afd.afd_set_kernel(ctx, "auto")
            step("ex2_%s_%s_4" % (shape, st), r)
        r = torch.empty_like(src)
        afd.afd_filter_ex(ctx, src, r, "f32", 1.0, 1.1, 0.1, 6, "rational", None, 2)
        step("ex_%s_f32_2" % (shape,), r)
        afd.afd_set_kernel(ctx, "two_stage")
        r = torch.empty_like(src)
        afd.afd_filter_ex(ctx, src, r, "f32", 1.0, 1.1, 0.1, 6, "rational", None, 2)
        afd.afd_set_kernel(ctx, "auto")
        step("ex2_%s_f32_2" % (shape,), r)
    # a resident batch with odd widths, float32 and float16; a short service
    shapes = [(3, 5, 7), (40, 70, 129), (9, 20, 33), (17, 40, 196)]
    for storage, dt_ in (("f32", torch.float32), ("f16", torch.float16)):
        b = afd.afd_batch_create(ctx, shapes, storage, 1.0)
        qs = []
        for i, s in enumerate(shapes):
            t = cube(s)
            if storage == "f16":
                q = torch.empty(s, dtype=torch.float16, device="cuda")
                afd.afd_quantize(ctx, t, q, "f16", 1.0)
                t = q
            afd.afd_batch_set(b, i, t)
            qs.append(t)
        afd.afd_batch_filter(b, [-1.5] * len(shapes), 0.125, 5, "rational")
        for i, s in enumerate(shapes):
            step("batch_%s_%d" % (storage, i),
                 afd.afd_batch_get(b, i, torch.empty(s, dtype=dt_, device="cuda")))
        if storage == "f16":
            srv = afd.afd_serve_create(b, 1 << 28, 8)
            tk = [afd.afd_serve_submit(srv, 1, 1.2, 0.125, 4, "rational"),
                  afd.afd_serve_submit(srv, 3, 0.9, 0.1, 3, "exponential")]
            for _ in range(1000):
                afd.afd_serve_step(srv, wait=True)
                if all(afd.afd_serve_poll(srv, t)[0] == 2 for t in tk):
                    break
            for j, t in enumerate(tk):
                c = (1, 3)[j]
                step("serve_%d" % j, afd.afd_serve_result(srv, t, torch.empty_like(qs[c])))
                afd.afd_serve_release(srv, t)
            srv.close()
        b.close()
    # smoothing: aligned (streamed) and unaligned (plain) separable passes, rotated
    for shape in [(20, 17, 70), (24, 40, 64)]:
        src = cube(shape)
        flat = torch.zeros(src.numel() + 1, device="cuda")
        flat[1:] = src.reshape(-1)
        shifted = flat[1:].view(shape)
        for tag, x in (("al", src), ("un", shifted)):
            for N in ((3, 5, 3), (9, 1, 1), (1, 1, 13)):
                o = torch.empty(shape, device="cuda")
                afd.afd_smooth_box(ctx, x, o, N)
                step("box_%s_%s_%s" % (shape, tag, N), o)
            o = torch.empty(shape, device="cuda")
            afd.afd_smooth_gauss(ctx, x, o, (3.0, 5.0, 3.0))
            step("gauss_%s_%s" % (shape, tag), o)
        o = torch.empty(shape, device="cuda")
        afd.afd_smooth_gauss(ctx, src, o, (3.0, 5.0, 2.0), (20.0, 30.0, 40.0))
        step("gauss_rot_%s" % (shape,), o)
    # the entry point without a context
    src = cube((9, 35, 132))
    out = torch.empty_like(src)
    afd.afd_filter_noalloc(src, out, 1.2, 0.1, 4, "rational")
    torch.cuda.synchronize()
    res["noalloc"] = out.cpu().view(torch.uint8).numpy().copy()

    np.savez(path, checked=np.array(afd.afd_checked_build()),
             **{"r_" + k: v for k, v in res.items()},
             **{"c_" + k: v for k, v in checks.items()})
    ctx.close()


if __name__ == "__main__":
    main(sys.argv[1])
