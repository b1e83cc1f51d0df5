"""Host logic of bench.py on the CPU: the roofline arithmetic of the
precision rows, the profile gate on the reported figures, the issue rate,
the line's summary, the scale helper, the one-cube z-slab mode on two gloo
ranks, and the reference arm's JSON line (the FP64 oracle on the host
cores, no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_ceilings_pick_the_lower_bound(monkeypatch):
    counts = {"f32/1": 29.9, "f16/1": 30.86, "i16/4": 43.0}
    monkeypatch.setattr(bench, "figure", lambda section, key: counts.get(key))
    f32 = bench.ceilings("f32", 1, 780.0, 6786.2)
    assert f32["bound"] == "hbm"
    assert f32["hbm_ceiling"] == pytest.approx(6786.2 / 8.0)
    assert f32["frac_of_bound"] == pytest.approx(780.0 / (6786.2 / 8.0))
    f16 = bench.ceilings("f16", 1, 798.0, 6786.2)
    assert f16["hbm_ceiling"] == pytest.approx(6786.2 / 4.0)
    assert f16["bound"] == "issue"
    assert f16["issue_ceiling"] == pytest.approx(152 * 4 * 32 * 2.07e9 / 30.86 / 1e9)
    t4 = bench.ceilings("i16", 4, 418.0, 6786.2)
    assert t4["hbm_ceiling"] == pytest.approx(6786.2 / 7.0)   # 7 bytes per voxel-iteration
    assert t4["bound"] == "issue"
    unknown = bench.ceilings("f16", 8, 100.0, 6786.2)  # no instruction count recorded
    assert unknown["issue_ceiling"] is None and unknown["bound"] == "hbm"


def test_figures_used_only_for_the_profiled_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    rel = os.path.relpath(str(src), ROOT)
    h = bench.files_hash([rel])
    assert len(h) == 16 and int(h, 16) >= 0
    fig = tmp_path / "figures.json"
    fig.write_text(json.dumps({"dram_bytes_per_launch": {"pm_step_stream_f32_cube512": {
        "value": 123, "files": [rel], "sha256_16": h}}}))
    monkeypatch.setattr(bench, "FIGURES", str(fig))
    assert bench.profiled_traffic() == 123.0
    src.write_text("kernel v2")              # the kernel changed since the capture
    assert bench.profiled_traffic() is None
    assert bench.figure("thread_instr_per_voxel_iter", "f16/1") is None   # absent


def test_committed_figures_name_existing_files():
    with open(bench.FIGURES) as fh:
        d = json.load(fh)
    for section in ("dram_bytes_per_launch", "thread_instr_per_voxel_iter"):
        for key, ent in d[section].items():
            assert ent["value"] > 0 and len(ent["sha256_16"]) == 16, key
            for f in ent["files"] + [ent["summary"]]:
                assert os.path.exists(os.path.join(ROOT, f)), (key, f)


def test_issue_rate_follows_the_device_and_clock(monkeypatch):
    monkeypatch.setattr(bench.Issue, "sm_count", 100)
    monkeypatch.setattr(bench.Issue, "sm_mhz", 1000.0)
    assert bench.Issue.rate() == pytest.approx(100 * 4 * 32 * 1e9)
    monkeypatch.setattr(bench, "figure", lambda sec, key: 40.0)
    c = bench.ceilings("f16", 1, 100.0, 6786.2)
    assert c["issue_ceiling"] == pytest.approx(100 * 4 * 32 * 1e9 / 40.0 / 1e9)


def test_summary_is_short_and_last():
    row = {"storage": "f16", "t_block": 1, "value": 800.0, "speedup_vs_f32": 1.02,
           "err_vs_oracle": {"rms": 2e-5, "faint_max": 0.02}, "gate_pass": False}
    line = {"value": 780.0, "roofline": {"frac": 0.94}, "e2e": {"value": 769.0},
            "cpu_openmp": {"value": 3.1, "cores": 16, "roofline": {"frac": 0.3}},
            "cpu_baseline": {"value": 0.06},
            "lines": {"precision": {"rows": [row] * 13,
                                    "best_gate_pass": {"storage": "i16", "t_block": 4,
                                                       "value": 855.2, "speedup_vs_f32": 1.064}},
                      "batch": {"f32": {"value": 660.0}, "f16": {"value": 657.0}},
                      "serving": {"rates": [{"lambda_per_s": 50, "requests": 3000,
                                             "p50_ms": 1.3, "p99_ms": 3.8}] * 4,
                                  "saturation": {"saturation_gvox_iter_per_s": 600.0}}}}
    s = bench.summary(line)
    assert len(json.dumps(s)) < 1400
    assert s["precision"][0] == ["f16", 1, 800.0, 1.02, 2e-5, 0.02, False]
    assert s["precision_best_gate_pass"] == ["i16", 4, 855.0, 1.06]
    assert s["saturation_gvox_iter_per_s"] == 600.0


def test_i16_scale_is_the_finest_that_holds_the_range():
    # range 32767/1024 x scale = 31.999 x scale
    assert bench.i16_scale(10.58) == 0.5          # 16.0 holds 10.58, 8.0 does not
    assert bench.i16_scale(31.0) == 1.0
    assert bench.i16_scale(32.5) == 2.0
    assert bench.i16_scale(15.99) == 0.5
    assert bench.i16_scale(16.0) == 1.0           # 0.5 gives 15.9995 < 16
    assert bench.i16_scale(0.0) == 1.0 and bench.i16_scale(float("inf")) == 1.0


def test_pass_bytes():
    assert bench.pass_bytes("f32", 1) == 8.0 and bench.pass_bytes("f16", 1) == 4.0
    assert bench.pass_bytes("f16", 2) == 6.0      # 2 + 4 | 4 + 2 bytes over 2 iterations
    assert bench.pass_bytes("f16", 4) == 7.0      # 2 + 4 | 4 + 4 | 4 + 4 | 4 + 2 over 4
    assert bench.pass_bytes("i16", 8) == 7.5
    assert bench.pass_bytes("f32", 4) == 8.0


def test_pow2_near():
    assert bench.pow2_near(1.0) == 1.0
    assert bench.pow2_near(0.9997) == 1.0
    assert bench.pow2_near(3.0) == 4.0      # log2 3 = 1.58 rounds up
    assert bench.pow2_near(2.8) == 2.0      # log2 2.8 = 1.49 rounds down
    assert bench.pow2_near(0.0) == 1.0 and bench.pow2_near(float("nan")) == 1.0


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         check=True, timeout=600, cwd=ROOT)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]


def _slab_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(4)
        cube = rng.standard_normal((11, 6, 7)).astype(np.float32)

        def step(buf, its):
            buf.copy_(torch.from_numpy(oracle.pm_filter(buf.numpy(), 1.2, 0.125, its,
                                                        "rational")))

        z0, z1, res, sec = bench.split_slabs_run(
            cube, world, rank, 7, 3, step, 2,
            lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)),
            dist.barrier)
        out.put((rank, z0, z1, res.numpy(), sec))
    finally:
        dist.destroy_process_group()


def test_split_slabs_mode_on_two_gloo_ranks():
    import socket
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(z0, z1) for _, z0, z1, _, _ in parts] == [(0, 6), (6, 11)]
    assert all(sec > 0 for *_, sec in parts)
    rng = np.random.default_rng(4)
    cube = rng.standard_normal((11, 6, 7)).astype(np.float32)
    ref = oracle.pm_filter(cube, 1.2, 0.125, 7, "rational")
    got = np.concatenate([p[3] for p in parts])
    assert np.array_equal(got, ref)
