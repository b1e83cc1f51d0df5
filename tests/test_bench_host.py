"""Host logic of bench.py on the CPU: the roofline arithmetic of the
precision rows, the profile gate on the reported DRAM traffic, the scale
helper, and the reference arm's JSON line (the FP64 oracle on the host
cores, no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_ceilings_pick_the_lower_bound():
    f32 = bench.ceilings("f32", 1, 780.0, 6786.2)
    assert f32["bound"] == "hbm"
    assert f32["hbm_ceiling"] == pytest.approx(6786.2 / 8.0)
    assert f32["frac_of_bound"] == pytest.approx(780.0 / (6786.2 / 8.0))
    f16 = bench.ceilings("f16", 1, 798.0, 6786.2)
    assert f16["hbm_ceiling"] == pytest.approx(6786.2 / 4.0)
    assert f16["bound"] == "issue"
    assert f16["issue_ceiling"] == pytest.approx(152 * 4 * 32 * 2.07e9 / 30.86 / 1e9)
    t4 = bench.ceilings("i16", 4, 418.0, 6786.2)
    assert t4["hbm_ceiling"] == pytest.approx(6786.2)   # 1 byte per voxel-iteration
    assert t4["bound"] == "issue"
    unknown = bench.ceilings("f16", 8, 100.0, 6786.2)  # no instruction count recorded
    assert unknown["issue_ceiling"] is None and unknown["bound"] == "hbm"


def test_traffic_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    prof = tmp_path / "p.md"
    prof.write_text("kernel_source_sha256_16: %s\ndram_bytes_per_launch_full_size: 123\n" % h)
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic() == 123.0
    prof.write_text("kernel_source_sha256_16: %s\ndram_bytes_per_launch_full_size: 123\n"
                    % ("0" * 16))
    assert bench.profiled_traffic() is None   # the kernel changed since the capture


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
