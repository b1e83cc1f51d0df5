"""The synthetic inputs are reproducible: the same call gives the same bytes,
different seeds give different cubes, and on the machine and numpy version
that wrote tests/golden/synth_sha256.json (by make_synth_sha256.py) every
small workload has its recorded SHA-256."""
import json
import os
import platform

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "synth_sha256.json")


def test_same_call_same_bytes():
    assert synth.sha256(synth.cube64()) == synth.sha256(synth.cube64())
    assert synth.sha256(synth.cutout((24, 40, 64), 400)) == \
        synth.sha256(synth.cutout((24, 40, 64), 400))


def test_seeds_differ():
    assert synth.sha256(synth.cube64(0)) != synth.sha256(synth.cube64(1))
    assert synth.sha256(synth.cutout((24, 40, 64), 1)) != \
        synth.sha256(synth.cutout((24, 40, 64), 2))


def test_recorded_digests():
    with open(GOLDEN) as fh:
        rec = json.load(fh)
    if rec["machine"] != platform.machine() or rec["numpy"] != np.__version__:
        pytest.skip("digests recorded on %s with numpy %s" % (rec["machine"], rec["numpy"]))
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_synth_sha256", os.path.join(os.path.dirname(GOLDEN), "make_synth_sha256.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert mod.digests() == rec["sha256"]
