"""Writes synth_sha256.json: the SHA-256 of the small generated workloads on
this machine (numpy's transcendental functions may round differently on
another CPU architecture, so the machine and numpy version are recorded and
test_synth.py compares only on a matching one).  Calls only synth/."""
import json
import os
import platform
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import synth  # noqa: E402


def digests():
    cube, model, roi = synth.model_b()
    return {
        "cube64": synth.sha256(synth.cube64()),
        "cutout_24x40x64_seed400": synth.sha256(synth.cutout((24, 40, 64), 400)),
        "cutout_shapes_300": synth.sha256(np.array(synth.cutout_shapes(0, 300), dtype=np.int64)),
        "serving_cube_0": synth.sha256(synth.serving_cube(0)),
        "model_b_cube": synth.sha256(cube),
        "model_b_model": synth.sha256(model),
        "noiseless_disk64": synth.sha256(synth.noiseless_disk64()),
    }


if __name__ == "__main__":
    out = {"machine": platform.machine(), "numpy": np.__version__, "sha256": digests()}
    with open(os.path.join(HERE, "synth_sha256.json"), "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(out, indent=1))
