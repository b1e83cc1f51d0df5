"""The bounds-checked debug build (-DAFD_CHECK): no kernel of the battery in
checked_workload.py computes an index outside its buffer, and the checked
build's results equal the release build's bit for bit (the checks change no
arithmetic).  Each build runs in its own process, chosen by AFD_LIB."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def run_workload(lib, out):
    env = dict(os.environ, AFD_LIB=lib)
    subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py"), out], env=env,
                   check=True, timeout=600)
    return np.load(out)


def test_checked_build_has_no_violations_and_same_results(tmp_path):
    from paper_1609_03782_gb300 import _build
    checked_lib = _build.build(checked=True)
    release_lib = _build.build()
    a = run_workload(release_lib, str(tmp_path / "release.npz"))
    b = run_workload(checked_lib, str(tmp_path / "checked.npz"))
    assert int(a["checked"]) == 0 and int(b["checked"]) == 1
    names = [k[2:] for k in b.files if k.startswith("c_")]
    assert len(names) > 60
    bad = {n: b["c_" + n].tolist() for n in names if b["c_" + n][0] != 0}
    assert not bad, bad                       # (count, first code, first index) per step
    for k in a.files:
        if k.startswith("r_"):
            assert np.array_equal(a[k], b[k]), k
