"""The oracle's pins must catch plausible mistakes.

Each mutant below is a copy of ``oracle/afd_oracle.c`` with one typical slip
planted (a dropped axis, a flipped difference, a wrong conductance, a missing
spacing factor, an in-place Gauss-Seidel sweep, an extra iteration, a
Dirichlet instead of a zero-flux boundary, a wrong stride, a wrong exponent;
for the F diagnostic a strict mask threshold, the filtered intensities in
S_of, and the original mask in place of the filtered one; for smoothing a
window one tap short and transposed weights).
It is compiled on the CPU into a temporary library and run through the same
pins as ``test_oracle_pins.py``; at least one pin must fail for every mutant.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from test_oracle_pins import (fdiag_hand_cubes, frac_pm_facewise, heat_closed_form, impulse,
                              smooth_library)

SRC = os.path.join(os.path.dirname(oracle.__file__), "afd_oracle.c")

MUTANTS = {
    "drop_z_axis": ("for (int a = 0; a < 3; ++a) {\n                        for (int s",
                    "for (int a = 0; a < 2; ++a) {\n                        for (int s"),
    "flipped_difference": ("double d = (cur[q] - cur[p]) / h[a];",
                           "double d = (cur[p] - cur[q]) / h[a];"),
    "rational_without_square": ("return 1.0 / (1.0 + r * r);",
                                "return 1.0 / (1.0 + fabs(r));"),
    "exponential_half": ("return exp(-(r * r));", "return exp(-(r * r) / 2.0);"),
    "flux_missing_spacing": ("acc += orc_conductance(d, K, cond) * d / h[a];",
                             "acc += orc_conductance(d, K, cond) * d;"),
    "gauss_seidel": ("double *cur = I, *nxt = J;\n\n    for (int it = 0; it < n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc",
                     "double *cur = I, *nxt = I;\n\n    for (int it = 0; it < n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc"),
    "extra_iteration": ("for (int it = 0; it < n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc",
                        "for (int it = 0; it <= n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc"),
    "dirichlet_boundary": ("continue; /* zero flux through the boundary */",
                           "{ double d0 = -cur[p] / h[a]; acc += orc_conductance(d0, K, cond) * d0 / h[a]; continue; }"),
    "wrong_y_stride": ("const int64_t stride[3] = {1, nx, nx * ny};\n    double *cur = I, *nxt = J;\n\n    for (int it = 0; it < n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc",
                       "const int64_t stride[3] = {1, ny, nx * ny};\n    double *cur = I, *nxt = J;\n\n    for (int it = 0; it < n_iter; ++it) {\n        for (int64_t z = 0; z < nz; ++z)\n            for (int64_t y = 0; y < ny; ++y)\n                for (int64_t x = 0; x < nx; ++x) {\n                    const int64_t c[3] = {x, y, z};\n                    const int64_t p = x + nx * (y + ny * z);\n                    double acc"),
    "k_zero_passes_flux": ("if (K == 0.0)\n        return 0.0;", "if (K == 0.0)\n        return 1.0;"),
    "fdiag_strict_mask": ("const int mo = io >= t_o;", "const int mo = io > t_o;"),
    "fdiag_filtered_intensity": ("if (mf) {\n                    s_of += io;",
                                 "if (mf) {\n                    s_of += iff;"),
    "fdiag_swapped_masks": ("if (mf) {\n                    s_of += io;",
                            "if (mo) {\n                    s_of += io;"),
    "smooth_window_short": ("for (int dx = -rx; dx <= rx; ++dx) {",
                            "for (int dx = -rx; dx < rx; ++dx) {"),
    "smooth_transposed_weights": ("const double w = W[(dx + rx) + wx * ((dy + ry) + wy * (dz + rz))];",
                                  "const double w = W[(dy + ry) + wx * ((dx + rx) + wy * (dz + rz))];"),
}


def pins_hold(lib) -> bool:
    """The main pins of test_oracle_pins.py, run against ``lib``."""
    f = lambda c, *a, **k: oracle.pm_filter(c, *a, lib=lib, **k)
    try:
        r2 = f(impulse(), 1.0, 0.125, 2, "rational")
        if abs(r2[1, 1, 1] - 821 / 2696) > 1e-15 or abs(r2[1, 1, 0] - 117489 / 1385744) > 1e-15:
            return False
        r = f(impulse(), 1.0, 0.125, 1, "exponential")
        if abs(r[1, 1, 1] - (1 - 0.75 * math.exp(-1))) > 1e-15:
            return False
        r = f(impulse(), 1.0, 0.125, 1, "rational", spacing=(2.0, 1.0, 1.0))
        if abs(r[1, 1, 1] - 0.7) > 1e-15 or abs(r[1, 1, 2] - 1 / 40) > 1e-15:
            return False
        rng = np.random.default_rng(3)
        I0 = rng.standard_normal((3, 9, 4))
        got = f(I0, math.inf, 1 / 64, 5, "rational", spacing=(0.5, 1.0, 2.0))
        if np.abs(got - heat_closed_form(I0, 1 / 64, 5, (0.5, 1.0, 2.0))).max() > 1e-12 * 4:
            return False
        vals = rng.integers(-64, 65, size=(2, 3, 5)) / 16.0
        exact = frac_pm_facewise(vals.tolist(), 1.5, 0.0625, 3, (1.0, 0.5, 2.0))
        got = f(vals, 1.5, 0.0625, 3, "rational", spacing=(1.0, 0.5, 2.0))
        for (x, y, z), v in exact.items():
            if abs(got[z, y, x] - float(v)) > 1e-14 * 4:
                return False
        c = rng.standard_normal((5, 6, 7))
        if not np.array_equal(f(c, 0.0, 0.125, 5, "rational"), c):
            return False
        cs = rng.standard_normal((6, 7, 8)).astype(np.float32)
        ws = oracle.gauss_weights((3.0, 3.0, 2.0), (30.0, 0.0, 0.0))  # rx = ry, not x-y symmetric
        ref = smooth_library(cs, ws)
        if not np.allclose(oracle.smooth(cs, ws, lib=lib), ref, rtol=0, atol=1e-13):
            return False
        Io, If, Im = fdiag_hand_cubes()
        r = oracle.f_diagnostic(Io, If, Im, rms_o=1.0, rms_f=1.0, lib=lib)
        if (r["S_oo"], r["N_o"], r["S_of"], r["N_f"], r["S_mf"]) != (12.0, 3, 6.5, 4, 6.0):
            return False
    except ValueError:
        return False
    return True


def build_variant(src_text: str, tmpdir: str, name: str):
    c = os.path.join(tmpdir, name + ".c")
    so = os.path.join(tmpdir, name + ".so")
    with open(c, "w") as fh:
        fh.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=c11", "-o", so, c, "-lm"])
    return oracle.load_library(so)


@pytest.fixture(scope="module")
def tmpdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def test_unmutated_copy_passes(tmpdir):
    with open(SRC) as fh:
        src = fh.read()
    assert pins_hold(build_variant(src, tmpdir, "clean"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmpdir):
    with open(SRC) as fh:
        src = fh.read()
    old, new = MUTANTS[name]
    assert old in src, "mutation site vanished from the oracle source"
    lib = build_variant(src.replace(old, new, 1), tmpdir, name)
    assert not pins_hold(lib), "pins missed the planted mistake " + name
