"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a private copy of the C oracle (on the CPU,
in a temporary directory), points the oracle module at the mutant, and
checks that at least one pin in test_oracle_pins fails.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "nf_oracle.c")

FORCE_PINS = [
    pins.test_spline_coefficients_from_c2_join,
    pins.test_newtonian_tail_exact,
    lambda: pins.test_two_body_newtonian(1.7),
    lambda: pins.test_two_body_spline(0.5),
    pins.test_no_force_beyond_near_field,
    lambda: pins.test_cells_match_bruteforce(7, 900, "clustered"),
    pins.test_third_law_total_force_vanishes,
]
VJP_PINS = [lambda: pins.test_vjp_matches_central_differences(0.01, oracle.SPLINE),
            lambda: pins.test_vjp_matches_central_differences(0.08, oracle.SPLINE)]
PLUMMER_VJP_PINS = [lambda: pins.test_vjp_matches_central_differences(0.01, oracle.PLUMMER),
                    lambda: pins.test_vjp_matches_central_differences(0.08, oracle.PLUMMER)]
CUT_PINS = [pins.test_cutoff_without_dense_cells_is_the_direct_sum,
            pins.test_cutoff_with_one_particle_per_subcell_is_exact,
            pins.test_cutoff_error_of_a_generic_cluster_falls_as_its_size_cubed,
            pins.test_cutoff_error_of_a_symmetric_cluster_falls_as_its_size_to_the_fourth,
            pins.test_cutoff_keeps_the_27_near_cells_direct]

MUTANTS = [
    ("spline coefficient", "(10.0 - 15.0 * u + 6.0 * u * u)", "(10.0 - 15.0 * u + 5.0 * u * u)", FORCE_PINS),
    ("spline branch", "if (r < eps) {\n        double u", "if (r > eps) {\n        double u", FORCE_PINS),
    ("separation sign", "double ddx = ((xrel[3 * j] + dx) - xi) * w;", "double ddx = (xi - (xrel[3 * j] + dx)) * w;",
     FORCE_PINS),
    ("missing neighbour layer", "for (int dz = -R; dz <= R; dz++) {\n                    int64_t n = (wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);\n                    for (int64_t j = cell_start[n]; j < cell_start[n + 1]; j++) {\n                        double ddx",
     "for (int dz = -R; dz < R; dz++) {\n                    int64_t n = (wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);\n                    for (int64_t j = cell_start[n]; j < cell_start[n + 1]; j++) {\n                        double ddx",
     FORCE_PINS),
    ("no periodic wrap", "return c < 0 ? c + cpd : c;", "return c < 0 ? 0 : c;", FORCE_PINS),
    ("cell unit dropped", "double ddz = ((xrel[3 * j + 2] + dz) - zi) * w;", "double ddz = ((xrel[3 * j + 2] + dz) - zi);",
     FORCE_PINS),
    ("transposed cell index", "int64_t cz = c % cpd, cy = (c / cpd) % cpd, cx = c / (cpd * cpd);\n        double xi = xrel[3 * i], yi = xrel[3 * i + 1], zi = xrel[3 * i + 2];\n        double ax",
     "int64_t cx = c % cpd, cy = (c / cpd) % cpd, cz = c / (cpd * cpd);\n        double xi = xrel[3 * i], yi = xrel[3 * i + 1], zi = xrel[3 * i + 2];\n        double ax",
     FORCE_PINS),
    ("adjoint cotangent sign", "dw[k] = wv[3 * j + k] - wv[3 * i + k];", "dw[k] = wv[3 * j + k] + wv[3 * i + k];", VJP_PINS),
    ("adjoint Jacobian term", "return -3.0 / (r2 * r2 * r);", "return 3.0 / (r2 * r2 * r);", VJP_PINS),
    ("adjoint spline derivative", "(-15.0 / (eps * r) + 12.0 / (eps * eps))", "(-15.0 / (eps * r) + 6.0 / (eps * eps))",
     VJP_PINS),
    ("Plummer force power", "return 1.0 / (s * sqrt(s));", "return 1.0 / (s * s);",
     [pins.test_plummer_is_gradient_of_plummer_potential, pins.test_eps_conversion_matches_printed_factor]),
    ("Plummer adjoint exponent", "return -3.0 / (s * s * sqrt(s));", "return -2.0 / (s * s * sqrt(s));",
     PLUMMER_VJP_PINS),
    ("Plummer adjoint power of s", "return -3.0 / (s * s * sqrt(s));", "return -3.0 / (s * sqrt(s));",
     PLUMMER_VJP_PINS),
    ("Plummer adjoint softening dropped", "double s = r * r + eps * eps;\n        return -3.0",
     "double s = r * r;\n        return -3.0", PLUMMER_VJP_PINS),
    ("cutoff quadrupole sign", "ax += m * Rv[0] / r3 - QR[0] / r5", "ax += m * Rv[0] / r3 + QR[0] / r5", CUT_PINS),
    ("cutoff radial quadrupole factor", "2.5 * RQR * Rv[1] / r7", "1.5 * RQR * Rv[1] / r7", CUT_PINS),
    ("cutoff quadrupole trace", "3.0 * sv[a] * sv[bb] - (a == bb ? s2 : 0.0)", "3.0 * sv[a] * sv[bb]", CUT_PINS),
    ("cutoff centre of mass", "X[a] /= m;", "X[a] /= m + 1.0;", CUT_PINS),
    ("cutoff sub-cell binning", "floor((x[a] + 0.5) * CUT_K)", "floor((x[a] + 0.5) * (CUT_K - 1))", CUT_PINS),
    ("cutoff near layer", "int far = abs(dx) == 2 || abs(dy) == 2 || abs(dz) == 2;",
     "int far = abs(dx) >= 1 || abs(dy) >= 1 || abs(dz) >= 1;", CUT_PINS),
]


def _load_mutant(src_text, tmpdir):
    path = os.path.join(tmpdir, "mutant.c")
    so = os.path.join(tmpdir, "libmutant.so")
    open(path, "w").write(src_text)
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path, "-lm"])
    lib = ctypes.CDLL(so)
    ref = oracle.lib()
    for name in ("nf_oracle_forces", "nf_oracle_bruteforce", "nf_oracle_vjp", "nf_oracle_law", "nf_oracle_cutoff"):
        getattr(lib, name).argtypes = getattr(ref, name).argtypes
        getattr(lib, name).restype = getattr(ref, name).restype
    return lib


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, checks, monkeypatch):
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name!r} not found"
    mutated = text.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as tmp:
        lib = _load_mutant(mutated, tmp)
        monkeypatch.setattr(oracle, "_lib", lib)
        failures = 0
        for check in checks:
            try:
                check()
            except AssertionError:
                failures += 1
        assert failures >= 1, f"no pin caught the mutant {name!r}"


def _double_rounded_cell_coordinates(X, cpd, box):
    """The binning rule with the offset formed as (s - c) - 1/2 in double, then rounded again."""
    s = np.asarray(X, dtype=np.float64) * (float(cpd) / float(box))
    c = np.floor(s)
    return c.astype(np.int64), oracle.quantise((s - c) - 0.5)


def _truncated_cell_coordinates(X, cpd, box):
    """The binning rule with the offset truncated toward zero instead of rounded."""
    s = np.asarray(X, dtype=np.float64) * (float(cpd) / float(box))
    c = np.floor(s)
    q = np.trunc(((s - c) - 0.5) * 2.0 ** 22) * 2.0 ** -22
    return c.astype(np.int64), q.astype(np.float32)


@pytest.mark.parametrize("mutant", [_double_rounded_cell_coordinates, _truncated_cell_coordinates],
                         ids=["double-rounded offset", "truncated offset"])
def test_binning_pins_catch_mutant(mutant, monkeypatch):
    monkeypatch.setattr(oracle, "cell_coordinates", mutant)
    failures = 0
    for check in (pins.test_binning_rounds_each_offset_once_from_its_exact_value,
                  pins.test_binning_matches_python_restatement):
        try:
            check()
        except AssertionError:
            failures += 1
    assert failures >= 1, f"no pin caught the mutant {mutant.__name__}"
