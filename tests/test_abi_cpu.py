"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol the public header declares; argument validation that needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nearfield.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(nf_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libnf():
    from paper_1810_02916_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("nf_create", "nf_set_particles", "nf_forces", "nf_kick_drift", "nf_destroy", "nf_vjp",
                 "nf_forces_batched", "nf_bin_particles", "nf_get_particles", "nf_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libnf):
    missing = [n for n in _declared() if not hasattr(libnf, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_lists_every_declared_symbol():
    import paper_1810_02916_b300 as nfb
    assert sorted(nfb.EXPORTS) == _declared()


def test_library_exports_nothing_else(libnf):
    """Only the nf_* C ABI is visible (kernels and helpers are hidden)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", libnf._name], capture_output=True, text=True).stdout
    ours = [l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("nf_")]
    assert sorted(ours) == _declared()


def test_create_rejects_bad_arguments_without_gpu(libnf):
    """Argument checks run before any CUDA call, so they work on a CPU-only host."""
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()
    h = ctypes.c_void_p()
    assert L.nf_create(4, 2, 1e-3, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL       # cpd < 2R+1
    assert b"cpd" in L.nf_last_error(None)
    assert L.nf_create(9, 3, 1e-3, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL       # R != 2
    assert L.nf_create(9, 2, 0.2, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL        # eps >= cell width
    assert L.nf_create(9, 2, 0.0, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL        # eps <= 0
    w = 1.0 / 9
    assert L.nf_create(9, 2, w * 2.0**-21, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL   # eps < 2^-20 cell widths
    assert b"2^-20" in L.nf_last_error(None)
    assert L.nf_create(9, 2, 1e-3, -1.0, ctypes.byref(h)) == nfb.NF_EINVAL      # box <= 0
    assert L.nf_create(2000, 2, 1e-6, 1.0, ctypes.byref(h)) == nfb.NF_EINVAL    # cpd^3 >= 2^31
    assert h.value is None


def test_null_handles_are_rejected(libnf):
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()
    assert L.nf_forces(None, None) == nfb.NF_EINVAL
    assert L.nf_kick_drift(None, 0.1) == nfb.NF_EINVAL
    L.nf_destroy(None)


def test_plummer_to_spline_length_is_the_printed_factor(libnf):
    """Section 4.3.1: eps_s = 2.16 eps_p (host-only helper, no GPU)."""
    import json
    import os
    import paper_1810_02916_b300 as nfb
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "spline_law.json")))
    assert nfb.spline_eps_from_plummer(0.01) == pytest.approx(g["eps_s_over_eps_p"] * 0.01, rel=1e-15)


def test_failure_hook_validates_its_arguments_without_gpu(libnf):
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()
    assert L.nf_fail_allocations(-1, 1) == nfb.NF_EINVAL
    assert L.nf_fail_allocations(0, -1) == nfb.NF_EINVAL
    assert L.nf_fail_allocations(0, 0) == nfb.NF_OK
    g = ctypes.c_uint64()
    assert L.nf_generation(None, ctypes.byref(g)) == nfb.NF_EINVAL

