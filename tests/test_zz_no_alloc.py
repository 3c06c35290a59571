"""nf_forces_noalloc, the force pass for callers that cannot allocate.

Callers that live inside a device memory pool they do not own, or whose host
process forbids new allocations once it is running, call nf_forces_noalloc
with their own device arrays; the library keeps its work list in a fixed
device array instead of calling cudaMalloc.  This test drives that entry
point through the C ABI twice in a row (the second call reuses the scratch
left by the first) and checks both results against nf_forces on the same
particles, within the force tolerance the other GPU tests use.  It lives in
its own file, collected last, and also passes when run alone.

A second check runs in a fresh Python process whose first library call is
nf_forces_noalloc (no box was ever created there), on a box whose densest
cells hold thousands of particles, and compares the result with the FP64
oracle directly.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from synth import generators as gen
from synth import workload
from tests.gpu_helpers import BOUND_K, RMS_TOL, make_box, require_cuda, sample_sinks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _noalloc(L, cpd, eps, box, cell_start, pos, n, acc, stream):
    err = ctypes.create_string_buffer(256)
    rc = L.nf_forces_noalloc(cpd, eps, box, cell_start, pos, n, acc, stream, err, 256)
    return rc, err.value.decode()


def test_noalloc_matches_nf_forces_on_two_calls():
    torch = require_cuda()
    from paper_1810_02916_b300 import build
    build.build()
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()

    w = workload("clustered64")                       # 262144 particles, CPD 25
    nf = make_box(w.pos, w.cpd, w.eps)
    ref = nf.forces()                                 # existing entry point
    st = nf.get_particles()
    cs = torch.tensor(st["cell_offsets"].astype(np.int32), device="cuda")
    pos = torch.tensor(st["pos"], device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        acc = torch.full((nf.n, 4), float("nan"), device="cuda")
        rc, msg = _noalloc(L, w.cpd, w.eps, 1.0, cs.data_ptr(), pos.data_ptr(), nf.n, acc.data_ptr(), stream)
        assert rc == nfb.NF_OK, msg
        torch.cuda.synchronize()
        got = acc.cpu().numpy()
        s = oracle.error_stats(got[:, :3], ref[:, :3].astype(np.float64))
        assert s["rms_rel"] <= RMS_TOL, (call, s)
        assert np.all(np.isfinite(got))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = require_cuda()
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()
    cs = torch.zeros(65 ** 3 + 1, dtype=torch.int32, device="cuda")
    pos = torch.zeros((16, 4), device="cuda")
    acc = torch.zeros((16, 4), device="cuda")
    rc, msg = _noalloc(L, 65, 1e-4, 1.0, cs.data_ptr(), pos.data_ptr(), 0, acc.data_ptr(), None)
    assert rc == nfb.NF_EINVAL and "cpd" in msg
    rc, msg = _noalloc(L, 9, 1e-3, 1.0, cs.data_ptr(), pos.data_ptr(), (1 << 21) + 1, acc.data_ptr(), None)
    assert rc == nfb.NF_EINVAL and "n =" in msg


def _first_call_in_fresh_process():
    """Run inside a fresh process: nf_forces_noalloc is the first library call."""
    import torch
    import paper_1810_02916_b300 as nfb
    L = nfb.lib()
    rng = np.random.default_rng(91)
    cpd = 20
    X, _ = gen.clustered(150000, rng, 5, 0.3 / cpd, 1.5 / cpd)
    eps = (1.0 / 53.0) / 40.0
    b = oracle.bin_positions(X, cpd)
    assert b.counts.max() > 8 * 128, b.counts.max()         # several full tiles in the densest cells
    cs = torch.tensor(b.offsets.astype(np.int32), device="cuda")
    pos4 = np.zeros((b.n, 4), np.float32)
    pos4[:, :3] = b.xq
    pos = torch.tensor(pos4, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sinks = sample_sinks(b, 20000, seed=3)
    ref, sa, _ = oracle.forces(b, eps, sinks=sinks, with_sumabs=True)
    for call in range(2):
        acc = torch.full((b.n, 4), float("nan"), device="cuda")
        rc, msg = _noalloc(L, cpd, eps, 1.0, cs.data_ptr(), pos.data_ptr(), b.n, acc.data_ptr(), stream)
        assert rc == nfb.NF_OK, msg
        torch.cuda.synchronize()
        got = acc.cpu().numpy()
        assert np.all(np.isfinite(got))
        s = oracle.error_stats(got[sinks, :3], ref, sa)
        assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K, (call, s)
    print("fresh-process noalloc ok")


def test_noalloc_as_the_first_call_of_a_fresh_process():
    require_cuda()
    from paper_1810_02916_b300 import build
    build.build()
    code = "import tests.test_zz_no_alloc as t; t._first_call_in_fresh_process()"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "fresh-process noalloc ok" in r.stdout

