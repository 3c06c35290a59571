"""nf_forces_noalloc, the force pass for callers that cannot allocate.

Callers that live inside a device memory pool they do not own, or whose host
process forbids new allocations once it is running, call nf_forces_noalloc
with their own device arrays; the library keeps its work list in a fixed
device array instead of calling cudaMalloc.  This test drives that entry
point through the C ABI twice in a row (the second call reuses the scratch
left by the first) and checks both results against nf_forces on the same
particles, within the force tolerance the other GPU tests use.  It lives in
its own file, collected last, and also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import workload
from tests.gpu_helpers import RMS_TOL, make_box, require_cuda

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
