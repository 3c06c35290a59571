"""Host-side failure paths on the GPU: injected allocation failures (NF_ENOMEM)
leave every box usable, and the autograd wrapper refuses a backward pass whose
box was reloaded after its forward pass.

Failures are made on the host (nf_fail_allocations fails an allocation before
cudaMalloc is called); nothing here faults the GPU.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from synth import generators as gen
from tests.gpu_helpers import BOUND_K, RMS_TOL, make_box, oracle_side, require_cuda, sample_sinks

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(autouse=True)
def _cuda_and_reset():
    require_cuda()
    from paper_1810_02916_b300 import build
    build.build()
    import paper_1810_02916_b300 as nfb
    yield
    nfb.fail_allocations(0, 0)


def _check(nf, X, cpd, eps, k=3000):
    acc = nf.forces()
    b = oracle_side(X, cpd)
    sinks = sample_sinks(b, k)
    ref, sa, _ = oracle.forces(b, eps, sinks=sinks, with_sumabs=True)
    s = oracle.error_stats(acc[sinks, :3], ref, sa)
    assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K, s


@pytest.mark.parametrize("skip", [0, 4, 11])
def test_create_reports_enomem_and_frees(skip):
    import paper_1810_02916_b300 as nfb
    nfb.fail_allocations(skip, 1)
    with pytest.raises(nfb.NearFieldError) as e:
        nfb.NearField(9, 1e-3)
    assert e.value.code == nfb.NF_ENOMEM and "injected" in str(e.value)
    nfb.fail_allocations(0, 0)
    X = np.random.default_rng(1).random((4000, 3))
    nf = make_box(X, 9, 1e-3)
    _check(nf, X, 9, 1e-3)


@pytest.mark.parametrize("skip", [0, 6])
def test_load_that_cannot_grow_leaves_an_empty_usable_box(skip):
    import paper_1810_02916_b300 as nfb
    rng = np.random.default_rng(2)
    cpd, eps = 10, 1e-3
    X1 = rng.random((3000, 3))
    X2, _ = gen.clustered(40000, rng, 3, 0.3 / cpd, 1.5 / cpd)
    nf = make_box(X1, cpd, eps)
    nf.forces()
    nfb.fail_allocations(skip, 1)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.bin_particles(X2)
    assert e.value.code == nfb.NF_ENOMEM
    nfb.fail_allocations(0, 0)
    assert nf.n == 0
    with pytest.raises(nfb.NearFieldError) as e:
        nf.forces()
    assert e.value.code == nfb.NF_ESTATE
    with pytest.raises(nfb.NearFieldError) as e:
        nf.kick_drift(1e-6)
    assert e.value.code == nfb.NF_ESTATE
    nf.bin_particles(X2)
    _check(nf, X2, cpd, eps)


def test_cutoff_that_cannot_allocate_stays_exact():
    import paper_1810_02916_b300 as nfb
    rng = np.random.default_rng(3)
    cpd, eps = 12, 0.01 / 12
    X, _ = gen.clustered(120000, rng, 5, 0.3 / cpd, 1.0 / cpd)
    nf = make_box(X, cpd, eps)
    exact = nf.forces()
    nfb.fail_allocations(0, 1)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.set_cutoff(1024)
    assert e.value.code == nfb.NF_ENOMEM and "exact" in str(e.value)
    nfb.fail_allocations(0, 0)
    assert np.array_equal(nf.forces(), exact)
    nf.set_cutoff(1024)
    b = oracle_side(X, cpd)
    assert int((b.counts >= 1024).sum()) >= 2
    sinks = sample_sinks(b, 3000)
    s = oracle.error_stats(nf.forces()[sinks, :3], oracle.cutoff(b, eps, 1024, sinks))
    assert s["rms_rel"] <= RMS_TOL, s


def _batched_enomem_in_fresh_process(skip):
    """Run inside a fresh process, where no batch plan exists yet: the first batched call must
    allocate its plan (17 device buffers), and the skip-th allocation of it fails."""
    import torch
    import paper_1810_02916_b300 as nfb
    rng = np.random.default_rng(4)
    specs = gen.batched_boxes(3, rng, n_lo=2000, n_hi=8000)
    boxes = [make_box(s.pos, s.cpd, s.eps) for s in specs]
    outs = [torch.zeros((b.n, 4), device="cuda") for b in boxes]     # device outputs: no staging buffers
    nfb.fail_allocations(skip, 1)
    try:
        nfb.forces_batched(boxes, outs)
        raise AssertionError("the batched call did not fail")
    except nfb.NearFieldError as e:
        assert e.code == nfb.NF_ENOMEM, e
    nfb.fail_allocations(0, 0)
    nfb.forces_batched(boxes, outs)
    for s, acc in zip(specs, outs):
        b = oracle_side(s.pos, s.cpd)
        ref, sa, _ = oracle.forces(b, s.eps, with_sumabs=True)
        st = oracle.error_stats(acc.cpu().numpy()[:, :3], ref, sa)
        assert st["rms_rel"] <= RMS_TOL and st["max_bound_ratio"] <= BOUND_K, st
    print("batched enomem ok")


@pytest.mark.parametrize("skip", [0, 5, 16])
def test_batched_launch_that_cannot_allocate_recovers(skip):
    code = f"import tests.test_gpu_failures as t; t._batched_enomem_in_fresh_process({skip})"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "batched enomem ok" in r.stdout


def test_backward_refuses_a_box_reloaded_after_forward():
    torch = require_cuda()
    from paper_1810_02916_b300.autograd import nearfield_forces
    cpd, eps = 8, 2e-3
    X, _ = gen.clustered(5000, np.random.default_rng(5), 2, 0.05, 0.2)
    nf = make_box(X, cpd, eps)
    st = nf.get_particles()
    pos = torch.tensor(st["pos"], device="cuda", requires_grad=True)
    offs = torch.tensor(st["cell_offsets"], device="cuda")
    cnts = torch.tensor(st["counts"], device="cuda")
    acc = nearfield_forces(pos, nf, offs, cnts)
    g0 = nf.generation
    nf.bin_particles(X)                       # the box now holds a new load
    assert nf.generation != g0
    with pytest.raises(RuntimeError, match="changed between forward and backward"):
        acc.sum().backward()
    acc2 = nearfield_forces(pos, nf, offs, cnts)
    acc2.sum().backward()                     # an untouched box differentiates as before
    assert pos.grad is not None and torch.isfinite(pos.grad).all()
