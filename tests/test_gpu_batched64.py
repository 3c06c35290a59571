"""The batched configuration at its stated size: 64 independent periodic boxes,
N log-uniform in [32^3, 128^3], CPD for 30-60 particles per cell, half of them
clustered, all in one persistent launch from one device work queue (the many
slabs per GPU of the paper's pipeline, Section 2.2), run directly and replayed
from a captured CUDA graph.  Every box is checked against the FP64 oracle on
sampled sinks (half from its densest cells), its binning bit-exact, and its
pair count exactly."""
import numpy as np
import pytest

import oracle
from synth import generators as gen
from tests.gpu_helpers import BOUND_K, RMS_TOL, make_box, oracle_side, require_cuda, sample_sinks

pytestmark = pytest.mark.gpu


def test_sixty_four_boxes_one_launch_and_graph_replay_every_box_against_the_oracle():
    torch = require_cuda()
    from paper_1810_02916_b300 import build
    build.build()
    import paper_1810_02916_b300 as nfb

    specs = gen.batched_boxes(64, gen.rng_for(3))
    assert len(specs) == 64
    assert min(s.n for s in specs) >= 32 ** 3 and max(s.n for s in specs) <= 128 ** 3
    assert 0 < sum(s.meta["kind"] == "clustered" for s in specs) < 64
    boxes = [make_box(s.pos, s.cpd, s.eps) for s in specs]
    st = torch.cuda.Stream()
    for b in boxes:
        b.set_stream(st)
    outs = [torch.full((b.n, 4), float("nan"), device="cuda") for b in boxes]
    with torch.cuda.stream(st):
        nfb.forces_batched(boxes, outs)                  # plans the batch, then one launch
    torch.cuda.synchronize()
    direct = [o.cpu().numpy() for o in outs]

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        nfb.forces_batched(boxes, outs)
    for o in outs:
        o.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for o, d in zip(outs, direct):
        assert np.array_equal(o.cpu().numpy(), d)        # replay reproduces the direct launch bit for bit

    for k, (s, nf, acc) in enumerate(zip(specs, boxes, direct)):
        b = oracle_side(s.pos, s.cpd)
        lay = nf.get_particles()
        assert np.array_equal(lay["cell_offsets"], b.offsets), k
        assert np.array_equal(lay["perm"], b.order), k
        assert nf.pair_count() == oracle.pair_count(b), k
        sinks = sample_sinks(b, 2000, seed=100 + k)
        ref, sa, _ = oracle.forces(b, s.eps, sinks=sinks, with_sumabs=True)
        e = oracle.error_stats(acc[sinks, :3], ref, sa)
        assert e["rms_rel"] <= RMS_TOL and e["max_bound_ratio"] <= BOUND_K, (k, s.n, s.cpd, e)
        assert np.all(np.isfinite(acc)), k
