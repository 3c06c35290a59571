"""GPU parity of the rest of the path: kick-drift with re-binning, the adjoint
(and its autograd wrapper), the batched persistent launch (also under a
captured CUDA graph), the launch-shape tuner, and sampled parity at the full
workload sizes."""
import os

import numpy as np
import pytest

import oracle
from synth import generators as gen
from synth import workload
from tests.gpu_helpers import BOUND_K, RMS_TOL, make_box, oracle_side, require_cuda, sample_sinks

pytestmark = pytest.mark.gpu

VJP_RMS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    from paper_1810_02916_b300 import build
    build.build()


def _global_by_id(st, cpd, box=1.0):
    C = cpd
    counts = st["counts"].astype(np.int64)
    cell = np.repeat(np.arange(C ** 3), counts)
    xyz = np.stack([cell // (C * C), (cell // C) % C, cell % C], axis=1).astype(np.float64)
    X = (xyz + 0.5 + st["pos"][:, :3].astype(np.float64)) * (box / C)
    out = np.empty_like(X)
    out[st["perm"]] = X
    v = np.empty((len(X), 3))
    v[st["perm"]] = st["vel"][:, :3]
    return out, v


def _min_image(d, box=1.0):
    return d - box * np.round(d / box)


# ------------------------------------------------------------------ kick / drift

def test_one_kick_drift_step_matches_oracle():
    cpd, eps = 8, 2e-3
    rng = np.random.default_rng(21)
    X, _ = gen.clustered(20000, rng, 4, 0.05, 0.2)
    w = 1.0 / cpd
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    nf.forces(False)
    dt = float(np.sqrt(0.1 * eps / np.abs(nf.forces64()).max()))   # max |a| dt^2 = 0.1 eps
    V = (rng.standard_normal((len(X), 3)) * 0.1 * w / dt).astype(np.float32)
    vel = np.zeros((nf.n, 4), np.float32)
    vel[:, :3] = V[b.order]
    nf.set_velocities(vel)
    nf.kick_drift(dt)
    Xg, Vg = _global_by_id(nf.get_particles(), cpd)
    # oracle: FP64 forces on the same quantised start, FP64 kick and drift, re-binned
    A = np.empty((len(X), 3))
    A[b.order] = oracle.forces(b, eps)
    X0 = np.empty((len(X), 3))
    X0[b.order] = oracle.global_positions(b)
    X1, V1 = oracle.kick_drift(X0, V.astype(np.float64), A, dt, 1.0)
    b1 = oracle.bin_positions(X1, cpd)
    X1q = np.empty_like(X1)
    X1q[b1.order] = oracle.global_positions(b1)
    # velocities: FP32 storage (2^-24 relative) plus the FP32 force error times dt
    vtol = 2.0 ** -23 * np.abs(V1) + 1e-5 * np.abs(A).max() * dt
    assert np.all(np.abs(Vg - V1) <= vtol)
    # positions: one quantum of the 2^-22 grid on each side plus the velocity error times dt
    q = 2.0 ** -22 * w
    ptol = 2 * q + vtol * dt
    assert np.all(np.abs(_min_image(Xg - X1q)) <= ptol + 1e-15)


def test_kick_drift_follows_the_fp64_rule_bit_for_bit():
    """Every particle's new velocity, cell and offset equal the stated FP64 rule evaluated in NumPy
    on the box's own state and FP64 forces: v' = fl32(v + a dt); s = (c + 1/2 + x_rel) + (v' dt) cpd;
    new cell floor(s) wrapped, offset rounded once from (s - floor(s) - 1/2) 2^22, half to even.
    A third of the particles get velocities that put the exact offset on a half-quantum tie."""
    cpd, eps = 8, 1e-3                                   # cpd a power of two: cpd / box is exact
    rng = np.random.default_rng(31)
    X = rng.random((40000, 3))
    nf = make_box(X, cpd, eps)
    st0 = nf.get_particles()
    n = nf.n
    dt = 2.0 ** -30
    # drifts m = v' dt cpd = v' 2^-27 cell widths, within the 0.8-cell limit
    V = (np.clip(rng.standard_normal((n, 3)), -3.5, 3.5) * 0.2 * 2.0 ** 27).astype(np.float32)
    tie = rng.random(n) < 1 / 3
    j = rng.integers(-3_000_000, 3_000_000, (n, 3))
    V[tie] = ((j[tie] + 0.5) * 32.0).astype(np.float32)     # m = (j + 1/2) 2^-22 when the kick adds nothing
    vel = np.zeros((n, 4), np.float32)
    vel[:, :3] = V
    nf.set_velocities(vel)
    nf.forces(False)
    A = nf.forces64()
    nf.kick_drift(dt)
    st1 = nf.get_particles()
    # expected, per storage index of the state before the step
    v1 = (V.astype(np.float64) + A * dt).astype(np.float32)
    m = (v1.astype(np.float64) * dt) * float(cpd)
    cell0 = np.repeat(np.arange(cpd ** 3), st0["counts"].astype(np.int64))
    c0 = np.stack([cell0 // (cpd * cpd), (cell0 // cpd) % cpd, cell0 % cpd], axis=1).astype(np.float64)
    s = ((c0 + 0.5) + st0["pos"][:, :3].astype(np.float64)) + m
    c1, q1 = oracle.cell_coordinates(s, 1, 1.0)             # cpd = box = 1: the coordinate is s itself
    c1 = np.mod(c1, cpd)
    cell1 = (c1[:, 0] * cpd + c1[:, 1]) * cpd + c1[:, 2]
    # the state after the step, per particle id
    ids0 = st0["perm"]
    cell_after = np.repeat(np.arange(cpd ** 3), st1["counts"].astype(np.int64))
    by_id_pos = np.empty((n, 3), np.float32)
    by_id_vel = np.empty((n, 3), np.float32)
    by_id_cell = np.empty(n, np.int64)
    by_id_pos[st1["perm"]] = st1["pos"][:, :3]
    by_id_vel[st1["perm"]] = st1["vel"][:, :3]
    by_id_cell[st1["perm"]] = cell_after
    assert np.array_equal(by_id_cell[ids0], cell1)
    assert np.array_equal(by_id_pos[ids0].view(np.uint32), q1.view(np.uint32))
    assert np.array_equal(by_id_vel[ids0].view(np.uint32), v1.view(np.uint32))
    # the tie particles whose kick added nothing did land on ties, so the half-to-even rule was exercised
    exact_tie = tie[:, None] & (v1 == V) & (np.abs(m) <= 0.8)
    assert exact_tie.sum() > 10000


def test_ten_steps_track_the_oracle_trajectory():
    """Ten leapfrog steps of a smooth system stay within a small multiple of the grid quantum."""
    cpd, eps = 6, 0.3 / 6
    rng = np.random.default_rng(22)
    X = rng.random((6000, 3))
    nf = make_box(X, cpd, eps)
    nf.forces(False)
    dt = float(np.sqrt(0.05 * eps / np.abs(nf.forces64()).max()))
    b = oracle_side(X, cpd)
    Xo = np.empty_like(X)
    Xo[b.order] = oracle.global_positions(b)
    Vo = np.zeros_like(X)
    for _ in range(10):
        nf.forces(False)
        nf.kick_drift(dt)
        bo = oracle.bin_positions(Xo, cpd)
        A = np.empty_like(X)
        A[bo.order] = oracle.forces(bo, eps)
        Xo, Vo = oracle.kick_drift(Xo, Vo, A, dt, 1.0)
    Xg, _ = _global_by_id(nf.get_particles(), cpd)
    err = np.abs(_min_image(Xg - Xo)).max() * cpd
    assert err < 1e-4, err      # in cell widths


def test_kick_drift_keeps_canonical_order():
    """After a drift the layout equals a fresh binning of the drifted particles."""
    import paper_1810_02916_b300 as nfb
    cpd = 8                          # power of two: global <-> cell coordinates are exact
    rng = np.random.default_rng(23)
    X = rng.random((30000, 3))
    nf = make_box(X, cpd, 1e-3)
    vel = np.zeros((nf.n, 4), np.float32)
    vel[:, :3] = rng.standard_normal((nf.n, 3)).astype(np.float32) * 0.3
    nf.set_velocities(vel)
    nf.forces(False)
    dt = min(0.05, float(np.sqrt(0.01 * (1.0 / cpd) / np.abs(nf.forces64()).max())))
    nf.kick_drift(dt)
    st = nf.get_particles()
    Xg, _ = _global_by_id(st, cpd)
    nf2 = nfb.NearField(cpd, 1e-3)
    nf2.bin_particles(Xg)
    st2 = nf2.get_particles()
    assert np.array_equal(st["cell_offsets"], st2["cell_offsets"])
    assert np.array_equal(st["pos"], st2["pos"])
    assert np.array_equal(st["perm"], st2["perm"])


# ------------------------------------------------------------------ adjoint

def test_vjp_matches_oracle_gradient():
    w = workload("clustered64")
    nf = make_box(w.pos, w.cpd, w.eps)
    b = oracle_side(w.pos, w.cpd)
    rng = np.random.default_rng(24)
    W = np.zeros((nf.n, 4), np.float32)
    W[:, :3] = gen.cotangent(nf.n, rng).astype(np.float32)
    g = nf.vjp(W)
    sinks = sample_sinks(b, 20000)
    ref = oracle.vjp(b, w.eps, W[:, :3].astype(np.float64), sinks)
    s = oracle.error_stats(g[sinks, :3], ref)
    assert s["rms_rel"] <= VJP_RMS_TOL, s


def test_autograd_function_backward_is_the_adjoint():
    torch = require_cuda()
    from paper_1810_02916_b300.autograd import nearfield_forces
    cpd, eps = 8, 2e-3
    X, _ = gen.clustered(20000, np.random.default_rng(25), 3, 0.05, 0.2)
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    st = nf.get_particles()
    pos = torch.tensor(st["pos"], device="cuda", requires_grad=True)
    offs = torch.tensor(st["cell_offsets"], device="cuda")
    cnts = torch.tensor(st["counts"], device="cuda")
    W = torch.zeros((nf.n, 4), device="cuda")
    W[:, :3] = torch.tensor(gen.cotangent(nf.n, np.random.default_rng(26)), dtype=torch.float32)
    acc = nearfield_forces(pos, nf, offs, cnts)
    (acc * W).sum().backward()
    ref_acc, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    s = oracle.error_stats(acc.detach().cpu().numpy()[:, :3], ref_acc, sa)
    assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K
    ref_g = oracle.vjp(b, eps, W.cpu().numpy()[:, :3].astype(np.float64)) * (1.0 / cpd)   # d/d(offset in cells)
    s = oracle.error_stats(pos.grad.cpu().numpy()[:, :3], ref_g)
    assert s["rms_rel"] <= VJP_RMS_TOL, s


# ------------------------------------------------------------------ batched, graphs, tuning

def _boxes(k=6, seed=27):
    rng = np.random.default_rng(seed)
    specs = gen.batched_boxes(k, rng, n_lo=2000, n_hi=40000)
    return specs, [make_box(s.pos, s.cpd, s.eps) for s in specs]


def test_batched_matches_single_box_launches():
    """One launch over all boxes gives each box's forces; the batch splits long items against the
    whole batch's work, so sums may be grouped differently than in a single-box launch (rounding only)."""
    import paper_1810_02916_b300 as nfb
    specs, boxes = _boxes()
    single = [b.forces() for b in boxes]
    batched = nfb.forces_batched(boxes)
    again = nfb.forces_batched(boxes)
    for a, c, d in zip(single, batched, again):
        assert np.array_equal(c, d)                     # deterministic
        s = oracle.error_stats(c[:, :3], a[:, :3].astype(np.float64))
        assert s["rms_rel"] <= RMS_TOL, s              # both sides are within RMS_TOL of the oracle
    for s, a in zip(specs[:2], batched[:2]):
        ob = oracle_side(s.pos, s.cpd)
        ref, sa, _ = oracle.forces(ob, s.eps, with_sumabs=True)
        st = oracle.error_stats(a[:, :3], ref, sa)
        assert st["rms_rel"] <= RMS_TOL and st["max_bound_ratio"] <= BOUND_K


def test_batched_under_cuda_graph_replay():
    torch = require_cuda()
    import paper_1810_02916_b300 as nfb
    _, boxes = _boxes(5, seed=28)
    ref = nfb.forces_batched(boxes)                 # the same plan, launched without a graph
    s = torch.cuda.Stream()
    for b in boxes:
        b.set_stream(s)
    outs = [torch.zeros((b.n, 4), device="cuda") for b in boxes]
    with torch.cuda.stream(s):
        nfb.forces_batched(boxes, outs)              # plans the batch (allocation happens here)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nfb.forces_batched(boxes, outs)
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)


def test_tuner_picks_a_shape_and_keeps_results():
    w = workload("clustered64")
    nf = make_box(w.pos, w.cpd, w.eps)
    a0 = nf.forces()
    rep = nf.tune()
    assert "->" in rep or rep == "cached"
    a1 = nf.forces()
    b = oracle_side(w.pos, w.cpd)
    ref, sa, _ = oracle.forces(b, w.eps, with_sumabs=True)
    for a in (a0, a1):
        s = oracle.error_stats(a[:, :3], ref, sa)
        assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= 2 * 256 + 64


# ------------------------------------------------------------------ full sizes (sampled sinks)

@pytest.mark.parametrize("name", ["clustered256", "zeldovich512"])
def test_full_size_sampled_parity(name):
    """The bench's workloads at full size, in the bench's launch shape, on sampled sinks."""
    w = workload(name)
    nf = make_box(w.pos, w.cpd, w.eps)
    b = oracle_side(w.pos, w.cpd)
    st = nf.get_particles()
    assert np.array_equal(st["cell_offsets"], b.offsets)
    assert np.array_equal(st["perm"], b.order)
    assert np.array_equal(st["pos"][:, :3], b.xq)
    del st
    acc = nf.forces()
    sinks = sample_sinks(b, 4000, seed=29)
    ref, sa, _ = oracle.forces(b, w.eps, sinks, with_sumabs=True)
    s = oracle.error_stats(acc[sinks, :3], ref, sa)
    assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K, s
    assert nf.pair_count() == oracle.pair_count(b)


def test_choose_dt_matches_oracle():
    cpd, eps = 8, 2e-3
    rng = np.random.default_rng(41)
    X, _ = gen.clustered(30000, rng, 4, 0.05, 0.2)
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    V = rng.standard_normal((nf.n, 3)).astype(np.float32)
    vel = np.zeros((nf.n, 4), np.float32)
    vel[:, :3] = V
    nf.set_velocities(vel)
    nf.forces(False)
    dt, parts = nf.choose_dt(0.15, 1.0)
    A = oracle.forces(b, eps)
    dto, po = oracle.choose_dt(b, V.astype(np.float64), A, 0.15, 1.0)
    assert dt == pytest.approx(dto, rel=1e-5)
    for k in ("dt_acc", "dt_drift", "dt_max"):
        assert parts[k] == pytest.approx(po[k], rel=1e-5)


@pytest.mark.parametrize("order", [0, 3, 8])
def test_cell_multipoles_match_oracle(order):
    w = workload("clustered64")
    nf = make_box(w.pos, w.cpd, w.eps)
    b = oracle_side(w.pos, w.cpd)
    M = nf.multipoles(order)
    ref = oracle.multipoles(b, order)
    tol = 1e-13 * b.counts.astype(np.float64)[:, None] + 1e-12 * np.abs(ref)
    assert np.all(np.abs(M - ref) <= tol)
    assert np.array_equal(M[:, 0], b.counts.astype(np.float64))


def test_tuner_result_persists_in_the_cache_file(tmp_path):
    """A second process reads the tuned shape back from NF_TUNE_CACHE instead of timing again."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r); import numpy as np; import paper_1810_02916_b300 as nfb; "
            "nf = nfb.NearField(9, 1e-3); nf.bin_particles(np.random.default_rng(1).random((40000, 3))); "
            "nf.forces(False); print(nf.tune())") % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),)
    env = dict(os.environ, NF_TUNE_CACHE=str(cache))
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert first.returncode == 0, first.stderr
    assert "->" in first.stdout and cache.exists() and cache.read_text().count("\t") == 6
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert second.returncode == 0, second.stderr
    assert second.stdout.strip() == "cached"


TILINGS = [(96, 64, 32, 1024), (96, 40, 18, 1024), (80, 48, 24, 1024), (112, 40, 20, 1024), (96, 40, 18, 512),
           (96, 40, 18, 2048), (64, 32, 16, 128), (128, 64, 32, 1 << 20)]


@pytest.mark.parametrize("tiling", TILINGS, ids=["-".join(map(str, t)) for t in TILINGS])
def test_every_tiling_matches_the_oracle(tiling):
    """The tuner's candidate tilings (and the extremes of the allowed range) all give the
    oracle's forces: a clustered box whose cells hold every remainder 1..127."""
    X, _ = gen.clustered(60000, np.random.default_rng(33), 5, 0.3 / 9, 1.5 / 9)
    nf = make_box(X, 9, 1e-3)
    nf.set_tiling(*tiling)
    assert nf.tuning()["c4"] == tiling[0] and nf.tuning()["split_floor"] == tiling[3]
    acc = nf.forces()
    b = oracle_side(X, 9)
    ref, sa, _ = oracle.forces(b, 1e-3, with_sumabs=True)
    s = oracle.error_stats(acc[:, :3], ref, sa)
    assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K, s


def test_tuner_keys_on_the_occupancy_profile():
    """Two boxes of the same size but different clustering get separate tuning runs; a third box
    with the first one's profile reuses its result."""
    rng = np.random.default_rng(34)
    Xu = rng.random((120000, 3))
    Xc, _ = gen.clustered(120000, np.random.default_rng(35), 6, 0.3 / 14, 1.2 / 14)
    a, b = make_box(Xu, 14, 1e-3), make_box(Xc, 14, 1e-3)
    ra, rb = a.tune(), b.tune()
    assert "->" in ra and "->" in rb and "tiles" in ra
    c = make_box(np.random.default_rng(36).random((120000, 3)), 14, 1e-3)
    assert c.tune() == "cached" and c.tuning() == a.tuning()
    ref = oracle.forces(oracle_side(Xc, 14), 1e-3)
    s = oracle.error_stats(b.forces()[:, :3], ref)
    assert s["rms_rel"] <= RMS_TOL, s



def test_class_profile_accounts_for_every_item_and_pair():
    """nf_profile(2): the per-class item counts and tiled pairs add up (lane items' pairs are
    the rest), the clocks are positive where items ran, and the forces are the same as
    without the profile."""
    X, _ = gen.clustered(12000, np.random.default_rng(37), 3, 0.2 / 16, 0.6 / 16)
    bg = np.random.default_rng(38).random((2 * 16 ** 3, 3))           # sparse background: lane items
    X = np.concatenate([X, bg])
    nf = make_box(X, 16, 1e-3)
    plain = nf.forces()
    nf.profile(2)
    prof = nf.forces()
    nf.profile_read()
    raw = nf.profile_classes()
    assert np.array_equal(plain, prof)
    classes = {k: v for k, v in raw.items() if isinstance(v, tuple)}
    assert sum(v[1] for v in classes.values()) > 0
    tiled_pairs = sum(v[2] for k, v in classes.items() if not k.startswith("lane"))
    assert classes["lane items"][1] > 0 and classes["lane items"][2] == 0
    assert 0 < tiled_pairs < nf.pair_count()
    for k, (cyc, items, _) in classes.items():
        assert (cyc > 0) == (items > 0), k
    assert raw["warps"] > 0 and raw["warp_lifetime_cycles"] >= sum(v[0] for v in classes.values())
    assert nf.profile_classes()["warps"] == 0           # reading resets the sums
