"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Indexing (cells, offsets, order, quantised positions) must be bit-exact;
forces must meet the rms relative error and max-error bound of the FP32 path.
"""
import numpy as np
import pytest

import oracle
from synth import generators as gen
from synth import workload
from tests.gpu_helpers import (BOUND_K, RMS_TOL, RMS_TOL_PLAIN, make_box, oracle_side, require_cuda,
                               sample_sinks)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    require_cuda()
    from paper_1810_02916_b300 import build
    build.build()


def _assert_same_layout(nf, b):
    st = nf.get_particles()
    assert np.array_equal(st["cell_offsets"], b.offsets)
    assert np.array_equal(st["counts"].astype(np.int64), b.counts)
    assert np.array_equal(st["perm"], b.order)
    assert np.array_equal(st["pos"][:, :3], b.xq)
    assert np.all(st["pos"][:, 3] == 0)
    return st


def _check_forces(acc, ref, sa, tol=RMS_TOL, k=BOUND_K):
    s = oracle.error_stats(acc[:, :3], ref, sa)
    assert s["rms_rel"] <= tol, s
    assert s["max_bound_ratio"] <= k, s
    return s


# ------------------------------------------------------------------ indexing

@pytest.mark.parametrize("case", ["uniform32k", "clustered", "edges"])
def test_binning_is_bit_exact(case):
    rng = np.random.default_rng(1)
    if case == "uniform32k":
        w = workload("uniform32k")
        X, cpd = w.pos, w.cpd
    elif case == "clustered":
        X, _ = gen.clustered(60000, rng, 5, 0.5 / 12, 3.0 / 12)
        cpd = 12
    else:
        cpd = 7
        X = rng.random((5000, 3))
        X[:300] = np.floor(X[:300] * cpd) / cpd               # on cell faces
        X[300:320] = np.nextafter(1.0, 0.0)                   # just below the box edge
        X[320:340] = -1e-9                                    # wraps to the last cell
        X[340:360] = 1.0                                      # wraps to the first cell
        X[360:2000] = X[360]                                  # one crowded cell, order by id
        X[2000:2100] = 5.3                                    # far outside: periodic wrap
    nf = make_box(X, cpd, 1e-4)
    _assert_same_layout(nf, oracle_side(X, cpd))


def test_pair_count_matches_oracle():
    X, _ = gen.clustered(80000, np.random.default_rng(2), 6, 0.5 / 15, 3.0 / 15)
    nf = make_box(X, 15, 1e-4)
    assert nf.pair_count() == oracle.pair_count(oracle_side(X, 15))


# ------------------------------------------------------------------ forces

@pytest.mark.parametrize("mode", [0, 1], ids=["compensated", "plain"])
def test_uniform32k_all_sinks(mode):
    w = workload("uniform32k")
    nf = make_box(w.pos, w.cpd, w.eps, mode=mode)
    b = oracle_side(w.pos, w.cpd)
    _assert_same_layout(nf, b)
    acc = nf.forces()
    ref, sa, pairs = oracle.forces(b, w.eps, with_sumabs=True)
    assert nf.pair_count() == pairs
    _check_forces(acc, ref, sa, tol=RMS_TOL if mode == 0 else RMS_TOL_PLAIN)


@pytest.mark.parametrize("mode", [0, 1], ids=["compensated", "plain"])
def test_clustered64_all_sinks(mode):
    w = workload("clustered64")
    nf = make_box(w.pos, w.cpd, w.eps, mode=mode)
    b = oracle_side(w.pos, w.cpd)
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, w.eps, with_sumabs=True)
    _check_forces(acc, ref, sa, tol=RMS_TOL if mode == 0 else RMS_TOL_PLAIN)
    f64 = nf.forces64()
    assert np.array_equal(f64.astype(np.float32), acc[:, :3])


def test_every_tile_shape_and_ragged_tails():
    """Cells of 1..300 particles (split mode, 1/2/4 sinks per lane, several tiles, ragged tails)."""
    cpd = 9
    rng = np.random.default_rng(3)
    parts = []
    for c in range(cpd ** 3):
        k = c % 41 if c < 600 else (129 + c % 172)
        cx, cy, cz = c // (cpd * cpd), (c // cpd) % cpd, c % cpd
        parts.append((np.array([cx, cy, cz]) + rng.random((k, 3))) / cpd)
    X = np.concatenate(parts)
    X = X[rng.permutation(len(X))]
    eps = 0.3 / cpd
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    _assert_same_layout(nf, b)
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, ref, sa)


def test_one_dense_cell_many_tiles():
    """A 6000-particle cell (largest occupancy class) amid sparse cells."""
    cpd = 6
    rng = np.random.default_rng(4)
    X = np.concatenate([rng.random((3000, 3)), (np.array([2, 3, 1]) + 0.5 + 0.1 * rng.standard_normal((6000, 3))) / cpd])
    X = np.mod(X, 1.0)
    eps = 0.05 / cpd
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    assert b.counts.max() >= 4096
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, ref, sa)


def test_softening_close_to_the_cell_width():
    """eps = 0.95 cell widths: many near-cell pairs fall inside eps (across cell
    faces, coincident copies included), far-cell pairs start at u = 1.05; dense
    clumps on cell faces give 1-, 2- and 4-sink tiles."""
    cpd = 7
    rng = np.random.default_rng(17)
    w = 1.0 / cpd
    centres = (rng.integers(0, cpd, (6, 3)) + np.array([0.0, 0.5, 0.5])) * w   # on x faces
    clumps = [c + 0.25 * w * rng.standard_normal((600, 3)) for c in centres]
    X = np.concatenate([rng.random((2000, 3))] + clumps)
    X = np.concatenate([X, X[rng.choice(len(X), 50, replace=False)]])           # coincident copies
    X = np.mod(X, 1.0)
    eps = 0.95 * w
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    assert b.counts.max() > 64
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, ref, sa)


def test_cpd5_every_pair_once_against_bruteforce():
    cpd = 5
    X, _ = gen.clustered(3000, np.random.default_rng(5), 3, 0.1, 0.3)
    eps = 0.01
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    acc = nf.forces()
    brute = oracle.bruteforce(b, eps)
    _, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, brute, sa)


def test_degenerate_inputs():
    # empty box
    nf = make_box(np.zeros((0, 3)), 5, 0.01)
    assert nf.forces().shape == (0, 4)
    assert nf.pair_count() == 0
    # one particle: no force
    nf = make_box(np.array([[0.3, 0.6, 0.9]]), 5, 0.01)
    assert np.all(nf.forces() == 0)
    # coincident distinct particles: F(0) = 0, no NaN; plus an exact two-body pair
    X = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.1, 0.1, 0.1], [0.1, 0.1, 0.13]])
    nf = make_box(X, 5, 0.01)
    acc = nf.forces()
    b = oracle_side(X, 5)
    ref = oracle.forces(b, 0.01)
    assert np.all(np.isfinite(acc))
    assert np.allclose(acc[:, :3], ref, rtol=2e-6, atol=0)
    # a particle exactly at a cell corner and its neighbour across the periodic boundary
    X = np.array([[0.0, 0.0, 0.0], [1.0 - 1e-3, 1.0 - 1e-3, 1.0 - 1e-3]])
    nf = make_box(X, 7, 1e-4)
    acc = nf.forces()
    ref = oracle.forces(oracle_side(X, 7), 1e-4)
    assert np.allclose(acc[:, :3], ref, rtol=2e-6, atol=0)


# ------------------------------------------------------------------ invariants

def test_whole_cell_translation_is_bit_identical():
    cpd = 8
    X, _ = gen.clustered(40000, np.random.default_rng(6), 4, 0.05, 0.2)
    X = np.floor(X * 2.0 ** 30) * 2.0 ** -30          # dyadic: the shift below is exact
    nf = make_box(X, cpd, 1e-3)
    b = oracle_side(X, cpd)
    a0 = nf.forces()
    shift = np.array([3, 1, 6]) / cpd
    X2 = np.mod(X + shift, 1.0)
    b2 = oracle_side(X2, cpd)
    # same particles must keep their cell-relative offsets for the test to apply
    assert np.array_equal(b2.xq[np.argsort(b2.order)], b.xq[np.argsort(b.order)])
    nf2 = make_box(X2, cpd, 1e-3)
    a1 = nf2.forces()
    # map by particle id
    assert np.array_equal(a1[np.argsort(b2.order)], a0[np.argsort(b.order)])


def test_third_law_on_gpu():
    X, _ = gen.clustered(50000, np.random.default_rng(7), 5, 0.05, 0.2)
    nf = make_box(X, 10, 1e-3)
    b = oracle_side(X, 10)
    nf.forces(False)
    a64 = nf.forces64()
    _, sa, _ = oracle.forces(b, 1e-3, with_sumabs=True)
    assert np.abs(a64.sum(axis=0)).max() <= 64 * 2.0 ** -24 * sa.sum()


def test_lattice_zero_on_gpu():
    cpd = 9
    g = (np.arange(cpd) + 0.5) / cpd
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + np.array([0.1, 0.2, -0.3]) / cpd
    nf = make_box(X, cpd, 0.01 / cpd)
    acc = nf.forces()
    _, sa, _ = oracle.forces(oracle_side(X, cpd), 0.01 / cpd, with_sumabs=True)
    assert np.abs(acc[:, :3]).max() <= 8 * 2.0 ** -24 * sa.max()


# ------------------------------------------------------------------ state, validation

def test_checkpoint_resume_is_bit_identical():
    import paper_1810_02916_b300 as nfb
    X, _ = gen.clustered(30000, np.random.default_rng(8), 3, 0.05, 0.2)
    nf = make_box(X, 9, 1e-3)
    a0 = nf.forces()
    st = nf.get_particles()
    nf2 = nfb.NearField(9, 1e-3)
    nf2.set_particles(st["cell_offsets"], st["counts"], st["pos"])
    assert np.array_equal(nf2.forces(), a0)


def test_set_particles_rejects_bad_input_and_keeps_state():
    import paper_1810_02916_b300 as nfb
    X, _ = gen.clustered(5000, np.random.default_rng(9), 2, 0.05, 0.2)
    nf = make_box(X, 6, 1e-3)
    a0 = nf.forces()
    st = nf.get_particles()
    bad = st["cell_offsets"].copy()
    bad[5] += 1
    with pytest.raises(nfb.NearFieldError) as e:
        nf.set_particles(bad, st["counts"], st["pos"])
    assert e.value.code == nfb.NF_EINVAL
    pos = st["pos"].copy()
    pos[7, 1] = 0.75
    with pytest.raises(nfb.NearFieldError):
        nf.set_particles(st["cell_offsets"], st["counts"], pos)
    pos[7, 1] = np.nan
    with pytest.raises(nfb.NearFieldError):
        nf.set_particles(st["cell_offsets"], st["counts"], pos)
    with pytest.raises(nfb.NearFieldError):
        nf.bin_particles(np.full((10, 3), np.inf))
    assert np.array_equal(nf.forces(), a0)


def test_kick_drift_requires_forces_and_respects_drift_limit():
    import paper_1810_02916_b300 as nfb
    X = np.random.default_rng(10).random((2000, 3))
    nf = make_box(X, 7, 1e-3)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.kick_drift(0.01)
    assert e.value.code == nfb.NF_ESTATE
    nf.forces(False)
    st0 = nf.get_particles()
    v = np.zeros((nf.n, 4), np.float32)
    v[3, 0] = 1.0                      # moves 1.0 * dt * 7 cells
    nf.set_velocities(v)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.kick_drift(0.2)
    assert e.value.code == nfb.NF_EINVAL
    st1 = nf.get_particles()
    assert np.array_equal(st0["pos"], st1["pos"]) and np.array_equal(st0["perm"], st1["perm"])


# ------------------------------------------------------------------ Plummer softening (Eq. eqn:plummer)

@pytest.mark.parametrize("name", ["uniform32k", "clustered64"])
def test_plummer_forces_match_oracle(name):
    import paper_1810_02916_b300 as nfb
    w = workload(name)
    eps_p = w.eps / 2.16
    nf = nfb.NearField(w.cpd, eps_p)
    nf.set_softening(nfb.PLUMMER)
    nf.bin_particles(w.pos)
    acc = nf.forces()
    b = oracle_side(w.pos, w.cpd)
    ref, sa, _ = oracle.forces(b, eps_p, soft=oracle.PLUMMER, with_sumabs=True)
    _check_forces(acc, ref, sa)
    # the spline pass of the same box differs (the laws differ inside eps)
    nf.set_softening(nfb.SPLINE)
    assert not np.array_equal(nf.forces(), acc)


def test_plummer_adjoint_matches_oracle():
    import paper_1810_02916_b300 as nfb
    w = workload("clustered64")
    nf = nfb.NearField(w.cpd, w.eps / 2.16)
    nf.set_softening(nfb.PLUMMER)
    nf.bin_particles(w.pos)
    W = np.zeros((nf.n, 4), np.float32)
    W[:, :3] = gen.cotangent(nf.n, np.random.default_rng(31)).astype(np.float32)
    g = nf.vjp(W)
    b = oracle_side(w.pos, w.cpd)
    sinks = sample_sinks(b, 20000)
    ref = oracle.vjp(b, w.eps / 2.16, W[:, :3].astype(np.float64), sinks, soft=oracle.PLUMMER)
    s = oracle.error_stats(g[sinks, :3], ref)
    assert s["rms_rel"] <= 1e-5, s


@pytest.mark.parametrize("mode", [0, 1], ids=["compensated", "plain"])
def test_sparse_cells_lane_items(mode):
    """About one particle per cell: nearly every cell is computed through lane items
    (runs of sparse cells, one sink per lane), columns that wrap the box in z included."""
    rng = np.random.default_rng(32)
    cpd = 25
    X = rng.random((20000, 3))
    X[:40] = X[0] + 0.001 * rng.standard_normal((40, 3))          # one crowded cell keeps the general path busy
    X = np.mod(X, 1.0)
    eps = 0.02 / cpd
    nf = make_box(X, cpd, eps, mode=mode)
    b = oracle_side(X, cpd)
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, ref, sa, tol=RMS_TOL if mode == 0 else RMS_TOL_PLAIN)
    W = np.zeros((nf.n, 4), np.float32)
    W[:, :3] = gen.cotangent(nf.n, rng).astype(np.float32)
    g = nf.vjp(W)
    gref = oracle.vjp(b, eps, W[:, :3].astype(np.float64))
    s = oracle.error_stats(g[:, :3], gref)
    assert s["rms_rel"] <= 1e-5, s


def test_lane_items_mixed_occupancy():
    """Cells of 0..24 particles (lane cells hold at most 16 and see at most 1000 sources):
    lane runs that end at a tiled cell, at 32 sinks, at 32 cells (a long empty stretch)
    and at the row end, next to tiled cells; spline and Plummer laws."""
    import paper_1810_02916_b300 as nfb
    cpd = 11
    rng = np.random.default_rng(41)
    counts = rng.choice([0, 0, 1, 1, 2, 3, 4, 4, 5, 8, 12, 16, 17, 24], size=cpd ** 3)
    counts[3 * cpd * cpd: 3 * cpd * cpd + 40] = 0                  # 40 empty cells in a row
    counts[5 * cpd * cpd + 2 * cpd: 5 * cpd * cpd + 3 * cpd] = 4     # a row of 44 sinks in lane cells
    cells = np.repeat(np.arange(cpd ** 3), counts)
    base = np.stack([cells // (cpd * cpd), (cells // cpd) % cpd, cells % cpd], 1)
    X = (base + rng.random((len(cells), 3))) / cpd
    X = X[rng.permutation(len(X))]
    eps = 0.2 / cpd
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, with_sumabs=True)
    _check_forces(acc, ref, sa)
    nf.set_softening(nfb.PLUMMER)
    acc = nf.forces()
    ref, sa, _ = oracle.forces(b, eps, soft=oracle.PLUMMER, with_sumabs=True)
    _check_forces(acc, ref, sa)



# ------------------------------------------------------------------ cut-off acceleration of dense cells

def _dense_box():
    rng = np.random.default_rng(51)
    X, _ = gen.clustered(200000, rng, 6, 0.3 / 16, 1.2 / 16)
    return X, 16, 0.01 / 16


@pytest.mark.parametrize("mode", [0, 1], ids=["compensated", "plain"])
def test_cutoff_matches_its_oracle(mode):
    """Dense far cells through sub-cell quadrupoles: parity with the FP64 oracle of the same
    approximation, the approximation's own error against the exact sum, fewer direct pairs,
    and the exact pass back once the cut-off is 0."""
    X, cpd, eps = _dense_box()
    nf = make_box(X, cpd, eps, mode=mode)
    b = oracle_side(X, cpd)
    assert int((b.counts >= 1024).sum()) >= 10
    exact = nf.forces()
    exact_pairs = nf.pair_count()
    nf.set_cutoff(1024)
    acc = nf.forces()
    assert nf.pair_count() < exact_pairs
    sinks = sample_sinks(b, 20000)
    ref = oracle.cutoff(b, eps, 1024, sinks)
    s = oracle.error_stats(acc[sinks, :3], ref)
    assert s["rms_rel"] <= (RMS_TOL if mode == 0 else RMS_TOL_PLAIN), s
    s_exact = oracle.error_stats(acc[sinks, :3], oracle.forces(b, eps, sinks=sinks))
    assert s_exact["rms_rel"] <= 1e-4, s_exact
    assert not np.array_equal(acc, exact)
    nf.set_cutoff(0)
    assert np.array_equal(nf.forces(), exact)


def test_cutoff_without_dense_cells_is_the_exact_pass():
    X, cpd, eps = _dense_box()
    nf = make_box(X, cpd, eps)
    exact = nf.forces()
    nf.set_cutoff(1 << 40)
    assert np.array_equal(nf.forces(), exact)


def test_cutoff_follows_kick_drift_and_refuses_exact_only_calls():
    import paper_1810_02916_b300 as nfb
    X, cpd, eps = _dense_box()
    nf = make_box(X, cpd, eps)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.set_cutoff(100)
    assert e.value.code == nfb.NF_EINVAL
    nf.set_cutoff(1024)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.set_softening(nfb.PLUMMER)
    assert e.value.code == nfb.NF_ESTATE
    W = np.zeros((nf.n, 4), np.float32)
    with pytest.raises(nfb.NearFieldError) as e:
        nf.vjp(W)
    assert e.value.code == nfb.NF_ESTATE
    with pytest.raises(nfb.NearFieldError) as e:
        nfb.forces_batched([nf])
    assert e.value.code == nfb.NF_EINVAL
    # a step re-plans the dense cells from the drifted particles
    acc = nf.forces()
    amax = float(np.abs(acc[:, :3]).max())
    nf.kick_drift(0.2 * np.sqrt(eps / amax))
    acc2 = nf.forces()
    st = nf.get_particles()
    b2 = oracle.from_sorted(cpd, 1.0, st["cell_offsets"], st["pos"][:, :3])   # the drifted layout as held
    sinks = sample_sinks(b2, 5000)
    s = oracle.error_stats(acc2[sinks, :3], oracle.cutoff(b2, eps, 1024, sinks))
    assert s["rms_rel"] <= RMS_TOL, s


def test_cutoff_with_lane_items_and_split_pieces():
    """One particle per cell of background (lane items) around two dense halos (cut-off
    moments, source pieces): forces against the cut-off oracle, and the direct-pair count
    against a window sum over the cell counts (sparse cells over 5^3, dense ones over 3^3)."""
    cpd = 30
    rng = np.random.default_rng(61)
    cells = np.arange(cpd ** 3)
    base = np.stack([cells // (cpd * cpd), (cells // cpd) % cpd, cells % cpd], 1)
    bg = (base + rng.random(base.shape)) / cpd
    halos = [np.array([7.5, 8.5, 9.5]) / cpd + 0.6 / cpd * rng.standard_normal((9000, 3)),
             np.array([21.5, 20.5, 3.5]) / cpd + 0.4 / cpd * rng.standard_normal((6000, 3))]
    X = np.mod(np.concatenate([bg] + halos), 1.0)
    eps = 0.02 / cpd
    n_min = 1024
    nf = make_box(X, cpd, eps)
    nf.set_cutoff(n_min)
    acc = nf.forces()
    b = oracle_side(X, cpd)
    assert int((b.counts >= n_min).sum()) >= 2 and int((b.counts <= 8).sum()) > cpd ** 3 // 2
    sinks = sample_sinks(b, 20000)
    s = oracle.error_stats(acc[sinks, :3], oracle.cutoff(b, eps, n_min, sinks))
    assert s["rms_rel"] <= RMS_TOL, s
    cnt = b.counts.reshape(cpd, cpd, cpd).astype(np.int64)

    def window(a, r):
        for ax in range(3):
            a = sum(np.roll(a, k, axis=ax) for k in range(-r, r + 1))
        return a
    dense = np.where(cnt >= n_min, cnt, 0)
    direct = int((cnt * (window(cnt - dense, 2) + window(dense, 1))).sum())
    assert nf.pair_count() == direct


def test_cutoff_compact_halo_in_one_particle_per_cell():
    """A compact halo (one dense cell) in a background of one particle per cell: the
    background cells at Chebyshev distance 2 from the halo see it only through its sub-cell
    moments, so none of them may become a lane item (which would sum the halo pair by pair).
    Every sink in those 98 cells is checked one by one against the cut-off oracle, tightly
    enough that the exact sum would fail; the direct-pair count matches the window sum."""
    cpd = 20
    rng = np.random.default_rng(71)
    cells = np.arange(cpd ** 3)
    base = np.stack([cells // (cpd * cpd), (cells // cpd) % cpd, cells % cpd], 1)
    bg = (base + 0.1 + 0.8 * rng.random(base.shape)) / cpd
    hc = np.array([10, 9, 11])
    halo = (hc + 0.5) / cpd + 0.1 / cpd * rng.standard_normal((3000, 3))
    halo = np.clip(halo, hc / cpd + 1e-6, (hc + 1) / cpd - 1e-6)        # the whole halo in one cell
    X = np.mod(np.concatenate([bg, halo]), 1.0)
    eps = 0.02 / cpd
    n_min = 1024
    nf = make_box(X, cpd, eps)
    nf.set_cutoff(n_min)
    acc = nf.forces()
    b = oracle_side(X, cpd)
    hid = (hc[0] * cpd + hc[1]) * cpd + hc[2]
    assert b.counts[hid] == 3001 and int((b.counts >= n_min).sum()) == 1
    cxyz = np.stack([np.arange(cpd ** 3) // (cpd * cpd), (np.arange(cpd ** 3) // cpd) % cpd,
                     np.arange(cpd ** 3) % cpd], 1)
    dist = np.abs((cxyz - hc + cpd // 2) % cpd - cpd // 2).max(1)
    ring = np.concatenate([np.arange(b.offsets[c], b.offsets[c + 1]) for c in np.nonzero(dist == 2)[0]])
    assert ring.size == 98
    sinks = np.unique(np.concatenate([ring, sample_sinks(b, 4000)]))
    ref = oracle.cutoff(b, eps, n_min, sinks)
    exact = oracle.forces(b, eps, sinks=sinks)
    got = acc[sinks, :3].astype(np.float64)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    rel_exact = np.linalg.norm(exact - ref, axis=1) / np.linalg.norm(ref, axis=1)
    on_ring = np.isin(sinks, ring)
    assert rel_exact[on_ring].max() > 1e-5          # the test can tell the two sums apart
    assert rel[on_ring].max() <= 2e-6, rel[on_ring].max()
    s = oracle.error_stats(got, ref)
    assert s["rms_rel"] <= RMS_TOL, s
    cnt = b.counts.reshape(cpd, cpd, cpd).astype(np.int64)

    def window(a, r):
        for ax in range(3):
            a = sum(np.roll(a, k, axis=ax) for k in range(-r, r + 1))
        return a
    dense = np.where(cnt >= n_min, cnt, 0)
    assert nf.pair_count() == int((cnt * (window(cnt - dense, 2) + window(dense, 1))).sum())


# ------------------------------------------------------------------ the paper's largest-cell regime

def _giant_cell_box():
    """One cell of 200,000 particles (the largest cell late in the paper's run holds over
    200,000, Section 2.2) and two dense cells at Chebyshev distance 2 from it, in a sparse
    background (4 particles per cell)."""
    w = workload("giantcell")
    return w.pos, w.cpd, w.eps


def test_giant_cell_splits_across_pieces_and_cells():
    X, cpd, eps = _giant_cell_box()
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    assert b.counts.max() >= 200000
    acc1 = nf.forces()
    acc2 = nf.forces()
    assert np.array_equal(acc1, acc2)                    # split pieces reduce in a fixed order
    giant = int(np.argmax(b.counts))
    rng = np.random.default_rng(82)
    in_giant = rng.choice(np.arange(b.offsets[giant], b.offsets[giant + 1]), 2000, replace=False)
    others = rng.choice(b.n, 2000, replace=False)
    sinks = np.unique(np.concatenate([in_giant, others]))
    ref, sa, _ = oracle.forces(b, eps, sinks=sinks, with_sumabs=True)
    s = oracle.error_stats(acc1[sinks, :3], ref, sa)
    assert s["rms_rel"] <= RMS_TOL and s["max_bound_ratio"] <= BOUND_K, s
    assert nf.pair_count() == oracle.pair_count(b)



# ------------------------------------------------------------------ stored positions' fourth word

def test_stored_cell_z_index_stays_internal():
    """The library keeps each particle's cell z index in the fourth word of its stored
    position (lane items read source z offsets from it); every load, binning and drift must
    write it, and nf_get_particles must hand back the documented pad 0, to host and to
    device memory alike."""
    torch = require_cuda()
    import paper_1810_02916_b300 as nfb
    cpd, eps = 9, 1e-3
    rng = np.random.default_rng(91)
    X = rng.random((30000, 3))
    nf = make_box(X, cpd, eps)
    b = oracle_side(X, cpd)
    ref = oracle.forces(b, eps)

    def check(tag):
        st = nf.get_particles()
        assert not st["pos"][:, 3].any(), tag
        dev = torch.full((nf.n, 4), 7.0, dtype=torch.float32, device="cuda")
        nf._call("nf_get_particles", None, None, nfb._ptr(dev), None, None)
        got = dev.cpu().numpy()
        assert not got[:, 3].any(), tag
        assert np.array_equal(got[:, :3], st["pos"][:, :3]), tag
        return st

    st = check("after binning")
    assert np.array_equal(st["pos"][:, :3], b.xq.astype(np.float32))
    # a caller-binned load with garbage in the pad word: ignored on input, 0 on output
    pos = st["pos"].copy()
    pos[:, 3] = rng.standard_normal(nf.n).astype(np.float32)
    nf.set_particles(st["cell_offsets"], st["counts"], pos)
    check("after nf_set_particles")
    acc = nf.forces()
    s = oracle.error_stats(acc[:, :3], ref)
    assert s["rms_rel"] <= RMS_TOL, s
    # a step that moves every particle up to 0.4 cell widths per axis (many change cells) while
    # the kick moves it by at most 0.01 cell widths
    w = 1.0 / cpd
    dt = float(np.sqrt(0.01 * w / np.abs(nf.forces64()).max()))
    vel = np.zeros((nf.n, 4), np.float32)
    vel[:, :3] = (rng.uniform(-0.4, 0.4, (nf.n, 3)) * w / dt).astype(np.float32)
    nf.set_velocities(vel)
    nf.kick_drift(dt)
    st2 = check("after a drift")
    moved = np.repeat(np.arange(cpd ** 3), np.diff(st2["cell_offsets"]))[np.argsort(st2["perm"])]
    before = np.repeat(np.arange(cpd ** 3), np.diff(st["cell_offsets"]))   # ids = storage order of the load
    assert (moved != before).mean() > 0.2
    # forces after the drift (its re-binning wrote the new cells' z) against the oracle on the
    # box's own state
    counts = st2["counts"].astype(np.int64)
    b2 = oracle.Binned(cpd=cpd, box=1.0, order=st2["perm"].astype(np.int64),
                       cell=np.repeat(np.arange(cpd ** 3), counts), xq=st2["pos"][:, :3].copy(),
                       offsets=st2["cell_offsets"].astype(np.int64), counts=counts)
    acc2 = nf.forces()
    s2 = oracle.error_stats(acc2[:, :3], oracle.forces(b2, eps))
    assert s2["rms_rel"] <= RMS_TOL, s2
