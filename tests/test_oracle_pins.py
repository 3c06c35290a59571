"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a
closed form, a derivation from a property the paper states, an independent
brute-force code path, a symmetry, or finite differences.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import generators as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "spline_law.json")


def _two_body(cpd, box, eps, X1, X2, soft=oracle.SPLINE):
    b = oracle.bin_positions(np.array([X1, X2], dtype=np.float64), cpd, box)
    acc = oracle.forces(b, eps, soft=soft)
    Xq = oracle.global_positions(b)
    # undo the sort so rows are (particle 1, particle 2)
    inv = np.empty(2, dtype=np.int64)
    inv[b.order] = np.arange(2)
    return acc[inv], Xq[inv]


def _min_image(d, box):
    return d - box * np.round(d / box)


# ------------------------------------------------------------------ pair law

def test_spline_coefficients_from_c2_join():
    """Section 4.3.1: F = (a + b u + c u^2) r/eps^3 joined to r^-2 with C^2 smoothness.

    Solving the three join conditions reproduces the printed coefficients,
    and the oracle's law matches the solved polynomial inside eps.
    """
    g = json.load(open(GOLDEN))
    # F(u) eps^2 = a u + b u^2 + c u^3 ; at u = 1 match 1, -2, 6 (value, d/du, d2/du2 of u^-2)
    A = np.array([[1.0, 1.0, 1.0], [1.0, 2.0, 3.0], [0.0, 2.0, 6.0]])
    coef = np.linalg.solve(A, np.array([1.0, -2.0, 6.0]))
    assert np.allclose(coef, g["spline_coefficients"], rtol=0, atol=1e-12)
    for eps in (1e-3, 0.0078125, 0.37):
        for u in np.linspace(0.0, 0.999, 37):
            r = u * eps
            expect = (coef[0] * u + coef[1] * u ** 2 + coef[2] * u ** 3) / eps ** 2
            assert oracle.law(r, eps) == pytest.approx(expect, rel=1e-13, abs=1e-300)


def test_newtonian_tail_exact():
    """Beyond eps the law is exactly r/r^3 (|F| = 1/r^2)."""
    eps = 0.01
    for r in (0.01, 0.010000001, 0.02, 0.1, 0.7, 3.0):
        assert oracle.law(r, eps) == pytest.approx(1.0 / r ** 2, rel=1e-15)


def test_c2_continuity_numerical():
    """Value, first and second derivative of |F(r)| agree on both sides of eps."""
    eps = 0.05
    h = 1e-4 * eps

    def one_sided(sign):
        rs = eps + sign * h * np.arange(0, 5)
        f = np.array([oracle.law(r, eps) for r in rs])
        # polynomial fit of degree 4 in (r - eps) on one side
        p = np.polyfit(rs - eps, f, 4)
        return p[-1], p[-2], 2 * p[-3]

    lv, ld, ldd = one_sided(-1.0)
    rv, rd, rdd = one_sided(+1.0)
    assert lv == pytest.approx(1 / eps ** 2, rel=1e-9)
    assert rv == pytest.approx(1 / eps ** 2, rel=1e-9)
    assert ld == pytest.approx(-2 / eps ** 3, rel=1e-5)
    assert rd == pytest.approx(-2 / eps ** 3, rel=1e-5)
    assert ldd == pytest.approx(6 / eps ** 4, rel=2e-3)
    assert rdd == pytest.approx(6 / eps ** 4, rel=2e-3)


def test_plummer_is_gradient_of_plummer_potential():
    """Eq. (eqn:plummer): |F| = -dPhi/dr with Phi = -1/sqrt(r^2 + eps^2)."""
    eps = 0.02
    for r in (1e-4, 0.01, 0.02, 0.05, 0.3):
        h = 1e-6 * max(r, eps)
        phi = lambda x: -1.0 / math.sqrt(x * x + eps * eps)
        dphi = (phi(r + h) - phi(r - h)) / (2 * h)
        assert oracle.law(r, eps, oracle.PLUMMER) == pytest.approx(dphi, rel=1e-7)


def test_eps_conversion_matches_printed_factor():
    """Section 4.3.1: equal minimum pairwise dynamical time gives eps_s = 2.16 eps_p.

    The largest angular frequency^2 F(r)/r of each law (at r -> 0) is read off
    the oracle; equating them gives the conversion factor.
    """
    g = json.load(open(GOLDEN))
    r = 1e-9
    w2_spline = oracle.law(r, 1.0, oracle.SPLINE) / r        # times eps_s^-3
    w2_plummer = oracle.law(r, 1.0, oracle.PLUMMER) / r      # times eps_p^-3
    ratio = (w2_spline / w2_plummer) ** (1.0 / 3.0)
    assert ratio == pytest.approx(g["eps_s_over_eps_p"], rel=5e-3)


# ------------------------------------------------------------------ two-body closed forms

@pytest.mark.parametrize("sep_cells", [0.3, 0.9, 1.7, 2.4])
def test_two_body_newtonian(sep_cells):
    cpd, box = 5, 1.0
    w = box / cpd
    eps = 0.01 * w
    direction = np.array([0.48, -0.6, 0.64])
    X1 = np.array([0.5, 0.5, 0.5]) + 0.013
    X2 = X1 + sep_cells * w * direction
    acc, Xq = _two_body(cpd, box, eps, X1, X2)
    d = _min_image(Xq[1] - Xq[0], box)
    r = np.linalg.norm(d)
    assert np.linalg.norm(acc[0]) == pytest.approx(1.0 / r ** 2, rel=1e-12)
    assert np.allclose(acc[0], d / r ** 3, rtol=1e-12, atol=0)
    assert np.array_equal(acc[0], -acc[1])


@pytest.mark.parametrize("u", [0.0, 0.1, 0.5, 0.9, 0.999])
def test_two_body_spline(u):
    cpd, box = 7, 2.0
    w = box / cpd
    eps = 0.05 * w
    X1 = np.array([1.0, 0.3, 1.9])
    d0 = np.array([0.0, 0.6, 0.8]) * (u * eps)
    acc, Xq = _two_body(cpd, box, eps, X1, X1 + d0)
    d = _min_image(Xq[1] - Xq[0], box)
    r = np.linalg.norm(d)
    uu = r / eps
    expect = (10 * uu ** 3 - 15 * uu ** 4 + 6 * uu ** 5) / r ** 2 if r > 0 else 0.0
    assert np.linalg.norm(acc[0]) == pytest.approx(expect, rel=1e-11, abs=1e-300)
    assert np.array_equal(acc[0], -acc[1])


def test_no_force_beyond_near_field():
    """Particles more than R cells apart (per axis) do not interact in the near field."""
    cpd, box = 9, 1.0
    w = box / cpd
    X1 = np.array([0.5, 0.5, 0.5]) * w + np.array([4, 4, 4]) * w
    far = X1 + np.array([3.0, 0.0, 0.0]) * w
    acc, _ = _two_body(cpd, box, 1e-3, X1, far)
    assert np.all(acc == 0.0)
    near = X1 + np.array([2.0, -2.0, 2.0]) * w
    acc, _ = _two_body(cpd, box, 1e-3, X1, near)
    assert np.all(np.abs(acc) > 0)


# ------------------------------------------------------------------ brute force & symmetry

@pytest.mark.parametrize("cpd,n,kind", [(5, 300, "uniform"), (6, 500, "uniform"), (7, 900, "clustered"),
                                        (5, 400, "clustered")])
def test_cells_match_bruteforce(cpd, n, kind):
    rng = np.random.default_rng(cpd * 1000 + n)
    if kind == "uniform":
        X = rng.random((n, 3))
    else:
        X, _ = gen.clustered(n, rng, 3, 0.3 / cpd, 1.0 / cpd)
    eps = 0.02 / cpd
    b = oracle.bin_positions(X, cpd)
    a_cells = oracle.forces(b, eps)
    a_brute = oracle.bruteforce(b, eps)
    scale = np.abs(a_brute).max()
    assert np.abs(a_cells - a_brute).max() <= 1e-12 * scale


def test_third_law_total_force_vanishes():
    rng = np.random.default_rng(3)
    X, _ = gen.clustered(4000, rng, 4, 0.05, 0.2)
    b = oracle.bin_positions(X, 8)
    acc, sa, _ = oracle.forces(b, 2e-3, with_sumabs=True)
    assert np.abs(acc.sum(axis=0)).max() <= 1e-13 * sa.sum()


def test_lattice_forces_vanish():
    """Section 2.1 lattice test: the same offset in every cell gives zero near force."""
    cpd = 7
    w = 1.0 / cpd
    g = (np.arange(cpd) + 0.5) * w
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + np.array([0.1, -0.2, 0.3]) * w
    b = oracle.bin_positions(X, cpd)
    acc, sa, _ = oracle.forces(b, 0.01 * w, with_sumabs=True)
    assert np.abs(acc).max() <= 1e-14 * sa.max()


def test_whole_cell_translation_permutes_forces_exactly():
    rng = np.random.default_rng(7)
    cpd = 6
    X, _ = gen.clustered(1500, rng, 3, 0.1, 0.3)
    b = oracle.bin_positions(X, cpd)
    a0 = oracle.forces(b, 1e-3)
    xyz = b.cell_xyz()
    shifted = (xyz + np.array([2, 5, 1])) % cpd
    cell2 = (shifted[:, 0] * cpd + shifted[:, 1]) * cpd + shifted[:, 2]
    order = np.argsort(cell2, kind="stable")
    counts = np.bincount(cell2, minlength=cpd ** 3)
    off = np.concatenate([[0], np.cumsum(counts)])
    b2 = oracle.from_sorted(cpd, 1.0, off, b.xq[order])
    a1 = oracle.forces(b2, 1e-3)
    assert np.array_equal(a1, a0[order])


def test_pair_count_two_ways():
    rng = np.random.default_rng(11)
    X, _ = gen.clustered(3000, rng, 3, 0.05, 0.2)
    b = oracle.bin_positions(X, 7)
    _, _, pairs = oracle.forces(b, 1e-3, with_sumabs=True)
    assert pairs == oracle.pair_count(b)
    b5 = oracle.bin_positions(X[:700], 5)
    assert oracle.pair_count(b5) == 700 * 700          # every pair is near at cpd = 2R+1


# ------------------------------------------------------------------ binning

def _exact_offset(s):
    """(floor(s), offset in quanta) for a double s: the offset (s - c - 1/2) 2^22 rounded half to
    even in exact rational arithmetic, as a float that keeps the sign of a negative value rounded to 0."""
    c = math.floor(s)
    t = (Fraction(s) - c - Fraction(1, 2)) * 2 ** 22
    q = round(t)                                  # Fraction rounding: half to even
    return c, (-0.0 if (q == 0 and t < 0) else float(q))


def _bin_python(X, cpd, box):
    """Per-particle pure-Python restatement of the binning rule (small inputs)."""
    inv_w = float(cpd) / float(box)
    rows = []
    for idx, p in enumerate(X.tolist()):
        cxyz, rel = [], []
        for v in p:
            c, q = _exact_offset(v * inv_w)
            rel.append(q / 2 ** 22)
            cxyz.append(c % cpd)
        cell = (cxyz[0] * cpd + cxyz[1]) * cpd + cxyz[2]
        rows.append((cell, idx, rel))
    rows.sort(key=lambda t: (t[0], t[1]))
    return rows


def test_binning_matches_python_restatement():
    rng = np.random.default_rng(5)
    cpd, box = 5, 1.0
    X = rng.random((400, 3))
    X[:20] = np.floor(X[:20] * cpd) / cpd            # exactly on cell faces
    X[20:25] = np.nextafter(1.0, 0.0)                # just below the box edge
    X[25:30] = -1e-3                                 # outside, wraps
    X[30:35] = 1.0 + 1e-3                            # outside, wraps
    X[35:60] = X[35]                                 # many in one cell: stability
    b = oracle.bin_positions(X, cpd, box)
    rows = _bin_python(X, cpd, box)
    assert b.cell.tolist() == [r[0] for r in rows]
    assert b.order.tolist() == [r[1] for r in rows]
    assert np.array_equal(b.xq.astype(np.float64), np.array([r[2] for r in rows]))
    assert int(b.offsets[-1]) == 400 and np.array_equal(np.diff(b.offsets), b.counts)
    assert np.all(np.abs(b.xq) <= 0.5)


def test_binning_rounds_each_offset_once_from_its_exact_value():
    """Offsets bit for bit against exact rational rounding, where a double-precision (s - c) - 1/2
    would round twice: -1 < s < 1/4 with bits below 2^-53, half-quantum ties, offsets that round to
    -0, and coordinates far outside the box."""
    q22 = 2.0 ** -22
    s_vals = [
        -(2.5 + 2.0 ** -40) * q22,        # double rounding lands on a tie that breaks the wrong way
        -(1.5 + 2.0 ** -40) * q22, (0.5 - 2.0 ** -40) * q22, 3.5 * q22, -3.5 * q22,
        2.0 ** -60, -2.0 ** -60, 5e-324, -5e-324, 0.0, -0.0,
        0.5 - 0.3 * q22, 0.5 + 0.3 * q22, 0.5 - 0.5 * q22, 0.5 + 0.5 * q22, 1.5 - 0.5 * q22,
        0.25 - 2.0 ** -70, 0.125 + 2.0 ** -80, -0.75 + 2.0 ** -70, 2.0 ** 31 + 0.5 - 2.0 ** -22,
        -(2.0 ** 33) - 0.25, 1e9 + 0.5, -1e9 - 0.75,
    ]
    rng = np.random.default_rng(41)
    s_vals += (rng.uniform(-1, 1, 300) * 2.0 ** rng.integers(-60, 0, 300)).tolist()
    s_vals += (rng.uniform(-3, 3, 300)).tolist()
    s = np.array(s_vals, dtype=np.float64)
    c, xq = oracle.cell_coordinates(s[:, None], 1, 1.0)      # cpd = box = 1: the coordinate is s itself
    for k, v in enumerate(s_vals):
        ce, qe = _exact_offset(v)
        assert int(c[k, 0]) == ce, v
        want = np.float32(qe * q22)
        assert xq[k, 0].view(np.uint32) == want.view(np.uint32), (v, float(xq[k, 0]) / q22, qe)
    # the first case separates the two roundings: a double (s - c) - 1/2 gives one quantum more
    v = s_vals[0]
    twice = np.rint((((v - math.floor(v)) - 0.5)) * 2.0 ** 22)
    assert twice == _exact_offset(v)[1] + 1


def test_quantised_offsets_make_fp32_separations_exact():
    """With x on the 2^-22 grid, (x_j + D) - x_i is exact in FP32 for |D| <= 2."""
    rng = np.random.default_rng(9)
    xi = oracle.quantise(rng.uniform(-0.5, 0.5, 20000))
    xj = oracle.quantise(rng.uniform(-0.5, 0.5, 20000))
    for D in (-2, -1, 0, 1, 2):
        f32 = (xj + np.float32(D)) - xi
        f64 = (xj.astype(np.float64) + D) - xi.astype(np.float64)
        assert np.array_equal(f32.astype(np.float64), f64)


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("soft", [oracle.SPLINE, oracle.PLUMMER], ids=["spline", "plummer"])
@pytest.mark.parametrize("eps", [0.01, 0.08])
def test_vjp_matches_central_differences(eps, soft):
    """Adjoint against central differences of the oracle's own forces.

    Spline law: eps = 0.08 puts most close pairs inside the spline, 0.01 most
    outside.  Plummer law (Eq. eqn:plummer, eps = eps_p): at 0.08 the softening
    dominates the close pairs' (r^2 + eps_p^2), at 0.01 the separation does.
    """
    rng = np.random.default_rng(13)
    cpd = 6
    X, _ = gen.clustered(800, rng, 2, 0.05, 0.15)
    b = oracle.bin_positions(X, cpd)
    wv = gen.cotangent(b.n, rng)
    g = oracle.vjp(b, eps, wv, soft=soft)
    x64 = b.xq.astype(np.float64)
    h = 1e-3 * eps
    for k in rng.choice(b.n, 12, replace=False):
        for ax in range(3):
            vals = []
            for sgn in (+1, -1):
                xp = x64.copy()
                xp[k, ax] += sgn * h / b.w
                bp = oracle.Binned(b.cpd, b.box, b.order, b.cell, xp, b.offsets, b.counts)
                vals.append(float((oracle.forces(bp, eps, soft=soft) * wv).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert fd == pytest.approx(g[k, ax], rel=2e-5, abs=1e-6 * np.abs(g).max())


# ------------------------------------------------------------------ kick / drift

def test_drift_without_force_is_exact():
    X = np.array([[0.1, 0.2, 0.3], [0.95, 0.5, 0.01]])
    V = np.array([[0.25, -0.5, 0.125], [0.5, 0.0, -0.25]])
    X1, V1 = oracle.kick_drift(X, V, np.zeros_like(X), 0.125, 1.0)
    assert np.array_equal(V1, V)
    assert np.array_equal(X1, np.mod(X + V * 0.125, 1.0))


def test_two_body_circular_orbit_closes_at_second_order():
    """Leapfrog on a near-field two-body circular orbit: phase error ~ dt^2."""
    cpd, box = 5, 1.0
    eps = 1e-3
    r = 0.1
    vrel = math.sqrt(2.0 / r)            # equal unit masses, G m = 1: |a_rel| = 2/r^2
    period = 2 * math.pi * r / vrel

    def run(nsteps):
        dt = period / nsteps
        X = np.array([[0.5 - r / 2, 0.5, 0.5], [0.5 + r / 2, 0.5, 0.5]])
        V = np.array([[0.0, -vrel / 2, 0.0], [0.0, vrel / 2, 0.0]])

        def acc_of(X):
            b = oracle.bin_positions(X, cpd, box)
            a = np.empty((2, 3))
            a[b.order] = oracle.forces(b, eps)
            return a

        A = acc_of(X)
        V = V - 0.5 * dt * A            # leapfrog: velocities at half steps
        for _ in range(nsteps):
            A = acc_of(X)
            X, V = oracle.kick_drift(X, V, A, dt, box)
        return np.linalg.norm(X[1] - X[0] - np.array([r, 0.0, 0.0]))

    e1, e2 = run(200), run(400)
    assert e1 < 0.05 * r
    assert 3.0 < e1 / e2 < 5.0


# ------------------------------------------------------------------ error statistics

def test_error_stats_definitions():
    ref = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 4.0]])
    test = ref + np.array([[1e-6, 0, 0], [0, 0, 0], [0, 0, 4e-3]])
    s = oracle.error_stats(test, ref, sumabs=np.array([1.0, 1.0, 1.0]))
    assert s["rms_rel"] == pytest.approx(math.sqrt((1e-12 + 16e-6) / 21.0))
    assert s["median"] == pytest.approx(1e-6)
    assert s["frac_gt_1e-4"] == pytest.approx(1 / 3)
    assert s["max_bound_ratio"] == pytest.approx(4e-3 * 2 ** 24)


# ------------------------------------------------------------------ time step (Section 4.2.1)

def test_time_step_criteria_on_a_hand_worked_case():
    """Two cells, values worked out by hand from the three criteria of Section 4.2.1."""
    cpd, box = 5, 1.0
    X = np.array([[0.01, 0.01, 0.01], [0.02, 0.01, 0.01], [0.5, 0.5, 0.5]])
    b = oracle.bin_positions(X, cpd, box)
    V = np.array([[1.0, 0, 0], [0, 2.0, 0], [0, 0, 0.1]])[b.order]
    A = np.array([[3.0, 0, 0], [0, 4.0, 0], [0, 0, 10.0]])[b.order]
    dt, parts = oracle.choose_dt(b, V, A, eta=0.15, dt_max=1.0)
    # cell of the first two: v_rms = sqrt(2.5), a_max = 4; the lone cold particle: 0.1 / 10
    # global: sqrt(5.01 / 3) / 10 = 0.12923 > 0.01, so the global value wins
    assert parts["dt_acc"] == pytest.approx(0.15 * math.sqrt(5.01 / 3) / 10.0, rel=1e-14)
    assert parts["dt_drift"] == pytest.approx(0.8 * 0.2 / 2.0, rel=1e-14)
    assert dt == pytest.approx(min(1.0, parts["dt_acc"], parts["dt_drift"]))
    # a hot, fast-accelerating cell: the cell criterion decides
    A2 = A.copy()
    A2[:] = [[0, 0, 0.01]] * 3
    _, p2 = oracle.choose_dt(b, V, A2, eta=0.3, dt_max=1.0)
    assert p2["dt_acc"] == pytest.approx(0.3 * math.sqrt(5.01 / 3) / 0.01, rel=1e-14)


# ------------------------------------------------------------------ cell multipoles (Section 2.1)

def test_multipoles_of_one_particle_are_its_monomials():
    X = np.array([[0.13, 0.71, 0.44]])
    b = oracle.bin_positions(X, 5)
    M = oracle.multipoles(b, 8)
    x, y, z = (float(v) for v in b.xq[0])
    c = int(b.cell[0])
    for t, (a, bb, k) in enumerate(oracle.multipole_terms(8)):
        assert M[c, t] == pytest.approx(math.pow(x, a) * math.pow(y, bb) * math.pow(z, k), rel=1e-14, abs=1e-300)
    assert len(oracle.multipole_terms(8)) == 165
    assert np.count_nonzero(np.abs(M).sum(axis=1)) == 1


def test_multipoles_obey_the_shift_theorem():
    """Moments about a shifted origin follow from the binomial expansion of (x + s)^a."""
    rng = np.random.default_rng(17)
    X = rng.random((400, 3)) * 0.2 + 0.4                     # all in one cell of a CPD 5 grid
    b = oracle.bin_positions(X, 5)
    p = 6
    M = oracle.multipoles(b, p)
    s = np.array([0.1, -0.05, 0.2])
    shifted = oracle.Binned(b.cpd, b.box, b.order, b.cell, b.xq.astype(np.float64) + s, b.offsets, b.counts)
    Ms = oracle.multipoles(shifted, p)
    terms = oracle.multipole_terms(p)
    index = {t: i for i, t in enumerate(terms)}
    c = int(b.cell[0])
    for t, (a, bb, k) in enumerate(terms):
        expect = 0.0
        for i in range(a + 1):
            for j in range(bb + 1):
                for l in range(k + 1):
                    expect += (math.comb(a, i) * math.comb(bb, j) * math.comb(k, l) * s[0] ** (a - i) *
                               s[1] ** (bb - j) * s[2] ** (k - l) * M[c, index[(i, j, l)]])
        assert Ms[c, t] == pytest.approx(expect, rel=1e-10, abs=1e-12)


def test_multipoles_of_a_symmetric_cell_have_no_odd_terms():
    rng = np.random.default_rng(18)
    h = rng.uniform(-0.2, 0.2, (50, 3))
    X = (np.concatenate([h, -h]) + 2.5) / 5.0                 # centre of cell (2, 2, 2), point-symmetric
    b = oracle.bin_positions(X, 5)
    M = oracle.multipoles(b, 8)
    c = int(b.cell[0])
    for t, (a, bb, k) in enumerate(oracle.multipole_terms(8)):
        if (a + bb + k) % 2:
            assert abs(M[c, t]) < 1e-15
    assert M[c, 0] == 100.0


# ------------------------------------------------------------------ cut-off acceleration of dense cells

def _far_cell_setup(cluster_cell_rel, sink_rel=(0.0, 0.0, 0.0), cpd=5):
    """One sink in cell (0,0,0) and a cluster (cell-relative offsets) in cell (2,0,0), Chebyshev distance 2."""
    w = 1.0 / cpd
    sink = (np.array([0.5, 0.5, 0.5]) + np.asarray(sink_rel)) * w
    cl = (np.array([2.5, 0.5, 0.5]) + np.asarray(cluster_cell_rel)) * w
    X = np.vstack([sink[None, :], cl])
    b = oracle.bin_positions(X, cpd, 1.0)
    k = int(np.flatnonzero(b.cell == 0)[0])
    return b, np.array([k], dtype=np.int64)


def test_cutoff_without_dense_cells_is_the_direct_sum():
    """n_min above every occupancy: the cut-off sum is the direct sum, term for term."""
    rng = np.random.default_rng(71)
    X, _ = gen.clustered(4000, rng, 4, 0.05, 0.2)
    b = oracle.bin_positions(X, 6, 1.0)
    eps = 0.01 / 6
    ref = oracle.forces(b, eps)
    cut = oracle.cutoff(b, eps, n_min=int(b.counts.max()) + 1)
    assert np.array_equal(ref, cut)


def test_cutoff_with_one_particle_per_subcell_is_exact():
    """A sub-cell holding a single particle has its centre of mass on it and Q = 0."""
    rng = np.random.default_rng(72)
    q = np.array([(a, bb, c) for a in range(4) for bb in range(4) for c in range(4)], dtype=np.float64)
    rel = (q + 0.5) / 4 - 0.5 + (rng.random(q.shape) - 0.5) * 0.2   # one particle inside each sub-cell
    b, sink = _far_cell_setup(rel, sink_rel=(0.21, -0.13, 0.37))
    eps = 0.01 / 5
    ref = oracle.forces(b, eps, sinks=sink)
    cut = oracle.cutoff(b, eps, n_min=1, sinks=sink)
    assert np.allclose(cut, ref, rtol=1e-12, atol=0)


def _cluster_error(offsets, sigma, sink_rel):
    centre = np.array([-0.125, 0.125, 0.125])   # centre of sub-cell (1, 2, 2)
    b, sink = _far_cell_setup(centre + sigma * offsets, sink_rel=sink_rel)
    eps = 0.01 / 5
    ref = oracle.forces(b, eps, sinks=sink)
    cut = oracle.cutoff(b, eps, n_min=1, sinks=sink)
    return float(np.linalg.norm(cut - ref) / np.linalg.norm(ref))


def test_cutoff_error_of_a_generic_cluster_falls_as_its_size_cubed():
    """The first term the quadrupole expansion drops is the octupole: error ~ sigma^3.
    (A missing or mis-signed quadrupole would leave an error ~ sigma^2.)"""
    rng = np.random.default_rng(73)
    off = rng.standard_normal((40, 3))
    for sink_rel in [(0.3, -0.2, 0.1), (-0.4, 0.45, -0.3)]:
        e1 = _cluster_error(off, 0.02, sink_rel)
        e2 = _cluster_error(off, 0.01, sink_rel)
        assert 1e-9 < e1 < 1e-3
        assert 0.09 < e2 / e1 < 0.16, (e1, e2)


def test_cutoff_error_of_a_symmetric_cluster_falls_as_its_size_to_the_fourth():
    """Points at +-s along each axis (and the centre) have no octupole: error ~ sigma^4."""
    off = np.vstack([np.zeros(3), np.eye(3), -np.eye(3), 0.7 * np.eye(3)[[1, 2, 0]], -0.7 * np.eye(3)[[1, 2, 0]]])
    e1 = _cluster_error(off, 0.04, (0.3, -0.2, 0.1))
    e2 = _cluster_error(off, 0.02, (0.3, -0.2, 0.1))
    assert 1e-10 < e1 < 1e-3
    assert 0.045 < e2 / e1 < 0.085, (e1, e2)


def test_cutoff_keeps_the_27_near_cells_direct():
    """A dense cell adjacent to the sink's is summed pair by pair even with n_min = 1."""
    rng = np.random.default_rng(74)
    cpd, w = 5, 0.2
    sink = np.array([[0.5, 0.5, 0.5]]) * w
    near = (np.array([1.5, 1.5, 0.5]) + (rng.random((300, 3)) - 0.5)) * w
    X = np.vstack([sink, near])
    b = oracle.bin_positions(X, cpd, 1.0)
    k = np.flatnonzero(b.cell == 0)
    eps = 0.01 / cpd
    assert np.array_equal(oracle.cutoff(b, eps, n_min=1, sinks=k), oracle.forces(b, eps, sinks=k))
