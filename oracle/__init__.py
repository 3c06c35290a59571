"""FP64 CPU oracle for the Abacus near-field direct sum.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import this package.  It shares no
code with the CUDA library (no common kernels, headers, helpers or
constants); the two meet only in the seeded inputs of the `synth` package.

Contents (each cites the passage it follows):
  bin_positions      cell ownership, cell-relative positions and the stable
                     sort by cell (Section 2.1, K^3 cells, every particle in
                     one cell; positions as offsets from cell centres)
  forces             plain FP64 near-field sum (Section 2.1, Section 4.3.1)
  bruteforce         all-pairs near-field sum without cell lists (pin)
  vjp                FP64 adjoint of the near-field accelerations
  kick_drift         FP64 leapfrog kick and drift (Table 1 rows Kick and
                     Drift) with re-binning
  error_stats        the paper's per-particle fractional-error statistics
                     (Section 4.5) plus the rms relative error
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nf_oracle.c")
_LIB = os.path.join(_HERE, "libnf_oracle.so")

SPLINE, PLUMMER = 0, 1
QUANTUM_BITS = 22      # cell-relative positions are multiples of 2^-22 cell widths


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, strict IEEE double)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        _lib.nf_oracle_forces.argtypes = [i64, cint, dbl, dbl, cint, p, p, i64, p, p, p, p, p]
        _lib.nf_oracle_bruteforce.argtypes = [i64, cint, dbl, dbl, cint, i64, p, p, p]
        _lib.nf_oracle_vjp.argtypes = [i64, cint, dbl, dbl, cint, p, p, p, i64, p, p, p]
        _lib.nf_oracle_cutoff.argtypes = [i64, dbl, dbl, i64, p, p, i64, p, p, p]
        _lib.nf_oracle_law.argtypes = [dbl, dbl, cint]
        _lib.nf_oracle_law.restype = dbl
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- binning

@dataclass
class Binned:
    """Particles sorted by cell: the layout the near-field sum works on."""

    cpd: int
    box: float
    order: np.ndarray        # int64[n]: input index of sorted particle k
    cell: np.ndarray         # int64[n]: cell id of sorted particle k
    xq: np.ndarray           # float32[n, 3]: quantised cell-relative position (cell widths)
    offsets: np.ndarray      # int64[cpd^3 + 1]
    counts: np.ndarray       # int64[cpd^3]

    @property
    def n(self) -> int:
        return int(self.order.shape[0])

    @property
    def w(self) -> float:
        return self.box / self.cpd

    def cell_xyz(self) -> np.ndarray:
        c = self.cell
        C = self.cpd
        return np.stack([c // (C * C), (c // C) % C, c % C], axis=1).astype(np.int64)


def cell_coordinates(X: np.ndarray, cpd: int, box: float):
    """Unwrapped integer cell coordinate and quantised offset from the cell centre.

    s = X * (cpd / box) in double precision (one rounding each) and c = floor(s).
    The offset (s - c) - 1/2, in cell widths, is rounded once from its exact
    value to a multiple of 2^-22, half to even; a negative offset that rounds
    to zero keeps its sign, as rint does (Section 2.1: positions are kept as
    offsets from their cell's centre; the paper fixes no grid, 2^-22 is a
    reading that makes every cross-cell separation exact in FP32).

    In quanta the exact offset is S - K with S = s 2^22 (an exact scaling) and
    K = c 2^22 + 2^21, an even integer, so its rounding is rint(S) - K: adding
    an even integer commutes with round-half-to-even.  rint(S) - c 2^22 is a
    difference of two doubles that is exact (for |s| < 2^30 both are integers
    below 2^52; beyond, both are integer-valued and within 2^22 of each other),
    and subtracting 2^21 from the result is exact too.  Forming
    (s - c) - 1/2 in double instead would round it a second time whenever
    -1 < s < 1/4 and s has bits below 2^-53.
    """
    inv_w = float(cpd) / float(box)
    s = np.asarray(X, dtype=np.float64) * inv_w
    c = np.floor(s)
    S = s * 2.0 ** QUANTUM_BITS
    R = np.rint(S)
    q = (R - c * 2.0 ** QUANTUM_BITS) - 2.0 ** (QUANTUM_BITS - 1)
    q = np.where((q == 0) & (S < R), -0.0, q)          # rounded to zero from below
    return c.astype(np.int64), (q * 2.0 ** -QUANTUM_BITS).astype(np.float32)


def quantise(x_rel: np.ndarray) -> np.ndarray:
    """Round cell-relative offsets to multiples of 2^-22 cell widths (half to even).

    With every offset on this grid, x_j + Delta - x_i is exact in FP32 for
    |Delta| <= 2 (|values| < 4 need at most 24 significant bits).
    """
    q = np.rint(np.asarray(x_rel, dtype=np.float64) * 2.0 ** QUANTUM_BITS) * 2.0 ** -QUANTUM_BITS
    return q.astype(np.float32)


def bin_positions(X: np.ndarray, cpd: int, box: float = 1.0) -> Binned:
    """Assign particles to the cpd^3 periodic cells and sort them by cell.

    Cell id = (cx cpd + cy) cpd + cz (x-major, z fastest); within a cell
    particles keep their input order (stable sort).  Cell-relative positions
    are quantised as `cell_coordinates` states.
    """
    c, xq = cell_coordinates(X, cpd, box)
    ci = np.mod(c, cpd)
    cell = (ci[:, 0] * cpd + ci[:, 1]) * cpd + ci[:, 2]
    order = np.argsort(cell, kind="stable")
    counts = np.bincount(cell, minlength=cpd ** 3).astype(np.int64)
    offsets = np.zeros(cpd ** 3 + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return Binned(cpd, float(box), order.astype(np.int64), cell[order].astype(np.int64),
                  xq[order], offsets, counts)


def from_sorted(cpd: int, box: float, offsets: np.ndarray, xq: np.ndarray, order=None) -> Binned:
    """A Binned built from an already cell-sorted layout (cell offsets + offsets in cells)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    counts = np.diff(offsets)
    cell = np.repeat(np.arange(cpd ** 3, dtype=np.int64), counts)
    n = int(offsets[-1])
    if order is None:
        order = np.arange(n, dtype=np.int64)
    return Binned(cpd, float(box), np.asarray(order, dtype=np.int64), cell,
                  np.asarray(xq, dtype=np.float32).reshape(n, 3), offsets, counts)


# ---------------------------------------------------------------- forces

def forces(b: Binned, eps: float, sinks=None, R: int = 2, soft: int = SPLINE,
           with_sumabs: bool = False):
    """FP64 near-field accelerations (box units) of the sinks (storage indices).

    Returns acc[nsink, 3] (and sum_j |F_ij| per sink, and the pair count).
    """
    if sinks is None:
        sinks = np.arange(b.n, dtype=np.int64)
    sinks = np.ascontiguousarray(sinks, dtype=np.int64)
    scell = np.ascontiguousarray(b.cell[sinks], dtype=np.int64)
    x = np.ascontiguousarray(b.xq, dtype=np.float64)
    off = np.ascontiguousarray(b.offsets, dtype=np.int64)
    acc = np.zeros((sinks.size, 3))
    sa = np.zeros(sinks.size)
    pairs = ctypes.c_int64(0)
    lib().nf_oracle_forces(b.cpd, R, b.w, float(eps), soft, _ptr(off), _ptr(x), sinks.size,
                           _ptr(sinks), _ptr(scell), _ptr(acc), _ptr(sa), ctypes.byref(pairs))
    if with_sumabs:
        return acc, sa, int(pairs.value)
    return acc


def cutoff(b: Binned, eps: float, n_min: int, sinks=None) -> np.ndarray:
    """FP64 accelerations (box units) with dense far cells (>= n_min particles, Chebyshev
    distance 2) replaced by the quadrupoles of their 4^3 sub-cells (see nf_oracle_cutoff)."""
    if sinks is None:
        sinks = np.arange(b.n, dtype=np.int64)
    sinks = np.ascontiguousarray(sinks, dtype=np.int64)
    scell = np.ascontiguousarray(b.cell[sinks], dtype=np.int64)
    x = np.ascontiguousarray(b.xq, dtype=np.float64)
    off = np.ascontiguousarray(b.offsets, dtype=np.int64)
    acc = np.zeros((sinks.size, 3))
    lib().nf_oracle_cutoff(b.cpd, b.w, float(eps), int(n_min), _ptr(off), _ptr(x), sinks.size, _ptr(sinks),
                           _ptr(scell), _ptr(acc))
    return acc


def bruteforce(b: Binned, eps: float, R: int = 2, soft: int = SPLINE) -> np.ndarray:
    """All-pairs near-field sum without cell lists (independent pin)."""
    xyz = np.ascontiguousarray(b.cell_xyz())
    x = np.ascontiguousarray(b.xq, dtype=np.float64)
    acc = np.zeros((b.n, 3))
    lib().nf_oracle_bruteforce(b.cpd, R, b.w, float(eps), soft, b.n, _ptr(xyz), _ptr(x), _ptr(acc))
    return acc


def vjp(b: Binned, eps: float, wv: np.ndarray, sinks=None, R: int = 2, soft: int = SPLINE):
    """Gradient of sum_i w_i . a_i w.r.t. the box-unit positions of the sinks."""
    if sinks is None:
        sinks = np.arange(b.n, dtype=np.int64)
    sinks = np.ascontiguousarray(sinks, dtype=np.int64)
    scell = np.ascontiguousarray(b.cell[sinks], dtype=np.int64)
    x = np.ascontiguousarray(b.xq, dtype=np.float64)
    wv = np.ascontiguousarray(wv, dtype=np.float64).reshape(b.n, 3)
    off = np.ascontiguousarray(b.offsets, dtype=np.int64)
    g = np.zeros((sinks.size, 3))
    lib().nf_oracle_vjp(b.cpd, R, b.w, float(eps), soft, _ptr(off), _ptr(x), _ptr(wv), sinks.size,
                        _ptr(sinks), _ptr(scell), _ptr(g))
    return g


def law(r: float, eps: float, soft: int = SPLINE) -> float:
    """|F| of a single pair at separation r (box units)."""
    return lib().nf_oracle_law(float(r), float(eps), soft)


def pair_count(b: Binned, R: int = 2) -> int:
    """Exact number of ordered (sink, source) evaluations, self pairs included."""
    C = b.cpd
    cnt = b.counts.reshape(C, C, C).astype(np.int64)
    nb = cnt.copy()
    for ax in range(3):
        nb = sum(np.roll(nb, s, axis=ax) for s in range(-R, R + 1))
    return int((cnt * nb).sum())


# ---------------------------------------------------------------- kick / drift

def global_positions(b: Binned) -> np.ndarray:
    """Box-unit positions X = (c + 1/2 + x_rel) w of the sorted particles."""
    return (b.cell_xyz().astype(np.float64) + 0.5 + b.xq.astype(np.float64)) * b.w


def kick_drift(X: np.ndarray, V: np.ndarray, A: np.ndarray, dt: float, box: float):
    """One FP64 leapfrog kick and drift: V += A dt, X += V dt, wrapped into the box."""
    V = V + A * dt
    X = np.mod(X + V * dt, box)
    X[X >= box] = 0.0
    return X, V


def multipole_terms(order: int):
    """(a, b, k) of every term, by degree n, then a = n..0, then b = n-a..0."""
    return [(a, b, n - a - b) for n in range(order + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def multipoles(bn: Binned, order: int = 8) -> np.ndarray:
    """Cartesian moments M_c[a, b, k] = sum_i x^a y^b z^k of every cell (Section 2.1), FP64.

    x = offset from the cell centre in cell widths, unit masses; (cpd^3, T) array.
    """
    terms = multipole_terms(order)
    x = bn.xq.astype(np.float64)
    out = np.zeros((bn.cpd ** 3, len(terms)))
    for t, (a, b, k) in enumerate(terms):
        np.add.at(out[:, t], bn.cell, x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** k)
    return out


def choose_dt(b: Binned, V: np.ndarray, A: np.ndarray, eta: float, dt_max: float):
    """Global time step of Section 4.2.1 (storage-order velocities V and accelerations A, box units).

    dt_acc = eta * max(min over cells of v_rms,c / a_max,c, v_rms / a_max) with
    v_rms = sqrt(mean |v|^2) and a_max = max |a| (cells with a_max = 0 skipped);
    dt_drift = 0.8 cell widths / max |v|; dt = min(dt_max, dt_acc, dt_drift).
    """
    V = np.asarray(V, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    ratio_min = np.inf
    for c in np.flatnonzero(b.counts):
        lo, hi = b.offsets[c], b.offsets[c + 1]
        amax = np.sqrt((A[lo:hi] ** 2).sum(axis=1).max())
        if amax > 0:
            vrms = np.sqrt((V[lo:hi] ** 2).sum(axis=1).mean())
            ratio_min = min(ratio_min, vrms / amax)
    vrms_g = np.sqrt((V ** 2).sum(axis=1).mean()) if len(V) else 0.0
    amax_g = np.sqrt((A ** 2).sum(axis=1).max()) if len(A) else 0.0
    glob = vrms_g / amax_g if amax_g > 0 else np.inf
    dt_acc = eta * max(ratio_min, glob)
    vmax = np.sqrt((V ** 2).sum(axis=1).max()) if len(V) else 0.0
    dt_drift = 0.8 * b.w / vmax if vmax > 0 else np.inf
    return min(dt_max, dt_acc, dt_drift), dict(dt_acc=dt_acc, dt_drift=dt_drift, dt_max=dt_max)


# ---------------------------------------------------------------- errors

def error_stats(a_test: np.ndarray, a_ref: np.ndarray, sumabs: np.ndarray | None = None) -> dict:
    """Error of a test force against the FP64 reference.

    rms_rel   sqrt(sum |da|^2 / sum |a|^2)
    median, p99, frac_gt_1e-4   per-particle |da| / |a| (Section 4.5's statistics)
    max_bound_ratio   max_i |da_i| / (2^-24 sum_j |F_ij|) when sumabs is given
    """
    a_test = np.asarray(a_test, dtype=np.float64)
    a_ref = np.asarray(a_ref, dtype=np.float64)
    da = np.linalg.norm(a_test - a_ref, axis=1)
    na = np.linalg.norm(a_ref, axis=1)
    out = dict(n=int(a_ref.shape[0]),
               rms_rel=float(np.sqrt((da ** 2).sum() / max((na ** 2).sum(), 1e-300))))
    with np.errstate(divide="ignore", invalid="ignore"):
        frac = np.where(na > 0, da / na, np.where(da > 0, np.inf, 0.0))
    out["median"] = float(np.median(frac)) if frac.size else 0.0
    out["p99"] = float(np.percentile(frac, 99)) if frac.size else 0.0
    out["frac_gt_1e-4"] = float((frac > 1e-4).mean()) if frac.size else 0.0
    if sumabs is not None:
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(sumabs > 0, da / (2.0 ** -24 * sumabs), 0.0)
        out["max_bound_ratio"] = float(ratio.max()) if ratio.size else 0.0
    return out
