"""Seeded particle distributions shaped like the paper's workloads.

The paper's own particle sets (the S2016 initial conditions and snapshots,
Section 2.3) are not available, so these synthetic sets stand in for them.
Their shapes follow the paper's description of the run: about 26 particles
per cell at R=2 (Section 2.2), the largest cell holding up to ~10^5
particles late in the run (Section 2.2), and clustered, halo-dominated
matter at late times (Section 2.3, Fig. 3).

Everything here is plain NumPy/SciPy on the host, seeded with PCG64.  All
positions are returned in box units as float64, wrapped into [0, box).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1810_02916

# Mass-function shape of the 256^3 clustered workload: power law
# dN/dM ~ M^-1.9, 2000 halos holding half of 256^3 particles, capped at
# 2e5 particles.  The cap is kept at the same multiple of the mean halo mass
# when the recipe is rescaled to other particle counts.
ALPHA = 1.9
REF_N = 256 ** 3
REF_HALOS = 2000
REF_CAP = 2.0e5
CAP_OVER_MEAN = REF_CAP / (0.5 * REF_N / REF_HALOS)


@dataclass
class Workload:
    """A particle set and the cell grid it is evaluated on."""

    name: str
    pos: np.ndarray          # (N, 3) float64, box units, in [0, box)
    cpd: int                 # cells per dimension
    eps: float               # spline softening length, box units
    box: float = 1.0
    R: int = 2
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def rng_for(config_id: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with 1810_02916 + config id (and a sub-stream)."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(config_id), int(stream)]))


def _wrap(pos: np.ndarray, box: float) -> np.ndarray:
    pos = np.mod(pos, box)
    pos[pos >= box] = 0.0          # np.mod can round a tiny negative up to box
    return pos


def uniform(n: int, rng: np.random.Generator, box: float = 1.0) -> np.ndarray:
    return rng.random((n, 3)) * box


# ---------------------------------------------------------------- halos

def _powerlaw_mean(m: float, mmax: float, alpha: float = ALPHA) -> float:
    a1, a2 = 1.0 - alpha, 2.0 - alpha
    num = (mmax ** a2 - m ** a2) / a2
    den = (mmax ** a1 - m ** a1) / a1
    return num / den


def solve_mmin(mean: float, mmax: float, alpha: float = ALPHA) -> float:
    """Lower mass limit that gives the truncated power law the requested mean."""
    if mean >= mmax:
        return mmax
    lo, hi = 1e-6, mmax * (1 - 1e-12)
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if _powerlaw_mean(mid, mmax, alpha) < mean:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def sample_powerlaw(rng, k: int, m: float, mmax: float, alpha: float = ALPHA) -> np.ndarray:
    """Inverse-CDF draw from dN/dM ~ M^-alpha on [m, mmax]."""
    a1 = 1.0 - alpha
    u = rng.random(k)
    return (m ** a1 + u * (mmax ** a1 - m ** a1)) ** (1.0 / a1)


def largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    """Integer counts proportional to weights that sum exactly to total."""
    q = weights * (total / weights.sum())
    base = np.floor(q).astype(np.int64)
    rem = int(total - base.sum())
    order = np.argsort(-(q - base), kind="stable")
    base[order[:rem]] += 1
    return base


def halo_counts(rng, n_halo_particles: int, n_halos: int, cap: float | None = None):
    """Particle counts of n_halos halos drawn from the M^-1.9 mass function.

    Returns (counts, overflow): counts are capped at `cap`; the particles cut
    by the cap (`overflow`) are given back to the uniform background.
    """
    mean = n_halo_particles / n_halos
    if cap is None:
        cap = min(float(n_halo_particles), CAP_OVER_MEAN * mean)
    mmin = solve_mmin(mean, cap)
    masses = sample_powerlaw(rng, n_halos, mmin, cap)
    counts = largest_remainder(masses, n_halo_particles)
    capped = np.minimum(counts, int(cap))
    return capped, int(counts.sum() - capped.sum())


def plummer_halos(rng, counts: np.ndarray, a_lo: float, a_hi: float, box: float = 1.0):
    """Particles of Plummer spheres with uniform centres and scale radii ~ U[a_lo, a_hi].

    Radii come from the inverse Plummer mass profile r = a (U^-2/3 - 1)^-1/2,
    redrawn when r > 10 a; directions are isotropic.
    """
    k = len(counts)
    centres = rng.random((k, 3)) * box
    a = rng.uniform(a_lo, a_hi, k)
    owner = np.repeat(np.arange(k), counts)
    total = owner.size
    a_p = a[owner]

    def radii(m):
        u = rng.random(m)
        with np.errstate(divide="ignore"):
            return (u ** (-2.0 / 3.0) - 1.0) ** -0.5

    r = radii(total) * a_p
    bad = np.flatnonzero(r > 10.0 * a_p)
    while bad.size:
        r[bad] = radii(bad.size) * a_p[bad]
        bad = bad[r[bad] > 10.0 * a_p[bad]]
    cz = rng.uniform(-1.0, 1.0, total)
    phi = rng.uniform(0.0, 2.0 * math.pi, total)
    s = np.sqrt(1.0 - cz * cz)
    pos = np.empty((total, 3))
    pos[:, 0] = centres[owner, 0] + r * s * np.cos(phi)
    pos[:, 1] = centres[owner, 1] + r * s * np.sin(phi)
    pos[:, 2] = centres[owner, 2] + r * cz
    return _wrap(pos, box), dict(centres=centres, a=a, counts=counts)


def clustered(n: int, rng, n_halos: int, a_lo: float, a_hi: float,
              frac: float = 0.5, box: float = 1.0, cap: float | None = None):
    """Half uniform background, half in power-law-mass Plummer halos."""
    n_h = int(round(n * frac))
    counts, overflow = halo_counts(rng, n_h, n_halos, cap)
    halos, info = plummer_halos(rng, counts, a_lo, a_hi, box)
    bg = uniform(n - n_h + overflow, rng, box)
    pos = np.concatenate([bg, halos])
    pos = pos[rng.permutation(pos.shape[0])]
    info["overflow"] = overflow
    return pos, info


# ---------------------------------------------------------------- Zel'dovich

def zeldovich_lattice(n_side: int, rng, index: float = -1.5, rms_disp: float = 0.5,
                      box: float = 1.0):
    """Lattice particles displaced by the Zel'dovich field of a Gaussian density.

    delta(k) has power P(k) ~ k^index for 0 < |k| <= k_Ny = pi n_side / box
    (sharp spherical cut).  The displacement psi(k) = i k / k^2 delta(k) is
    scaled so that the rms |psi| is `rms_disp` lattice spacings.
    """
    import scipy.fft as sfft

    n = n_side
    g = rng.standard_normal((n, n, n), dtype=np.float32)
    G = sfft.rfftn(g, workers=-1)
    del g
    f_full = np.fft.fftfreq(n, d=1.0 / n).astype(np.float32)       # integer wavenumbers
    f_half = np.fft.rfftfreq(n, d=1.0 / n).astype(np.float32)
    two_pi = np.float32(2.0 * math.pi / box)
    kx = (two_pi * f_full)[:, None, None]
    ky = (two_pi * f_full)[None, :, None]
    kz = (two_pi * f_half)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k_ny = math.pi * n / box
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where((k2 > 0) & (k2 <= k_ny * k_ny),
                       k2 ** np.float32(index / 4.0) / k2, np.float32(0.0)).astype(np.float32)
    del k2
    G *= amp
    del amp
    psi = []
    for kc in (kx, ky, kz):
        psi.append(sfft.irfftn(G * (1j * kc), s=(n, n, n), workers=-1).astype(np.float32))
    del G
    sq = psi[0].astype(np.float64) ** 2 + psi[1].astype(np.float64) ** 2 + psi[2].astype(np.float64) ** 2
    rms = math.sqrt(float(sq.mean()))
    del sq
    scale = rms_disp * (box / n) / rms
    q = (np.arange(n, dtype=np.float64) + 0.5) * (box / n)
    pos = np.empty((n * n * n, 3))
    pos[:, 0] = np.repeat(q, n * n) + scale * psi[0].reshape(-1)
    pos[:, 1] = np.tile(np.repeat(q, n), n) + scale * psi[1].reshape(-1)
    pos[:, 2] = np.tile(q, n * n) + scale * psi[2].reshape(-1)
    return _wrap(pos, box)


def zeldovich_clustered(n_side: int, rng, n_halos: int, a_lo: float, a_hi: float,
                        frac: float = 0.5, box: float = 1.0):
    """Zel'dovich-displaced lattice with a fraction of its particles moved into halos."""
    lattice = zeldovich_lattice(n_side, rng, box=box)
    n = lattice.shape[0]
    n_h = int(round(n * frac))
    counts, overflow = halo_counts(rng, n_h, n_halos)
    halos, info = plummer_halos(rng, counts, a_lo, a_hi, box)
    keep = rng.permutation(n)[: n - n_h + overflow]
    keep.sort()
    pos = np.concatenate([lattice[keep], halos])
    del lattice
    pos = pos[rng.permutation(pos.shape[0])]
    info["overflow"] = overflow
    return pos, info


# ---------------------------------------------------------------- batches, cotangents

def batched_boxes(n_boxes: int, rng, n_lo: int = 32 ** 3, n_hi: int = 128 ** 3,
                  nbar_lo: float = 30.0, nbar_hi: float = 60.0, soft_frac: float = 1.0 / 40.0):
    """Independent periodic unit boxes with log-uniform particle counts.

    CPD targets ~45 particles per cell, clamped so that the mean occupancy
    lies in [nbar_lo, nbar_hi] and CPD >= 5; each box is uniform or clustered
    with probability 1/2; eps is 1/40 of the box's mean spacing.
    """
    out = []
    for b in range(n_boxes):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        c = int(round((n / 45.0) ** (1.0 / 3.0)))
        while c > 5 and n / c ** 3 < nbar_lo:
            c -= 1
        while n / c ** 3 > nbar_hi:
            c += 1
        c = max(c, 5)
        kind = "clustered" if rng.random() < 0.5 else "uniform"
        if kind == "clustered":
            k = max(1, int(round(REF_HALOS * n / REF_N)))
            pos, _ = clustered(n, rng, k, 0.5 / c, 3.0 / c)
        else:
            pos = uniform(n, rng)
        spacing = 1.0 / n ** (1.0 / 3.0)
        out.append(Workload(f"box{b}", pos, c, spacing * soft_frac, meta=dict(kind=kind)))
    return out


def cotangent(n: int, rng) -> np.ndarray:
    """Standard-normal cotangent vectors w_i for the adjoint (vector-Jacobian) product."""
    return rng.standard_normal((n, 3))


# ---------------------------------------------------------------- named workloads

def _uniform32k(scale: int = 32):
    rng = rng_for(1)
    n = scale ** 3
    return Workload(f"uniform{scale}^3", uniform(n, rng), 9 if scale == 32 else max(5, round((n / 45) ** (1 / 3))),
                    (1.0 / scale) / 40.0, meta=dict(config=1))


def _clustered(scale: int = 256, cpd: int | None = None, config: int = 2, soft_frac: float = 1.0 / 40.0):
    rng = rng_for(config)
    n = scale ** 3
    if cpd is None:
        cpd = max(5, int(round(125 * scale / 256)))
    n_halos = REF_HALOS if scale == 256 else max(1, int(round(REF_HALOS * n / REF_N)))
    w = 1.0 / cpd
    pos, info = clustered(n, rng, n_halos, 0.5 * w, 3.0 * w)
    return Workload(f"clustered{scale}^3", pos, cpd, (1.0 / scale) * soft_frac,
                    meta=dict(config=config, halos=n_halos, overflow=info["overflow"]))


def _zeldovich(scale: int = 512, cpd: int | None = None):
    rng = rng_for(4)
    if cpd is None:
        cpd = 405 if scale == 512 else max(5, int(round(405 * scale / 512)))
    # halo scale radii are 0.5-3 cell widths of the 256^3 clustered grid
    # (CPD 125), i.e. the same physical halos at 8x the mass resolution
    w_ref = 1.0 / 125.0
    n_halos = REF_HALOS if scale == 512 else max(1, int(round(REF_HALOS * scale ** 3 / 512 ** 3)))
    pos, info = zeldovich_clustered(scale, rng, n_halos, 0.5 * w_ref, 3.0 * w_ref)
    return Workload(f"zeldovich{scale}^3", pos, cpd, (1.0 / scale) / 50.0,
                    meta=dict(config=4, halos=n_halos, overflow=info["overflow"]))


def _clustered64():
    return _clustered(64, cpd=25, config=5)


def _tiles128(cpd: int = 40, per_cell: int = 128):
    """Exactly per_cell particles in every cell, uniform within it (cpd^3 cells): every work
    item is one full 128-sink tile against 125 x 128 sources (a profiling workload)."""
    rng = rng_for(6)
    c = np.repeat(np.arange(cpd ** 3), per_cell)
    base = np.stack([c // (cpd * cpd), (c // cpd) % cpd, c % cpd], 1)
    pos = (base + rng.random(base.shape)) / cpd
    n = pos.shape[0]
    return Workload(f"tiles{per_cell}", pos, cpd, (1.0 / n ** (1.0 / 3.0)) / 40.0, meta=dict(per_cell=per_cell))


def _giantcell():
    """One cell of 200,000 particles (the largest cell late in the paper's run holds over 200,000),
    two dense cells (30,000 and 20,000) at Chebyshev distance 2 from it, and a sparse background of
    4 particles per cell; CPD 12.  Each dense population is a Gaussian clipped to its cell."""
    cpd = 12
    rng = np.random.default_rng(81)
    bg = rng.random((4 * cpd ** 3, 3))

    def blob(cell, n, sigma):
        c = np.asarray(cell, float)
        x = (c + 0.5) / cpd + sigma / cpd * rng.standard_normal((n, 3))
        return np.clip(x, c / cpd + 1e-7, (c + 1) / cpd - 1e-7)
    pos = np.concatenate([bg, blob((3, 3, 3), 200000, 0.2), blob((5, 3, 3), 30000, 0.25),
                          blob((3, 5, 1), 20000, 0.3)])
    return Workload("giantcell", pos, cpd, (1.0 / 100.0) / 40.0, meta=dict(largest_cell=200000))


def _sparse2(cpd: int = 200, per_cell: int = 2):
    """Uniform random particles at per_cell per cell on average (cpd^3 cells): almost every cell
    is sparse, so nearly all work runs as lane items (a profiling workload)."""
    rng = rng_for(7)
    n = per_cell * cpd ** 3
    return Workload(f"sparse{per_cell}", uniform(n, rng), cpd, (1.0 / n ** (1.0 / 3.0)) / 40.0,
                    meta=dict(per_cell=per_cell))


WORKLOADS = {
    "uniform32k": _uniform32k,
    "clustered256": _clustered,
    "zeldovich512": _zeldovich,
    "clustered64": _clustered64,
    "tiles128": _tiles128,
    "sparse2": _sparse2,
    "giantcell": _giantcell,
}


def workload(name: str, **kw) -> Workload:
    """Named workload: uniform32k, clustered256, zeldovich512, clustered64, tiles128, sparse2, giantcell."""
    return WORKLOADS[name](**kw)
