"""Shared helpers of the GPU tests: the library box from a workload, and the
oracle's side of the same input.  Both sides start from the same seeded
global positions; each does its own binning."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

# Error contract of the FP32 path against the FP64 oracle.
RMS_TOL = 1e-6            # rms relative force error, compensated accumulation
RMS_TOL_PLAIN = 1e-5      # plain FP32 running sums (reported next to the compensated kernel)
STAGE = 128               # sources per accumulation block of the default launch shape
# |da_i| <= (B + 64) 2^-24 sum_j |F_ij|: B-term FP32 block sums, ~10 roundings per
# pair in the Newtonian branch and up to ~31 ulps of cancellation in the spline polynomial
BOUND_K = STAGE + 64


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_box(X, cpd, eps, box=1.0, mode=None):
    import paper_1810_02916_b300 as nfb
    nf = nfb.NearField(cpd, eps, box)
    if mode is not None:
        nf.set_accumulation(mode)
    nf.bin_particles(np.ascontiguousarray(X, dtype=np.float64))
    return nf


def oracle_side(X, cpd, box=1.0):
    return oracle.bin_positions(np.asarray(X, dtype=np.float64), cpd, box)


def sample_sinks(b: oracle.Binned, k: int, seed: int = 0) -> np.ndarray:
    """k storage indices: half uniform over particles, half from the densest cells."""
    rng = np.random.default_rng(seed)
    n = b.n
    if n <= k:
        return np.arange(n, dtype=np.int64)
    uni = rng.choice(n, k // 2, replace=False)
    dense_cells = np.argsort(b.counts)[::-1][:8]
    pool = np.concatenate([np.arange(b.offsets[c], b.offsets[c + 1]) for c in dense_cells])
    den = rng.choice(pool, min(k - k // 2, pool.size), replace=False)
    return np.unique(np.concatenate([uni, den])).astype(np.int64)
