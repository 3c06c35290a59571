"""Seeded synthetic particle sets for the near-field force workloads.

This package only draws particle positions (and the random cotangents used by
the adjoint tests).  It holds none of the near-field method's arithmetic: no
cell binning, no quantisation, no force law.  Both the FP64 oracle and the
CUDA library consume its output, so it is the one module they share.
"""
from .generators import (  # noqa: F401
    Workload,
    uniform,
    plummer_halos,
    clustered,
    zeldovich_lattice,
    zeldovich_clustered,
    batched_boxes,
    cotangent,
    workload,
    WORKLOADS,
)
