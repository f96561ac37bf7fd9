"""Seeded synthetic inputs for the AMG-DD solve phase.

This package is the one module shared by the CUDA library's callers and by the
CPU oracle. It holds the problem definitions only (finite-difference diffusion
matrices, box partitions of the unknowns, seeded right-hand sides and
coefficient fields) and none of the method's arithmetic: no hierarchy, no
smoother, no cycle.

The paper's test problems (Section 6: linear finite elements from MFEM on METIS
partitions) are not available; the finite-difference stencils below stand in
for them, with box subdomains standing in for the METIS partition.
"""
from .generators import (  # noqa: F401
    poisson2d, poisson3d, diffusion3d, checkerboard_kappa, box_partition,
    uniform_rhs, grid_shape_of, workload, WORKLOADS, gaussian_random_field, lognormal_kappa,
    batched_poisson, rotated_anisotropic2d, weak_link_chain,
)
