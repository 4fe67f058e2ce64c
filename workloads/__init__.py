"""Seeded synthetic problem definitions shared by the oracle tests, the GPU
parity tests and the benchmark.

This package only defines *problems*: coefficient fields, sources, boundary
data and closed-form solutions, as functions of point coordinates.  It holds
none of the solver's arithmetic (no spectral operators, no eliminations), so
both the CPU oracle and the CUDA path can take their inputs from here without
sharing any part of the method.

Every random draw uses ``numpy.random.default_rng(seed)`` and the seed is part
of each problem's description.
"""

from .problems import (  # noqa: F401
    Problem,
    poisson_poly_2d,
    helmholtz_bumps_2d,
    elliptic_3d,
    elliptic_2d,
    e1_dtn_2d,
    e2_iti_2d,
    e7_wavefront_3d,
    polynomial_field,
    poly_varcoef,
    sharp_source_3d,
    adaptive_3d,
    grid_interp_matrix,
    helmholtz_theta_2d,
)
