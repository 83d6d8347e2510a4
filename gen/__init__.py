"""Seeded synthetic catalogue generators (shared input side of tests, oracle and bench).

This package only draws random positions, weights and bin edges. It holds none of the
pair-counting arithmetic: no separations, no binning, no periodic wrapping of pairs.
"""
from .catalogs import (  # noqa: F401
    GEN_VERSION,
    Catalogue,
    Workload,
    log_edges,
    uniform_box,
    clustered_box,
    uniform_weights,
    sphere_patch,
    unit_sphere,
    survey_cone,
    workload,
    batch_sizes,
    batch_catalogue,
)
