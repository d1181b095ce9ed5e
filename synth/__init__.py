"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only *describes* inputs: unit template meshes for the analytic
primitives, convex hulls of random point sets, rigid poses and per-pair
parameters.  It contains none of the contact-manifold arithmetic (no SDF, no
witness-point solve, no reduction): that lives, written twice and
independently, in ``oracle/`` (FP64 CPU) and in the CUDA library.
"""

from .geometry import (  # noqa: F401
    KIND_BOX, KIND_CAPSULE, KIND_CYLINDER, KIND_ELLIPSOID, KIND_HULL, KIND_SQ_UNION, KIND_NAMES,
    Geometry, box_template, cylinder_template, capsule_template,
    icosphere_template, hull_from_points, primitive_geometry, support, support_point, interior_point,
    superellipsoid_surface, sq_union_geometry,
)
from .workloads import (  # noqa: F401
    Workload, random_quaternions, config_box_box, config_hull_vs_primitive,
    config_box_vs_sphere_hull, config_hull_vs_hull, config_mixed, config_mixed_pooled, serving_trace,
    make_config,
    SQ_RESOLUTIONS, random_sq_union, config_sq_union,
    SEED_BASE, PRIMITIVE_KINDS,
)
