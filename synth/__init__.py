"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side
tests/bench: triangle meshes (vertex coordinates + element-to-vertex lists),
initial-condition functions evaluated at caller-supplied points, and seeded
random field arrays.

This package holds none of the discontinuous Galerkin method's arithmetic:
no nodes, no operators, no flux, no time stepping.  Both the CUDA path and
the oracle receive exactly the arrays produced here.
"""
from .meshes import (  # noqa: F401
    square_grid_mesh,
    jittered_delaunay_mesh,
    relabel_mesh,
    n_for_target_elements,
)
from .fields import (  # noqa: F401
    gaussian_pulse,
    cavity_mode,
    random_fields,
    random_permittivity,
)
