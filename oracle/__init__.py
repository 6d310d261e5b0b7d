"""FP64 CPU oracle for the tetrahedral column-density projection.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py. The product package never imports it, and it
imports nothing from the product package.
"""
from .oracle import (  # noqa: F401
    Camera,
    render,
    render_crops,
    tet_volumes,
    gradient,
    frame_mass,
    chord,
    tet_vertices,
    render_soup,
    resample,
    point_density,
    centroids,
    hybrid,
    render_area,
)
