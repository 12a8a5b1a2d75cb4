"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This package holds input generators only (meshes, source fields, coefficient
fields, right-hand-side families).  It contains none of the method's
arithmetic: no quadrature, basis, operator, agglomeration or solver code.
"""
from .meshes import (jittered_square, kuhn_cube, batched_squares, square_with_holes,
                     Mesh, face_neighbors)
from .fields import (sin_source, sin_solution, sine_combination_sources,
                     smoothed_lognormal_kappa)

__all__ = ["jittered_square", "kuhn_cube", "batched_squares", "square_with_holes", "Mesh", "face_neighbors",
           "sin_source", "sin_solution", "sine_combination_sources",
           "smoothed_lognormal_kappa"]
