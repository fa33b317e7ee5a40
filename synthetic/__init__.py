"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package only builds inputs: point clouds, neighbour lists, physical fields and
species tables. It contains none of the radiative-transfer method's arithmetic (no
directions, quadrature, line profiles, transfer solves or level populations); each side
computes those itself.
"""
from .models import (  # noqa: F401
    Model, Species, CODATA,
    species_two_level, species_rotor, species_ladder,
    model_sphere_1d, model_clumpy_3d, model_disc, model_line_1d, model_tiny_3d,
    model_lattice_3d, model_batch, hubble_line_1d, hubble_sphere_1d, powerlaw_line_1d,
    knn_symmetric, shell_counts, shells_3d, hubble_shells_3d, vz_problem1,
)
