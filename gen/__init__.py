"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the density-fitting method itself: it only draws
geometries and lists basis exponents.  Both the CPU oracle and the CUDA path consume
what it produces; neither side imports the other.
"""
from .molecules import (  # noqa: F401
    Molecule,
    ORB_EXPONENTS,
    AUX_EXPONENTS,
    even_tempered,
    make_geometry,
    make_molecule,
    molecule_from_geometry,
    config_c0,
    config_c1,
    batch_sizes,
    batch_molecules,
)
