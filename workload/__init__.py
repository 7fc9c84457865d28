"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This package draws geometries, basis exponents and request streams.  It holds
none of the method's arithmetic: no normalisation, no integrals, no linear
algebra.  Everything it returns is plain data (lists and numpy arrays).
"""
from .water import (  # noqa: F401
    ANGSTROM_TO_BOHR,
    Molecule,
    Shell,
    single_water,
    water_cluster,
    cluster_basis_rules,
    single_water_basis_rules,
    expand_basis,
    serving_stream,
    molecule_for,
)
