"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds meshes, materials, fiber fields, pins and activation
sequences. It holds none of the solver's arithmetic: no deformation
gradients, energies, volumes or solves. Tet orientation is fixed
combinatorially (from the parity of the Kuhn permutation), not by evaluating
determinants.
"""
from .meshes import (  # noqa: F401
    MeshSpec,
    kuhn_grid,
    box_beam,
    muscle_tendon_unit,
    mtu_for_tet_count,
    batch_set,
    request_stream,
    single_tet,
    arm_assembly,
    gravity_forces,
    MUSCLE,
    TENDON,
    BONE,
)
