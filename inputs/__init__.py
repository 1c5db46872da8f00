"""Seeded synthetic inputs shared by the CPU oracle side and the CUDA side.

This package holds geometry and bookkeeping only: fcc lattice sites cut to a
cylinder, grip-plane labels, ragged batch packing, thermal jitter for static
force tests, and the workload definitions.  It contains none of the TB-SMA
energy, force, integrator or random-number arithmetic; each side implements
that on its own.
"""

from .wires import (  # noqa: F401
    A_LATTICE,
    KIND_MOBILE,
    KIND_GRIP_LEFT,
    KIND_GRIP_RIGHT,
    Wire,
    fcc_wire,
    fcc_ball,
    dimer,
    trimer,
    jitter,
    pack,
    Batch,
)
from .configs import WORKLOADS, workload, WireSpec  # noqa: F401
