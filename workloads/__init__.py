"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This package only builds inputs: tetrahedral box grids, boundary data, material
fields, spring targets and random numbers.  It holds none of the PBNG arithmetic
(no deformation gradients, forces, Hessians or colourings); the FP64 oracle under
``oracle/`` and the CUDA library under ``paper_2306_09021_gb300/`` each compute
those from these arrays independently.
"""

from .rng import splitmix64, uniform01, standard_normal
from .grids import box_grid, grid_vertex_id
from .problems import (
    Problem,
    twist_block,
    gravity_sag,
    contact_bar,
    batched_blocks,
    adjoint_block,
    adjoint_load_cases,
    concat_problems,
    two_blocks_hanging,
)

__all__ = [
    "splitmix64",
    "uniform01",
    "standard_normal",
    "box_grid",
    "grid_vertex_id",
    "Problem",
    "twist_block",
    "gravity_sag",
    "contact_bar",
    "batched_blocks",
    "adjoint_block",
    "adjoint_load_cases",
    "concat_problems",
    "two_blocks_hanging",
]
