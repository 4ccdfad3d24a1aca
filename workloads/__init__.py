"""Seeded synthetic inputs shared by the oracle, the CUDA path, the tests and
the benchmark: icosphere bead meshes, swimmer placements and random states.
Holds no arithmetic of the time step itself."""
from .mesh import icosphere, icosahedron, edges_of  # noqa: F401
from .configs import (  # noqa: F401
    SwimmerSpec, BoxSpec, assemble, single_swimmer_48, swimmer_pair, pair_boxes_256x128x128,
    pair_side_256cube, paper_box_1024x256x256, paper_study_box, PAPER_L_SWIM, adjoint_single_96, adjoint_small, balanced_drive, free_drive, fluid_box, random_populations, perturbed_nodes, PAIR_CASES,
    ensemble_boxes, ENSEMBLE_SIZES,
)
