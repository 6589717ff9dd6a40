"""Seeded synthetic inputs for the robust eigenvector path.

This package only draws random numbers and places them into matrices of the
shapes the method consumes (real Schur forms, generalized Schur pairs,
orthogonal factors, selection masks, batches of uneven sizes, chains of
reordering windows with random orthogonal accumulators).  It holds none
of the method's arithmetic, and both the CUDA path and the CPU oracle read
their inputs from here.
"""
from .schur_inputs import (  # noqa: F401
    SEED_BASE,
    adversarial_schur,
    batch_inputs,
    batch_pencils,
    batch_sizes,
    block_selection,
    config0_schur,
    generalized_pair,
    householder_orthogonal,
    random_eigen_selection,
    solve_system,
    window_chain,
)
