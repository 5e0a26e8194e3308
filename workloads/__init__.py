"""Seeded synthetic inputs for the semi-explicit eddy-current hot path.

This package only describes problems: grid size, spacing, per-cell conductivity
and nonlinear-material flags, coil geometry and waveform, and seeded random
vectors.  It holds none of the method's arithmetic (no incidence matrices, no
material averaging, no solver), so the FP64 oracle and the CUDA path can both
read the same inputs without sharing any computation.
"""
from .problems import (  # noqa: F401
    NU0, BRAUER_STEEL, Problem, config_linear_block, config_nonlinear_iron,
    scaled_nonlinear, random_problem, power_start_vector, random_vector,
    batched_instances,
)
