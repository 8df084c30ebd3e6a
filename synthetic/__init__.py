"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds input recipes only (initial states, diffusivity fields,
delay schedules, problem sizes).  It contains none of the Parareal method's
arithmetic: no propagator, no correction, no norm.  Both sides import it; it
imports neither side.
"""
from .generators import (  # noqa: F401
    sine_modes_1d,
    modes_and_bumps_2d,
    smoothed_noise_3d,
    gaussian_random_field,
    lognormal_kappa,
    delay_table,
    random_directions,
)
from .configs import preset, PRESETS  # noqa: F401
