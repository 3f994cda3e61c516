"""Seeded synthetic TPC events and time frames (input generator only).

This module simulates charged-particle helices in a uniform solenoidal field
and records where they cross the pad-row planes of the 36 trapezoidal TPC
sectors (Sec. 2 of the paper: 36 sectors, 152 pad rows). It produces the
inputs that both the CUDA path and the CPU oracle consume; it contains none
of the reconstruction arithmetic (no track propagation in local frames, no
Kalman filter, no cellular automaton). Helices are intersected with the row
planes in the *global* frame with a closed-form circle/line intersection, and
the injected space-charge distortion is evaluated with scipy's tensor-product
B-spline, so the generator is an implementation independent of both.
"""
from .events import (  # noqa: F401
    Geometry, Calib, Event, geometry, nominal_calib,
    gen_particles_single_sector, gen_particles_central, make_event,
    make_single_sector, make_central, make_timeframe, make_batched,
    make_adjoint, make_tiny, random_distortion, truth_tracks, pad_positions, sector_alpha,
    CONFIGS, make_config,
)
