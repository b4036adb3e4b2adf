"""Seeded synthetic array data shared by the oracle tests, the GPU tests and the benchmark.

This package holds the signal model only (plane waves of bandlimited complex-Gaussian
waveforms arriving at an array, plus white sensor noise). It contains none of the
beamspace-transform arithmetic, so both sides of every parity test can use it.
"""
from .planewave import (  # noqa: F401
    ArrayGeometry,
    Source,
    array_positions,
    draw_sources,
    array_record,
    waveform,
    ula_config,
    ura_config,
    uneven_ula_instances,
    interference_config,
    perturbed_geometry,
)
