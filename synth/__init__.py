"""Seeded synthetic 4D-STEM inputs shared by the tests, the benchmark and the oracle checks.

This package simulates acquisitions (the forward model of Eq. 1 with the Poisson dose model of
Sect. 8) and nothing else: it holds none of the reconstruction arithmetic, so that the CUDA path
and the CPU oracle can both consume its arrays without sharing any of the method's code.
"""
from .generator import (  # noqa: F401
    Acquisition,
    CONFIGS,
    config,
    object_phase,
    object_transfer,
    probe_fourier_grid,
    probe_real,
    frames,
    all_frames,
    raster_indices,
    serving_mix,
    serving_arrivals,
    SERVING_SIZES,
)
