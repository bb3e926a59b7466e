"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package only generates inputs: grids, material maps, source waveforms and
masks.  It holds none of the simulation or fitting arithmetic, so both the CUDA
path and the CPU oracle can draw the same inputs from it without sharing code.
"""
from .media import (  # noqa: F401
    gaussian_pulse,
    plane_amplitude_rate,
    voronoi_classes,
    voronoi_medium,
    two_layer_medium,
    homogeneous_medium,
    line_source_mask,
    config_c1,
    config_c2,
    config_c3,
    config_c5,
    serving_stream,
    WorkloadSpec,
)
