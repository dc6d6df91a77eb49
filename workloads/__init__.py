"""Seeded, synthetic inputs shared by the oracle, the CUDA path and the benchmark.

This package only *builds inputs*: phase-space meshes, WKB initial data and the
packet sets that sample it, plus seeded random packet sets for unit tests.  It
holds none of the hot path's arithmetic (no trajectory integration, no direct
sum, no least-squares correction), so neither side of a parity test can share a
mistake through it.

The one piece of the paper's method in here is the initial decomposition
(Step 1 of Algorithm 1, eq. 2.6 and 2.8), which turns the WKB data into packet
amplitudes.  It sits before the hot path; neither the oracle nor the CUDA
library implements it.
"""

from .wkb import (  # noqa: F401
    Mesh, WKB_TANH, WKB_LINEAR, config_workload, wkb_packets, mesh_for,
    random_packets, CONFIGS, mesh_axes, workload_axes,
)
