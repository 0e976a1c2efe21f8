"""Seeded synthetic inputs shaped like the GMRT software backend's workloads.

This package holds input generation only -- none of the correlator's own
arithmetic -- and is the one module shared by the oracle tests, the GPU
parity tests and the benchmark.
"""
from .streams import (  # noqa: F401
    CONFIGS,
    StreamSet,
    make_config,
    make_streams,
    uniform_params,
)
