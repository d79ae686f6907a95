"""GB300-native reciprocal-space Smooth Particle Mesh Ewald (SPME).

The compute path is the CUDA library ``libpme_gb300.so`` (C ABI in include/pme.h); ``pme`` is its thin
ctypes binding and ``workloads`` holds the seeded synthetic input generators.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "pme"]
