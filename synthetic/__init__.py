"""Seeded synthetic inputs (marker geometries, rigid velocities, problem sizes)
shared by the oracle-based tests and by the GPU path's tests and benchmark.

This package holds geometry and random draws only -- none of the method's
arithmetic (no kernel, no operator, no solve).
"""
from .workloads import *  # noqa: F401,F403
