"""Seeded synthetic workloads shared by the oracle tests, the CUDA-path tests and bench.py.

Holds no arithmetic of the method (see ``workloads.heat``).
"""
from . import heat  # noqa: F401
