"""Seeded synthetic inputs (meshes, frequency-set parameters, densities).

Shared by the CPU oracle and the CUDA path; contains no boundary element
arithmetic.
"""
from . import meshes, workloads  # noqa: F401
