"""Seeded synthetic inputs shared by the oracle and the CUDA path (geometry and excitation only)."""
from . import excitation, meshes, workloads  # noqa: F401
