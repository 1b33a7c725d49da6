"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library:
geometry node sets and meshes, grids, initial states, random right-hand sides
and manufactured exact solutions.  No arithmetic of the method lives here."""
from . import geometry, configs  # noqa: F401
