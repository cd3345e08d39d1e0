"""GB300 (sm_103a) library for the explicit cell-centred finite-volume step of
the 2D Euler equations on triangles with the Lax-Friedrichs flux (Nagy et al.,
Sec. 6).  The compute path is the CUDA library behind ``include/fv.h``;
``binding`` marshals arguments to it and ``workloads`` makes seeded inputs.

Importing the package does not load the CUDA library; ``binding.load()`` (or
constructing a ``Mesh``) does, and raises if it has not been built.
"""
__all__ = ["binding", "workloads", "build"]
