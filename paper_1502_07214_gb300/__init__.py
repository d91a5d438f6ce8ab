"""GB300 library for the parallel multicanonical simulation of the 3D
Blume-Capel model (hot path: typewriter Metropolis sweeps of many walkers
under a shared weight, histogram merge, FP64 weight update and acceptance
table, time-series reweighting).

``muca`` is the ctypes binding of ``libmuca.so``; ``workloads`` holds the
seeded synthetic-input generators.  Importing the package loads nothing.
"""
__all__ = ["muca", "workloads", "build"]
