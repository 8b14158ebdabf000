"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no step of the lensing method: it only draws particle
positions, replica transforms and bundle directions with the shapes of the
paper's workloads (point lens, NFW halo, cosmological boxes, light cones).
Both sides of every parity test receive the same arrays from here.
"""
from .generators import *  # noqa: F401,F403
