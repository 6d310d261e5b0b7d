"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This package holds no arithmetic of the projection method itself: it draws
Zel'dovich particle lattices (test tooling standing in for the paper's
simulation snapshots, which are not available) and builds camera descriptions.
"""
from .zeldovich import ZeldovichField, zeldovich_positions, fp16_offsets, decode_fp16_offsets  # noqa: F401
from .cameras import ortho_z, sphere_cameras, camera_dict  # noqa: F401
from .configs import CONFIGS, config  # noqa: F401
