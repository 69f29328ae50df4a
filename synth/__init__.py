"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

Holds field generators and workload recipes only; no part of the isosurface
method lives here.
"""
from . import fields, recipes  # noqa: F401
