"""Seeded synthetic inputs shaped like the paper's DECam workloads (Section 2.1, Section 4.1).

This module only draws inputs: it holds none of the search's arithmetic (no likelihood images,
no track rounding of the search, no clipping).  Both the CUDA path's tests/bench and the oracle
read the arrays it returns.
"""
from .stacks import *  # noqa: F401,F403
