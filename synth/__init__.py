"""Seeded synthetic workloads shaped like stabilised-video PRNU matching.

This package only draws random numbers and synthesises input frames: it holds
none of the detector's arithmetic (no residual, no correlation, no PCE, no
inverse warp).  Both the FP64 oracle and the CUDA path consume what it makes.
"""
from .generate import *  # noqa: F401,F403
