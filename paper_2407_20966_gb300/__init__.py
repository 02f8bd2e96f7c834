"""GB300-native kinetic-bounds limiter for high-order DG/FR Euler (arXiv 2407.20966).

The compute path is the C-ABI library ``libkbl.so`` (hand-written CUDA for
sm_103a, declared in ``include/kbl.h``); ``paper_2407_20966_gb300.kbl`` is a thin
ctypes binding with the same names.  ``inputs`` holds the seeded synthetic
problem set-ups.  Importing the package does not load the library; the first
call through ``kbl`` does, and raises if it is missing.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs"]
