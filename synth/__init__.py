"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds random draws and shape bookkeeping only. It performs none of the
Tensor-Train arithmetic (no contractions, no sweeps, no decompositions), so that the
FP64 oracle and the CUDA path share nothing but their input bytes.
"""
from .tt_inputs import *  # noqa: F401,F403
