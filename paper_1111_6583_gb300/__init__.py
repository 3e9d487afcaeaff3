"""GB300-native finite-volume step of Clawpack-classic and SharpClaw.

The compute path is the C-ABI library ``libclawgpu.so`` (hand-written CUDA for
sm_103a, declared in ``include/clawgpu.h``); ``claw`` is the thin ctypes
binding with the same names.  ``workloads`` holds the seeded synthetic inputs.

Importing the package does not load the CUDA library; ``claw`` loads it on
first use and raises if it is missing.
"""
__all__ = ["claw", "workloads"]
