"""GB300-native ball-harmonic rotational matching (expansion + marching gradient ascent over SO(3)).

The compute path is the C-ABI library ``libbh.so`` (hand-written CUDA for sm_103a); ``bh`` is its thin
Python binding and ``synth`` the seeded synthetic-workload generator.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "bh", "build"]
