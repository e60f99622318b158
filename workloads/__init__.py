"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds no arithmetic of the correlation method itself (see ``speckle``).
"""
from .speckle import Affine, Pair, Rigid, Sinusoidal, quantise, render_pair  # noqa: F401
from . import configs, swarm  # noqa: F401
