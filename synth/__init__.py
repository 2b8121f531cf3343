"""Seeded synthetic inputs for the TNEP hot path.

This package holds geometry and random-number recipes only: water boxes,
BaZrO3 supercells, water clusters, open anions, random-walk trajectories,
Poisson arrival times and random model parameters.  It contains none of the
TNEP arithmetic (no descriptor, network, partial force or spectrum), so both
the FP64 oracle and the CUDA path can take their inputs from here without
sharing any of the method's code.
"""

from .workloads import *  # noqa: F401,F403
