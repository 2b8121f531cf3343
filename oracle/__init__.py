"""FP64 CPU oracle for the TNEP tensor path (test infrastructure only).

Imported by tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline
and reference legs; never by the product package.
"""
from .tnep_oracle import *  # noqa: F401,F403
from .snes_oracle import *  # noqa: F401,F403
from .raman_oracle import *  # noqa: F401,F403
