"""GB300-native TNEP tensors (arXiv 2312.05233): dipole and polarizability
models evaluated by hand-written sm_103a CUDA kernels behind a C ABI.

The binding loads ``libtnep.so`` (built in-tree by ``build.build()``); there is
no CPU fallback.
"""

from .tnep import *  # noqa: F401,F403
from .tnep import Context, Model, TnepError, lib  # noqa: F401
