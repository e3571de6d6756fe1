"""libgcoreccd: GB300 (sm_103a) hole transport of G-CoReCCD (arXiv 2203.11043).

The C ABI is declared in include/gcoreccd.h; ``gcoreccd`` binds it with the
same function names.  ``inputs`` holds the seeded synthetic event generators.
"""
from .gcoreccd import *  # noqa: F401,F403
from .gcoreccd import Simulation, GcError, GcParams, load  # noqa: F401
