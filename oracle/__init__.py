"""FP64 CPU oracle for stochastic matrix-free equilibration.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
bench's CPU-baseline leg, never by the product path.  It shares no code with
the CUDA library; the two meet only through the seeded input generators and
the published Philox definition that each side implements on its own.
"""
from .oracle import *  # noqa: F401,F403
from . import ccp, mlp  # noqa: F401
