"""FP64 CPU oracle for approximate-ADMM semidefinite programming.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the product path.  It
shares no code with the CUDA library.  See oracle/sdp_oracle.c for what each
routine computes and which part of the paper it follows.
"""
from .oracle import *  # noqa: F401,F403
