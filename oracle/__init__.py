"""Plain FP64 CPU oracle for SAGE/EM direction-dependent calibration.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library; the only inputs
both sides share come from the seeded generators in
``paper_1910_13908_gb300.synth``.

See ``oracle.sagecal_oracle`` for the functions and what pins each of them.
"""
from .sagecal_oracle import *  # noqa: F401,F403
