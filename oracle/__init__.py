"""FP64 CPU oracle for depth-p QAOA on NAE-k-SAT.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may use it; the product path never does.  It shares no code with the
CUDA library.  See ``oracle.c`` for the conventions and citations.
"""
from .oracle import (  # noqa: F401
    build,
    cost_samples,
    cost_table,
    count_solutions,
    evolve,
    grad,
    library_path,
    running_time,
    sample,
    success_prob,
)
