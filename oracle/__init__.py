"""FP64 CPU oracle for the CRKSPH neighbor-sum path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  The product path (the CUDA library and its binding)
never does.  See ``crk_oracle.cpp`` for what is computed and where in the paper
each step comes from.
"""
from .oracle import (  # noqa: F401
    OracleParams, build, count_ops, count_pairs, default_params, forward, forward_species, forward_state, jvp, neighbors, kernel, num_threads,
    PARITY_UNPINNED,
)
from . import integrate  # noqa: F401,E402
