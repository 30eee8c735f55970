"""FP64 CPU oracle for the CGL exponential integrators (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  The CUDA library never does.
"""
from .cgl_oracle import *  # noqa: F401,F403
from .cgl_oracle import (OracleProblem, LinearOperator, integrate, rel_l2,  # noqa: F401
                         rel_inf, observed_order, SCHEMES, ORDERS)
