"""FP64 CPU oracle for multi-reference alignment (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may use
this package; the CUDA library never calls it.
"""
from .mra_oracle import *  # noqa: F401,F403
from .mra_oracle import __all__  # noqa: F401
