"""FP64 CPU oracle of the FIP-TOI hot path: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package.  The product never does.
"""
from . import toi_oracle  # noqa: F401
