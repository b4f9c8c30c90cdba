"""FP64 CPU oracle (test infrastructure only; see scd_oracle.py)."""
from .scd_oracle import *  # noqa: F401,F403
