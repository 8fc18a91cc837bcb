"""FP64 CPU oracle (test infrastructure only; see gerchberg.py)."""
from .gerchberg import *  # noqa: F401,F403
