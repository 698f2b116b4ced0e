"""CPU oracle (test infrastructure only; see moma_oracle.py's header)."""
from .moma_oracle import *  # noqa: F401,F403
