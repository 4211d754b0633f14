"""CPU FP64 oracle (test infrastructure; see reach_oracle)."""
from .reach_oracle import *  # noqa: F401,F403
from .reach_oracle import S0, S1, SQ, PROB01, PROB0_ONLY  # noqa: F401
