"""CPU FP64 oracle (test infrastructure only; see ``ssa_oracle``)."""
from .ssa_oracle import *  # noqa: F401,F403
