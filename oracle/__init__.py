"""FP64 CPU oracle (test infrastructure only; see dgf_oracle's docstring)."""
from .dgf_oracle import *  # noqa: F401,F403
