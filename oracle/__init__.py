"""FP64 CPU oracle (test infrastructure only; see krr_oracle)."""
from .krr_oracle import *  # noqa: F401,F403
