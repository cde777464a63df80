"""FP64 CPU oracle of the IBDL operator (test infrastructure only; see ibdl_oracle)."""
from .ibdl_oracle import *  # noqa: F401,F403
