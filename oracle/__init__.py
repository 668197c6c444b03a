"""FP64 CPU oracle (test infrastructure only; the product path never imports it)."""
from .lfa_oracle import *  # noqa: F401,F403
