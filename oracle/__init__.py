"""CPU oracle (test infrastructure only; see lru_oracle.py)."""
from .lru_oracle import *  # noqa: F401,F403
