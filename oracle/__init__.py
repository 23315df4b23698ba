"""FP64 CPU oracle (test infrastructure only; never used by the product path).

See amto_oracle.py for the equations it follows and the readings it takes.
"""
from .amto_oracle import *  # noqa: F401,F403
