"""FP64 CPU oracle for GFC -- test infrastructure only (see gfc_oracle.py)."""
from .gfc_oracle import *  # noqa: F401,F403
