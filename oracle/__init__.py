"""FP64 CPU oracle for GFC and its editing steps -- test infrastructure only (see gfc_oracle.py)."""
from .gfc_oracle import *  # noqa: F401,F403
from .gfc_edit_oracle import *  # noqa: F401,F403
from .gfc_edit_oracle import color_correct_with  # noqa: F401
