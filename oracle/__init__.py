"""FP64 CPU oracle for the randomized PCA (test infrastructure only; see rpca_oracle)."""
from .rpca_oracle import *  # noqa: F401,F403
from . import learned_oracle  # noqa: F401
