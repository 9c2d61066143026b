"""FP64 CPU oracle (test infrastructure): see oracle.py and memsynth_oracle.c."""
from .oracle import *  # noqa: F401,F403
from .oracle import build, forward, forward_gridded, mosaic_forward, adjoint, dirty_image, beam_fit, Problem  # noqa: F401
