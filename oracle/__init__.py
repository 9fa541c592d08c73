"""FP64 CPU oracle (test infrastructure only; never imported by the CUDA library)."""
from .optics import *  # noqa: F401,F403
from .optics import AS, FRESNEL_TF  # noqa: F401
