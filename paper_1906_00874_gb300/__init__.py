"""GB300-native H-LU: LU factorisation of hierarchical (H-) matrices from boundary
element methods, as a task graph of hand-written sm_103a CUDA kernels behind a
C ABI (include/hlu.h).  This package holds the CUDA sources (csrc/), the build
step (build.py) and the ctypes binding (hlu.py)."""
from .hlu import HLU, HLUError, HLU_FP32, HLU_FP32_CORE32, HLU_FP64, load  # noqa: F401
