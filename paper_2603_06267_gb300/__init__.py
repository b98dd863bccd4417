"""GB300-native explicit DG-SEM acoustic step with batched reduced-order PMUT
coupling (arXiv 2603.06267): CUDA kernels for sm_103a behind the C ABI of
include/dgsem.h, with a thin ctypes binding (dgsem.py)."""
from . import dgsem  # noqa: F401
