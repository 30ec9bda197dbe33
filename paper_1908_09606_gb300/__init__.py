"""I/O-aware single-GPU matrix multiplication for GB300 (sm_103a), after COSMA
(Kwasniewski et al., SC'19).  The compute path is the C-ABI library in
csrc/ (declared in include/cosma.h); `cosma` is its ctypes binding."""

from . import cosma  # noqa: F401
from .cosma import gemm, gemm_grouped, load  # noqa: F401
