"""GB300-native asynchronous block ILU(0) preconditioning with FGMRES.

The computation lives in libabilu.so (hand-written sm_103a CUDA behind the C
ABI of include/abilu.h); ``abilu`` is its thin Python binding.
"""
from .abilu import (AbiluError, Factors, Pattern, SolveResult, bsr_spmv, default_opts,  # noqa: F401
                    fgmres_solve, kernel_launches, version)
